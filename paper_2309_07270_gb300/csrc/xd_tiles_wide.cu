// Width-512 band tile (second fallback, and the cell-counting pass), the
// unbounded tier, validation and binning.
#include "xd_launch.h"
#include "xd_misc_kernels.cuh"
#include "xd_serve.h"

namespace xd {

cudaError_t launch_spill_512(bool count, int grid, const Job *jp, Spill in, Spill out,
                             cudaStream_t s)
{
    (void)cudaGetLastError();
    if (count) window_spill_kernel<32, 16, true><<<grid, 256, 0, s>>>(jp, in, out);
    else window_spill_kernel<32, 16, false><<<grid, 256, 0, s>>>(jp, in, out);
    return cudaGetLastError();
}

cudaError_t launch_window_count(const Job *jp, uint32_t task_base, uint32_t n_tasks, Spill sp,
                                cudaStream_t s)
{
    const uint64_t threads = (uint64_t)n_tasks * 32;
    const unsigned grid = (unsigned)((threads + 255) / 256);
    if (grid == 0) return cudaSuccess;
    (void)cudaGetLastError();
    window_kernel<32, 16, true><<<grid, 256, 0, s>>>(jp, task_base, n_tasks, sp);
    return cudaGetLastError();
}

cudaError_t launch_wide(bool count, int grid, const Job *jp, Spill in, int32_t *scratch,
                        int64_t scratch_per_cta, cudaStream_t s)
{
    (void)cudaGetLastError();
    if (count) wide_kernel<true><<<grid, WIDE_THREADS, 0, s>>>(jp, in, scratch, scratch_per_cta);
    else wide_kernel<false><<<grid, WIDE_THREADS, 0, s>>>(jp, in, scratch, scratch_per_cta);
    return cudaGetLastError();
}

cudaError_t launch_validate(const Job *jp, uint64_t n_pairs, uint32_t *n_bad, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    uint64_t blocks = (n_pairs + 255) / 256;
    unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
    (void)cudaGetLastError();
    validate_kernel<<<grid, 256, 0, s>>>(jp, n_bad);
    return cudaGetLastError();
}

cudaError_t launch_binning(const Job *jp, uint64_t n_pairs, int grid, uint32_t *hist,
                           uint32_t *offs, uint32_t *n_valid, uint32_t *order, cudaStream_t s)
{
    (void)n_pairs;
    (void)cudaGetLastError();
    bin_count_kernel<<<grid, BIN_THREADS, 0, s>>>(jp, hist);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bin_scan_kernel<<<1, 32, 0, s>>>(hist, offs, n_valid);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bin_scatter_kernel<<<grid, BIN_THREADS, 0, s>>>(jp, offs, order);
    return cudaGetLastError();
}

cudaError_t launch_length_hist(const Job *jp, int grid, uint32_t *hist, cudaStream_t s)
{
    (void)cudaGetLastError();
    bin_count_kernel<<<grid, BIN_THREADS, 0, s>>>(jp, hist);
    return cudaGetLastError();
}

cudaError_t launch_sample_pairs(const Pair *src, uint64_t n, uint32_t stride, uint32_t seed,
                                Pair *dst, uint64_t m, cudaStream_t s)
{
    if (!m) return cudaSuccess;
    (void)cudaGetLastError();
    const uint64_t blocks = (m + 255) / 256;
    sample_pairs_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, n, stride,
                                                                                seed, dst, m);
    return cudaGetLastError();
}

cudaError_t launch_plain_setup(uint64_t n_pairs, uint64_t sub_pairs, uint32_t *order, uint32_t *ctl,
                              cudaStream_t s)
{
    if (!n_pairs) return cudaSuccess;
    (void)cudaGetLastError();
    const uint64_t blocks = (2 * n_pairs + 255) / 256;
    plain_setup_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(n_pairs, sub_pairs,
                                                                               order, ctl);
    return cudaGetLastError();
}

cudaError_t launch_revcomp(const uint32_t *pk, int64_t n_words, const uint64_t *read_off,
                           const uint32_t *read_len, uint32_t n_reads, uint32_t *out,
                           cudaStream_t s)
{
    if (!n_reads) return cudaSuccess;
    (void)cudaGetLastError();
    const unsigned grid = n_reads < 4096u ? n_reads : 4096u;
    revcomp_kernel<<<grid, 128, 0, s>>>(pk, n_words, read_off, read_len, n_reads, out);
    return cudaGetLastError();
}

cudaError_t launch_best_seeds(const Pair *pairs, const int32_t *results, uint64_t n, int32_t match,
                              uint32_t *best, cudaStream_t s)
{
    if (!n) return cudaSuccess;
    (void)cudaGetLastError();
    const uint64_t blocks = (n + 255) / 256;
    best_seeds_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(pairs, results, n,
                                                                             match, best);
    return cudaGetLastError();
}

cudaError_t launch_max_len(const uint32_t *read_len, uint32_t n_reads, uint32_t *out,
                           cudaStream_t s)
{
    if (n_reads == 0) return cudaSuccess;
    unsigned grid = (n_reads + 255) / 256;
    if (grid > 1024) grid = 1024;
    (void)cudaGetLastError();
    max_len_kernel<<<grid, 256, 0, s>>>(read_len, n_reads, out);
    return cudaGetLastError();
}

// ---- dispatch over the tile families ----
cudaError_t launch_persistent_narrow(Tile, int, const Job *, const uint32_t *, const uint32_t *,
                                     uint32_t *, Spill, cudaStream_t, bool *);
cudaError_t launch_persistent_mid(Tile, int, const Job *, const uint32_t *, const uint32_t *,
                                  uint32_t *, Spill, cudaStream_t, bool *);
int occupancy_narrow(Tile);
int occupancy_mid(Tile);
cudaError_t launch_persistent_packed(Tile, int, const Job *, const uint32_t *, const uint32_t *,
                                     uint32_t *, Spill, cudaStream_t, bool *);
int occupancy_packed(Tile);
cudaError_t launch_serve_packed(Tile, int, const ServeArgs &, const uint32_t *, int64_t,
                                cudaStream_t, bool *);
int serve_occupancy_packed(Tile);
cudaError_t launch_spill_mid(int, const Job *, Spill, Spill, cudaStream_t);

cudaError_t launch_serve_narrow(Tile, int, const ServeArgs &, const uint32_t *, int64_t,
                                cudaStream_t, bool *);
cudaError_t launch_serve_mid(Tile, int, const ServeArgs &, const uint32_t *, int64_t, cudaStream_t,
                             bool *);
int serve_occupancy_narrow(Tile);
int serve_occupancy_mid(Tile);

cudaError_t launch_serve(Tile t, int grid, const ServeArgs &a, const uint32_t *pk, int64_t nw,
                         cudaStream_t s)
{
    bool handled = false;
    if (t.packed) {
        cudaError_t e = launch_serve_packed(t, grid, a, pk, nw, s, &handled);
        return handled ? e : cudaErrorInvalidValue;
    }
    cudaError_t e = launch_serve_narrow(t, grid, a, pk, nw, s, &handled);
    if (handled) return e;
    e = launch_serve_mid(t, grid, a, pk, nw, s, &handled);
    if (handled) return e;
    return cudaErrorInvalidValue;
}

int serve_blocks_per_sm(Tile t)
{
    if (t.packed) return serve_occupancy_packed(t);
    int b = serve_occupancy_narrow(t);
    if (b < 0) b = serve_occupancy_mid(t);
    return b;
}

const Tile kTiles[N_TILES] = {{4, 16}, {8, 8}, {16, 4}, {8, 16}, {16, 8}, {32, 4}, {32, 16}};

bool tile_supported(Tile t, bool persistent)
{
    if (!persistent) return !t.packed && t.lanes == 32 && t.c == 16;
    return persistent_blocks_per_sm(t) >= 0;
}

cudaError_t launch_window(Tile t, bool count, const Job *jp, uint32_t task_base,
                          uint32_t n_tasks, Spill spill, cudaStream_t s)
{
    (void)t;
    if (count) return launch_window_count(jp, task_base, n_tasks, spill, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_persistent(Tile t, int grid, const Job *jp, const uint32_t *order,
                              const uint32_t *n_tasks, uint32_t *counter, Spill spill,
                              cudaStream_t s)
{
    bool handled = false;
    if (t.packed) {
        cudaError_t e = launch_persistent_packed(t, grid, jp, order, n_tasks, counter, spill, s,
                                                 &handled);
        return handled ? e : cudaErrorInvalidValue;
    }
    cudaError_t e = launch_persistent_narrow(t, grid, jp, order, n_tasks, counter, spill, s,
                                             &handled);
    if (handled) return e;
    e = launch_persistent_mid(t, grid, jp, order, n_tasks, counter, spill, s, &handled);
    if (handled) return e;
    return cudaErrorInvalidValue;
}

int persistent_blocks_per_sm(Tile t)
{
    if (t.packed) return occupancy_packed(t);
    int b = occupancy_narrow(t);
    if (b < 0) b = occupancy_mid(t);
    return b;
}

cudaError_t launch_spill(Tile t, bool count, int grid, const Job *jp, Spill in, Spill out,
                         cudaStream_t s)
{
    if (t.lanes == 32 && t.c == 16) return launch_spill_512(count, grid, jp, in, out, s);
    if (!count && t.lanes == 32 && t.c == 4) return launch_spill_mid(grid, jp, in, out, s);
    return cudaErrorInvalidValue;
}

}  // namespace xd
