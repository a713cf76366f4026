// Host-side launchers of the device kernels (one translation unit per tile
// family, so the library builds in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "xd_types.cuh"

namespace xd {

struct Tile {
    int lanes;            // lanes per extension (4, 8, 16 or 32)
    int c;                // cells per lane per diagonal
    bool packed = false;  // 16-bit cells, two per register (xd_lockstep16.cuh)
    int width() const { return lanes * c; }
    bool same(const Tile &o) const { return lanes == o.lanes && c == o.c && packed == o.packed; }
};

// Band tiles the library is built with, narrowest first.
constexpr int N_TILES = 7;
extern const Tile kTiles[N_TILES];

bool tile_supported(Tile t, bool persistent);

// One task per group, tasks [task_base, task_base + n_tasks).
cudaError_t launch_window(Tile t, bool count, const Job *jp, uint32_t task_base,
                          uint32_t n_tasks, Spill spill, cudaStream_t s);
// Persistent: positions of `order` pulled from *counter up to *n_tasks.
cudaError_t launch_persistent(Tile t, int grid, const Job *jp, const uint32_t *order,
                              const uint32_t *n_tasks, uint32_t *counter, Spill spill,
                              cudaStream_t s);
// Tasks listed in `in`, overflow to `out`.
cudaError_t launch_spill(Tile t, bool count, int grid, const Job *jp, Spill in, Spill out,
                         cudaStream_t s);
// Blocks per SM of a persistent tile at 256 threads per block.
int persistent_block_threads(Tile t);  // threads per block of the persistent first tier
int persistent_blocks_per_sm(Tile t);
// Whether a scoring fits the packed 16-bit tiles exactly.
bool packed_scoring_ok(const Scoring &sc);
// A packed tile holds this scoring exactly (lanes of 32 slots need
// x + match <= 1022 beside packed_scoring_ok).
bool packed_tile_ok(Tile t, const Scoring &sc);
// The tile to run for this scoring: t itself if it holds it, else the
// packed 16-slot tile of the same width, else a 32-bit tile of its width.
Tile usable_tile(Tile t, const Scoring &sc);

cudaError_t launch_wide(bool count, int grid, const Job *jp, Spill in, int32_t *scratch,
                        int64_t scratch_per_cta, cudaStream_t s);
cudaError_t launch_validate(const Job *jp, uint64_t n_pairs, uint32_t *n_bad, cudaStream_t s);
cudaError_t launch_binning(const Job *jp, uint64_t n_pairs, int grid, uint32_t *hist,
                           uint32_t *offs, uint32_t *n_valid, uint32_t *order,
                           cudaStream_t s);
// Task length histogram of a job: hist[b] += tasks with
// ceil(log2(max(m, n) + 1)) = b (32 bins, invalid pairs left out).
cudaError_t launch_length_hist(const Job *jp, int grid, uint32_t *hist, cudaStream_t s);
// Stratified random sample of a pair table: dst[j] is one pair of the block
// [j*stride, (j+1)*stride), chosen by a hash of j and seed; m blocks.
cudaError_t launch_sample_pairs(const Pair *src, uint64_t n, uint32_t stride, uint32_t seed,
                                Pair *dst, uint64_t m, cudaStream_t s);
// Plain form: identity task order and per-sub-batch task counts / counters
// (ctl, 2 words per sub-batch of sub_pairs pairs).
cudaError_t launch_plain_setup(uint64_t n_pairs, uint64_t sub_pairs, uint32_t *order, uint32_t *ctl,
                              cudaStream_t s);
// Reverse complement of every read of `pk` (n_words words) into `out`, at
// the same offsets (reverse-strand pairs).
cudaError_t launch_revcomp(const uint32_t *pk, int64_t n_words, const uint64_t *read_off,
                           const uint32_t *read_len, uint32_t n_reads, uint32_t *out,
                           cudaStream_t s);
// Best seed of every read pair (consecutive records with equal a, b).
cudaError_t launch_best_seeds(const Pair *pairs, const int32_t *results, uint64_t n, int32_t match,
                              uint32_t *best, cudaStream_t s);
// Seed discovery over a read set on the device (xd_seeds.cu): the candidate
// pairs and their shared-k-mer counts, in (a, b) order, into host vectors.
// flags: XDROP_SEEDS_SORT selects the sort-based product (row-wise otherwise).  Synchronous on
// `s`.  Returns an XDROP_* code, with a message in err.
struct SeedStats {
    double ms = 0;              // CUDA events, first kernel to the last copy
    uint64_t occurrences = 0;   // k-mer occurrences
    uint64_t runs = 0;          // k-mers seen at least twice
    uint64_t candidates = 0;
    uint32_t product = 0;       // XDROP_SEEDS_ROWWISE or XDROP_SEEDS_SORT: the one that ran
    uint64_t nonzeros = 0;      // A's nonzeros, counted by the row-wise product
};
int find_candidates(cudaStream_t s, int sm_count, size_t budget, const uint32_t *packed,
                    const uint64_t *read_off, const uint32_t *read_len, uint32_t n_reads,
                    const uint32_t *h_len, uint32_t k, uint32_t stride, uint32_t lo, uint32_t hi,
                    uint32_t flags, std::vector<Pair> &out_pairs,
                    std::vector<uint32_t> &out_shared, SeedStats &stats, std::string &err);
// Adaptive acceptance flag of every aligned pair (xd_accept.cu).
cudaError_t launch_accept(const Pair *pairs, const int32_t *results, const uint32_t *read_len,
                          uint32_t n_reads, uint64_t n, int32_t match, int32_t mismatch,
                          uint32_t error_e4, uint32_t delta_e4, uint8_t *accept, cudaStream_t s);
cudaError_t launch_max_len(const uint32_t *read_len, uint32_t n_reads, uint32_t *out,
                           cudaStream_t s);

}  // namespace xd
