// Packed 16-bit band tiles (two window slots per register): 4x8 and 2x16
// (width 32, narrow bands such as x = 15), 4x16, 8x8 and 2x32 (width 64),
// 8x16, 16x8 and 4x32 (width 128).  Lanes of 32 slots spread each
// diagonal's per-lane bookkeeping over twice the cells.
#include "xd_launch.h"
#include "xd_serve_kernels.cuh"

namespace xd {

template <int L, int C2>
static cudaError_t packed_impl(int grid, const Job *jp, const uint32_t *order, const uint32_t *n,
                               uint32_t *ctr, Spill sp, cudaStream_t s)
{
    (void)cudaGetLastError();
    lockstep16_kernel<L, C2><<<grid, kPackedThreads, 0, s>>>(jp, order, n, ctr, sp, 1u);
    return cudaGetLastError();
}

template <int L, int C2>
static int packed_occupancy_impl()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lockstep16_kernel<L, C2>, kPackedThreads, 0);
    return b;
}

cudaError_t launch_persistent_packed(Tile t, int grid, const Job *jp, const uint32_t *order,
                                     const uint32_t *n, uint32_t *ctr, Spill sp,
                                     cudaStream_t s, bool *handled)
{
    *handled = true;
    if (t.packed) {
        if (t.lanes == 4 && t.c == 8) return packed_impl<4, 4>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 2 && t.c == 16) return packed_impl<2, 8>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 4 && t.c == 16) return packed_impl<4, 8>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 8 && t.c == 8) return packed_impl<8, 4>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 8 && t.c == 16) return packed_impl<8, 8>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 16 && t.c == 8) return packed_impl<16, 4>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 2 && t.c == 32) return packed_impl<2, 16>(grid, jp, order, n, ctr, sp, s);
        if (t.lanes == 4 && t.c == 32) return packed_impl<4, 16>(grid, jp, order, n, ctr, sp, s);
    }
    *handled = false;
    return cudaSuccess;
}

int occupancy_packed(Tile t)
{
    if (!t.packed) return -1;
    if (t.lanes == 4 && t.c == 8) return packed_occupancy_impl<4, 4>();
    if (t.lanes == 2 && t.c == 16) return packed_occupancy_impl<2, 8>();
    if (t.lanes == 4 && t.c == 16) return packed_occupancy_impl<4, 8>();
    if (t.lanes == 8 && t.c == 8) return packed_occupancy_impl<8, 4>();
    if (t.lanes == 8 && t.c == 16) return packed_occupancy_impl<8, 8>();
    if (t.lanes == 16 && t.c == 8) return packed_occupancy_impl<16, 4>();
    if (t.lanes == 2 && t.c == 32) return packed_occupancy_impl<2, 16>();
    if (t.lanes == 4 && t.c == 32) return packed_occupancy_impl<4, 16>();
    return -1;
}

bool packed_scoring_ok(const Scoring &sc) { return packed16_ok(sc); }

bool packed_tile_ok(Tile t, const Scoring &sc)
{
    return t.packed && (t.c == 32 ? packed32_ok(sc) : packed16_ok(sc));
}

Tile usable_tile(Tile t, const Scoring &sc)
{
    if (!t.packed || packed_tile_ok(t, sc)) return t;
    if (t.c == 32) {  // the 16-slot tile of the same width, or its 32-bit twin
        const Tile h{2 * t.lanes, 16, true};
        return packed16_ok(sc) ? h : Tile{h.lanes, 16, false};
    }
    if (t.width() < 64) return Tile{4, 16, false};  // no 32-bit tile this narrow
    return Tile{t.lanes, t.c, false};
}

int persistent_block_threads(Tile t) { return t.packed ? kPackedThreads : 256; }

template <int L1, int C2a, int L2, int C2>
static cudaError_t serve16_impl(int grid, const ServeArgs &a, const uint32_t *pk, int64_t nw,
                                cudaStream_t s)
{
    (void)cudaGetLastError();
    serve16_kernel<L1, C2a, L2, C2><<<grid, 256, 0, s>>>(a, pk, nw);
    return cudaGetLastError();
}

template <int L1, int C2a, int L2, int C2>
static int serve16_occupancy_impl()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, serve16_kernel<L1, C2a, L2, C2>, 256, 0);
    return b;
}

// Second tier as for the 32-bit tiles: 16x8 after a 64-slot first tier,
// 32x16 after a 128-slot one.
cudaError_t launch_serve_packed(Tile t, int grid, const ServeArgs &a, const uint32_t *pk,
                                int64_t nw, cudaStream_t s, bool *handled)
{
    *handled = true;
    if (t.packed) {
        // lanes of 32 slots serve as the 16-slot tile of the same width
        if (t.c == 32) t = Tile{2 * t.lanes, 16, true};
        if (t.lanes == 4 && t.c == 16) return serve16_impl<4, 8, 16, 8>(grid, a, pk, nw, s);
        if (t.lanes == 8 && t.c == 8) return serve16_impl<8, 4, 16, 8>(grid, a, pk, nw, s);
        if (t.lanes == 8 && t.c == 16) return serve16_impl<8, 8, 32, 16>(grid, a, pk, nw, s);
        if (t.lanes == 16 && t.c == 8) return serve16_impl<16, 4, 32, 16>(grid, a, pk, nw, s);
    }
    *handled = false;
    return cudaSuccess;
}

int serve_occupancy_packed(Tile t)
{
    if (!t.packed) return -1;
    if (t.c == 32) t = Tile{2 * t.lanes, 16, true};
    if (t.lanes == 4 && t.c == 16) return serve16_occupancy_impl<4, 8, 16, 8>();
    if (t.lanes == 8 && t.c == 8) return serve16_occupancy_impl<8, 4, 16, 8>();
    if (t.lanes == 8 && t.c == 16) return serve16_occupancy_impl<8, 8, 32, 16>();
    if (t.lanes == 16 && t.c == 8) return serve16_occupancy_impl<16, 4, 32, 16>();
    return -1;
}

}  // namespace xd
