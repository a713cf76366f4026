// Band tiles of width 64 (X around 50 with unit scores).
#include "xd_launch.h"
#include "xd_serve_kernels.cuh"

namespace xd {

template <int L, int C>
static cudaError_t persistent_impl(int grid, const Job *jp, const uint32_t *order,
                                   const uint32_t *n, uint32_t *ctr, Spill sp, cudaStream_t s)
{
    (void)cudaGetLastError();
    lockstep_kernel<L, C><<<grid, 256, 0, s>>>(jp, order, n, ctr, sp);
    return cudaGetLastError();
}

template <int L, int C>
static int occupancy_impl()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lockstep_kernel<L, C>, 256, 0);
    return b;
}

cudaError_t launch_persistent_narrow(Tile t, int grid, const Job *jp, const uint32_t *order,
                                     const uint32_t *n, uint32_t *ctr, Spill sp,
                                     cudaStream_t s, bool *handled)
{
    *handled = true;
    if (t.lanes == 4 && t.c == 16) return persistent_impl<4, 16>(grid, jp, order, n, ctr, sp, s);
    if (t.lanes == 8 && t.c == 8) return persistent_impl<8, 8>(grid, jp, order, n, ctr, sp, s);
    if (t.lanes == 16 && t.c == 4) return persistent_impl<16, 4>(grid, jp, order, n, ctr, sp, s);
    *handled = false;
    return cudaSuccess;
}

int occupancy_narrow(Tile t)
{
    if (t.lanes == 4 && t.c == 16) return occupancy_impl<4, 16>();
    if (t.lanes == 8 && t.c == 8) return occupancy_impl<8, 8>();
    if (t.lanes == 16 && t.c == 4) return occupancy_impl<16, 4>();
    return -1;
}


template <int L1, int C1, int L2, int C2>
static cudaError_t serve_impl(int grid, const ServeArgs &a, const uint32_t *pk, int64_t nw,
                              cudaStream_t s)
{
    (void)cudaGetLastError();
    serve_kernel<L1, C1, L2, C2><<<grid, 256, 0, s>>>(a, pk, nw);
    return cudaGetLastError();
}

template <int L1, int C1, int L2, int C2>
static int serve_occupancy_impl()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, serve_kernel<L1, C1, L2, C2>, 256, 0);
    return b;
}

cudaError_t launch_serve_narrow(Tile t, int grid, const ServeArgs &a, const uint32_t *pk, int64_t nw,
                           cudaStream_t s, bool *handled)
{
    *handled = true;
    if (t.lanes == 4 && t.c == 16) return serve_impl<4, 16, 16, 8>(grid, a, pk, nw, s);
    if (t.lanes == 8 && t.c == 8) return serve_impl<8, 8, 16, 8>(grid, a, pk, nw, s);
    if (t.lanes == 16 && t.c == 4) return serve_impl<16, 4, 16, 8>(grid, a, pk, nw, s);
    *handled = false;
    return cudaSuccess;
}

int serve_occupancy_narrow(Tile t)
{
    if (t.lanes == 4 && t.c == 16) return serve_occupancy_impl<4, 16, 16, 8>();
    if (t.lanes == 8 && t.c == 8) return serve_occupancy_impl<8, 8, 16, 8>();
    if (t.lanes == 16 && t.c == 4) return serve_occupancy_impl<16, 4, 16, 8>();
    return -1;
}

}  // namespace xd
