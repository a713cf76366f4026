// Adaptive acceptance of aligned pairs, one thread per pair (the reading
// and the per-pair arithmetic are in xd_accept.cuh).
#include <cuda_runtime.h>

#include "xd_accept.cuh"
#include "xd_launch.h"

namespace xd {

namespace {

__global__ void __launch_bounds__(256)
accept_kernel(const Pair *__restrict__ pairs, const int32_t *__restrict__ res,
              const uint32_t *__restrict__ read_len, uint32_t n_reads, uint64_t n, int32_t match,
              int32_t mismatch, uint32_t error_e4, uint32_t delta_e4, uint8_t *__restrict__ out)
{
    const __int128 expected = xa::expected_e8(match, mismatch, error_e4);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const Pair p = pairs[i];
        const int32_t *r = res + 7 * i;  // xdrop_result: 7 x int32, status last
        const uint32_t a = p.a, b = p.b & ~kPairRC;
        out[i] = (a < n_reads && b < n_reads)
                     ? xa::accept_one(r[6], r[0], r[3], p.seed_a, p.seed_b, p.seed_len,
                                      read_len[a], read_len[b], match, expected, delta_e4)
                     : 0;
    }
}

}  // namespace

cudaError_t launch_accept(const Pair *pairs, const int32_t *results, const uint32_t *read_len,
                          uint32_t n_reads, uint64_t n, int32_t match, int32_t mismatch,
                          uint32_t error_e4, uint32_t delta_e4, uint8_t *accept, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 4096 ? blocks : 4096);
    accept_kernel<<<grid, 256, 0, s>>>(pairs, results, read_len, n_reads, n, match, mismatch,
                                       error_e4, delta_e4, accept);
    return cudaGetLastError();
}

}  // namespace xd
