// Allocation-free entry point: the unbounded-band tier with its scratch in
// a file-scope device array instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory at the time they align: a
// process whose device memory is owned entirely by another allocator (a
// framework pool that must see every allocation), a latency-critical path
// that cannot afford cudaMalloc/cudaFree and their implicit device
// synchronisation, or code that issues its work while a stream is being
// captured, where allocation calls are not allowed.  xdrop_align_static
// serves them: it takes the caller's device inputs and output, launches one
// kernel on the caller's stream, and calls no allocating routine.
//
// The scratch is the static array below.  Every GPU that loads this library
// holds it (32 MiB) until the process exits; all calls on a device share it
// and it keeps the last call's contents.  The kernel initialises every word
// it reads, so nothing has to be cleared between calls.  Calls whose work
// overlaps on the GPU (different streams, or no ordering between them) race
// on the array and must not be issued that way.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "xd_device.cuh"
#include "xdrop.h"

namespace xd {

constexpr int64_t kStaticScratchWords = (int64_t)8 << 20;  // 8 Mi int32 = 32 MiB
constexpr int kStaticMaxCtas = 128;

static __device__ __align__(256) int32_t g_static_scratch[kStaticScratchWords];

// One CTA per task (all 2*n_pairs tasks, grid-stride), each CTA with its
// own slice of the static scratch.  Pairs that fail the limits get status
// XDROP_STATUS_INVALID and zero scores; a task whose extension is longer
// than the slice allows gets status XDROP_STATUS_TOO_LONG and zeros in its
// side's three fields.
__global__ void __launch_bounds__(WIDE_THREADS)
static_wide_kernel(Job J, int32_t *scratch, int64_t per_cta)
{
    int32_t *diag = scratch + (int64_t)blockIdx.x * per_cta;
    const uint64_t n_tasks = 2 * J.n_pairs;
    for (uint64_t t = blockIdx.x; t < n_tasks; t += gridDim.x) {
        const uint32_t task = (uint32_t)t;
        const Ext e = decode(J, task);
        int32_t *o = J.out + (size_t)e.pair * 7;
        if (!e.ok) {
            if (threadIdx.x == 0 && e.side == 0) {
                for (int k = 0; k < 6; ++k) o[k] = 0;
                o[6] = XDROP_STATUS_INVALID;
            }
            continue;
        }
        if ((int64_t)3 * (e.m + 1) > per_cta) {
            if (threadIdx.x == 0) {
                for (int k = 0; k < 3; ++k) o[3 * e.side + k] = 0;
                atomicOr(&o[6], XDROP_STATUS_TOO_LONG);
            }
            continue;
        }
        int32_t sc, bi, bj;
        int64_t cells;
        extend_wide<false>(e, J.sc, diag, sc, bi, bj, cells);
        if (threadIdx.x == 0) write_result(J, e, sc, bi, bj);
        __syncthreads();
    }
}

__global__ void static_clear_status(Job J)
{
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < J.n_pairs;
         p += (uint64_t)gridDim.x * blockDim.x)
        J.out[p * 7 + 6] = XDROP_STATUS_OK;
}

}  // namespace xd

namespace {

thread_local std::string g_static_err;

int static_fail(int code, const char *msg, cudaError_t e = cudaSuccess)
{
    g_static_err = msg;
    if (e != cudaSuccess) {
        g_static_err += ": ";
        g_static_err += cudaGetErrorString(e);
    }
    return code;
}

}  // namespace

extern "C" int xdrop_align_static(const uint32_t *packed, uint64_t n_words,
                                  const uint64_t *read_off, const uint32_t *read_len,
                                  uint32_t n_reads, const xdrop_pair *pairs, size_t n_pairs,
                                  const xdrop_scoring *s, uint32_t max_read_len,
                                  xdrop_result *out, void *stream)
{
    using namespace xd;
    if (!s) return static_fail(XDROP_EINVAL, "scoring is NULL");
    if (s->match <= 0 || s->mismatch > 0 || s->gap >= 0 || s->x < 0 ||
        (int64_t)s->x >= SCORE_LIMIT || s->match >= SCORE_LIMIT ||
        -(int64_t)s->mismatch >= SCORE_LIMIT || -(int64_t)s->gap >= SCORE_LIMIT)
        return static_fail(XDROP_EINVAL, "scoring outside the limits of xdrop.h");
    if (n_pairs == 0) return XDROP_OK;
    if (!packed || !n_words || !read_off || !read_len || !pairs || !out)
        return static_fail(XDROP_EINVAL, "NULL input or output array");
    if (2 * (uint64_t)n_pairs >= ((uint64_t)1 << 32))
        return static_fail(XDROP_EINVAL, "too many pairs in one call");
    const int64_t per_task = 3 * ((int64_t)max_read_len + 1);
    if (per_task > kStaticScratchWords) {
        char msg[160];
        snprintf(msg, sizeof msg,
                 "max_read_len %u exceeds the static scratch (reads up to %lld bases)",
                 max_read_len, (long long)(kStaticScratchWords / 3 - 1));
        return static_fail(XDROP_EINVAL, msg);
    }
    // In host code g_static_scratch names a host-side stand-in, not device
    // memory: the kernel gets the array's address on the current device,
    // looked up on every call (with that device current) so that a context
    // re-created after a device reset never sees a stale address.  The
    // first lookup on a device loads the module there, which is why the
    // first call on a device must come before any stream capture.
    void *sym = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&sym, g_static_scratch);
    if (e != cudaSuccess) return static_fail(XDROP_ECUDA, "cudaGetSymbolAddress", e);
    int32_t *scratch = (int32_t *)sym;
    int64_t per_cta = (per_task + 63) / 64 * 64;
    int grid = (int)std::min<int64_t>(kStaticMaxCtas, kStaticScratchWords / per_cta);
    if (grid < 1) grid = 1, per_cta = kStaticScratchWords;
    Job J{};
    J.packed = packed;
    J.n_words = (int64_t)n_words;
    J.read_off = read_off;
    J.read_len = read_len;
    J.n_reads = n_reads;
    J.pairs = (const Pair *)pairs;
    J.n_pairs = n_pairs;
    J.sc = Scoring{s->match, s->mismatch, s->gap, s->x};
    J.out = (int32_t *)out;
    J.cells = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();
    const uint64_t cb = (n_pairs + 255) / 256;
    static_clear_status<<<(unsigned)std::min<uint64_t>(cb, 1024), 256, 0, st>>>(J);
    static_wide_kernel<<<grid, WIDE_THREADS, 0, st>>>(J, scratch, per_cta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(XDROP_ECUDA, "kernel launch", e);
    return XDROP_OK;
}

extern "C" const char *xdrop_static_last_error(void) { return g_static_err.c_str(); }
