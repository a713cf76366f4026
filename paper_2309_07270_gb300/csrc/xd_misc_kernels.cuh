// Non-template kernels (validation, length binning, max read length).
// Included by exactly one translation unit.
#pragma once
#include "xd_device.cuh"

namespace xd {

// ---------------------------------------------------------------------------
// Validation (device submits): status per pair, zero scores for bad pairs.
// ---------------------------------------------------------------------------
__global__ void validate_kernel(const Job *jp, uint32_t *n_bad)
{
    const Job J = *jp;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < J.n_pairs;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const Pair pr = J.pairs[p];
        const bool ok = job_pair_ok(J, pr);
        int32_t *o = J.out + p * 7;
        if (!ok) {
            for (int k = 0; k < 6; ++k) o[k] = 0;
            o[6] = 1;
            atomicAdd(n_bad, 1u);
        } else {
            o[6] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Length binning (batched form): tasks sorted into bins by
// ceil(log2(max(m, n) + 1)), bins laid out longest first, so the persistent
// kernel starts the longest extensions first.
// ---------------------------------------------------------------------------
constexpr int NBINS = 32;
constexpr int BIN_THREADS = 256;

__device__ __forceinline__ int task_bin(const Job &J, uint32_t task)
{
    Ext e = decode(J, task);
    if (!e.ok) return -1;
    uint32_t w = (uint32_t)(e.m > e.n ? e.m : e.n);
    return 32 - __clz(w);
}

// hist[b] += tasks in bin b.  Block-local counts first, one global atomic
// per (block, bin).
__global__ void __launch_bounds__(BIN_THREADS)
bin_count_kernel(const Job *jp, uint32_t *hist)
{
    const Job J = *jp;
    __shared__ uint32_t h[NBINS];
    if (threadIdx.x < NBINS) h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t n_tasks = 2 * J.n_pairs;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tasks;
         t += (uint64_t)gridDim.x * blockDim.x) {
        int b = task_bin(J, (uint32_t)t);
        if (b >= 0) atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NBINS && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// offs[b] = start of bin b in the longest-first order; *n_valid = total.
__global__ void bin_scan_kernel(const uint32_t *hist, uint32_t *offs, uint32_t *n_valid)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t run = 0;
        for (int b = NBINS - 1; b >= 0; --b) {
            offs[b] = run;
            run += hist[b];
        }
        *n_valid = run;
    }
}

// order[offs[b] + rank] = task.  Each block takes a contiguous range of
// tasks, counts it per bin, reserves its slice of every bin with one
// atomic, then places its tasks.
__global__ void __launch_bounds__(BIN_THREADS)
bin_scatter_kernel(const Job *jp, uint32_t *offs, uint32_t *order)
{
    const Job J = *jp;
    __shared__ uint32_t h[NBINS];
    __shared__ uint32_t base[NBINS];
    const uint64_t n_tasks = 2 * J.n_pairs;
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x; t0 < n_tasks;
         t0 += (uint64_t)gridDim.x * blockDim.x) {
        if (threadIdx.x < NBINS) h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t t = t0 + threadIdx.x;
        int b = -1;
        uint32_t rank = 0;
        if (t < n_tasks) {
            b = task_bin(J, (uint32_t)t);
            if (b >= 0) rank = atomicAdd(&h[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < NBINS && h[threadIdx.x])
            base[threadIdx.x] = atomicAdd(&offs[threadIdx.x], h[threadIdx.x]);
        __syncthreads();
        if (b >= 0) order[base[b] + rank] = (uint32_t)t;
        __syncthreads();
    }
}

// Largest read length (for sizing the unbounded tier's scratch).
// Autotuning sample: one pair from every block of `stride` consecutive
// pairs, at an offset inside the block drawn from a hash of the block index
// and the seed (a stratified random sample that spans the whole job, so a
// sorted or clustered input is sampled evenly).
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void sample_pairs_kernel(const Pair *src, uint64_t n, uint32_t stride, uint32_t seed,
                                    Pair *dst, uint64_t m)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b0 = j * stride;
        const uint64_t len = (n - b0 < stride) ? n - b0 : stride;
        dst[j] = src[b0 + mix32((uint32_t)j * 0x9e3779b9u ^ seed) % len];
    }
}

// Plain form: the identity task order (tasks in pair order) and, for every
// sub-batch k of sub_pairs pairs, its task count (ctl[2k]) and a zeroed
// work counter (ctl[2k + 1]) for its first-tier launch.
__global__ void plain_setup_kernel(uint64_t n_pairs, uint64_t sub_pairs, uint32_t *order,
                                   uint32_t *ctl)
{
    const uint64_t n_tasks = 2 * n_pairs, n_sub = (n_pairs + sub_pairs - 1) / sub_pairs;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_tasks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        order[i] = (uint32_t)i;
        if (i < n_sub) {
            const uint64_t left = n_pairs - i * sub_pairs;
            ctl[2 * i] = (uint32_t)(2 * (left < sub_pairs ? left : sub_pairs));
            ctl[2 * i + 1] = 0;
        }
    }
}

__global__ void max_len_kernel(const uint32_t *read_len, uint32_t n_reads, uint32_t *out)
{
    uint32_t m = 0;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_reads;
         r += gridDim.x * blockDim.x)
        m = max(m, read_len[r]);
    m = __reduce_max_sync(FULL, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// Reverse complements of all reads (reverse-strand pairs): read r's reverse
// complement goes to the same word offsets of `out`.  Output base p of the
// read is the complement (code ^ 3) of input base len - 1 - p, so output
// word w is the reversed, complemented 16 input bases ending at len - 16 w;
// bases past the read's end in its last word are left arbitrary.
// ---------------------------------------------------------------------------
__global__ void revcomp_kernel(const uint32_t *pk, int64_t n_words, const uint64_t *read_off,
                               const uint32_t *read_len, uint32_t n_reads, uint32_t *out)
{
    for (uint32_t r = blockIdx.x; r < n_reads; r += gridDim.x) {
        const int64_t off = (int64_t)read_off[r];
        const int64_t len = (int64_t)read_len[r];
        const int64_t w0 = off >> 4;
        const int64_t nwr = (len + 15) >> 4;
        for (int64_t w = threadIdx.x; w < nwr; w += blockDim.x)
            out[w0 + w] = rev16(load16_u(pk, n_words, off + len - 16 * (w + 1))) ^ 0xFFFFFFFFu;
    }
}

// ---------------------------------------------------------------------------
// Several seeds per read pair: consecutive records with the same a and b
// form a group; the thread of a group's first record scans the group and
// writes the index of its best valid record (highest left + seed_len*match
// + right, lowest index on ties, 0xFFFFFFFF if none) for every member.
// ---------------------------------------------------------------------------
__global__ void best_seeds_kernel(const Pair *pairs, const int32_t *res, uint64_t n, int32_t match,
                                  uint32_t *best)
{
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const Pair q = pairs[p];
        if (p > 0) {
            const Pair r = pairs[p - 1];
            if (r.a == q.a && r.b == q.b) continue;  // not the first record of its group
        }
        uint32_t win = 0xFFFFFFFFu;
        int64_t top = 0;
        uint64_t e = p;
        for (; e < n; ++e) {
            const Pair r = pairs[e];
            if (e > p && (r.a != q.a || r.b != q.b)) break;
            const int32_t *o = res + e * 7;
            if (o[6] != 0) continue;
            const int64_t tot = (int64_t)o[0] + (int64_t)r.seed_len * match + (int64_t)o[3];
            if (win == 0xFFFFFFFFu || tot > top) {
                win = (uint32_t)e;
                top = tot;
            }
        }
        for (uint64_t k = p; k < e; ++k) best[k] = win;
    }
}

}  // namespace xd
