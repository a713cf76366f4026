// Seed discovery on the device: reliable k-mers and candidate read pairs
// (the per-element steps and the readings are in xd_seeds.cuh).
//
// Front steps, shared by both products, on one stream, tables in HBM:
//   1. kmer_kernel: one thread per k-mer occurrence computes its canonical
//      code (3 word loads, a 2-bit-group reversal), its read (binary search
//      of the per-read occurrence offsets) and its strand (one warp ballot
//      per 32 occurrences);
//   2. a stable radix sort of (code, occurrence id) over the code's 2k bits:
//      each k-mer's occurrences become one run, in read and position order;
//   3. the runs of length >= 2 (run-length encoding).
// Then A * A^T, A the read-by-reliable-k-mer matrix, one of two ways:
//   sort-based (XDROP_SEEDS_SORT): count_kernel and emit_kernel write one
//      entry per (read pair, shared reliable k-mer); a radix sort by pair, a
//      gather and a reduce-by-key with xs::CandMerge give one candidate per
//      pair;
//   row-wise (default): A's columns (csc_kernel) and rows
//      (csr_kernel), then row_kernel, one block per read a, accumulates a's
//      partners b > a in a shared-memory hash table (count + 64-bit minimum
//      seed key per partner, shared-memory atomics) in one pass, staging up
//      to 256 partners per read (a second pass rewrites the rare reads with
//      more); a radix sort of the few candidates orders them.  No per-entry
//      table exists.  A read with more partners than the table holds makes
//      the call take the sort-based product instead (same result).
// The sorts, run-length encoding, scans and reduce-by-key are CUB library
// primitives; everything else is the kernels here.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_run_length_encode.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/xdrop.h"
#include "xd_launch.h"
#include "xd_seeds.cuh"

namespace xd {

namespace {

constexpr int kThreads = 256;
constexpr uint64_t kMaxItems = (1ull << 31) - 1;  // CUB item counts are int

// ---------------------------------------------------------------- front

__global__ void __launch_bounds__(kThreads)
kmer_kernel(const uint32_t *__restrict__ packed, const uint64_t *__restrict__ read_off,
            const uint64_t *__restrict__ occ_off, uint32_t n_reads, uint64_t n_occ, uint32_t k,
            uint32_t stride, uint64_t *__restrict__ keys, uint32_t *__restrict__ occ,
            uint32_t *__restrict__ occ_rd, uint32_t *__restrict__ fwd_bits)
{
    const uint32_t lane = threadIdx.x & 31;
    // base is a multiple of 32 and the same for all lanes of a warp, so the
    // loop and the ballot are warp-uniform
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n_occ;
         base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = base + lane;
        bool fwd = false;
        if (q < n_occ) {
            uint32_t r;
            keys[q] = xs::occurrence(packed, read_off, occ_off, n_reads, k, stride, q, &r, &fwd);
            occ[q] = (uint32_t)q;
            occ_rd[q] = r;
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, fwd);
        if (lane == 0) fwd_bits[base >> 5] = m;
    }
}

// ---------------------------------------------------- sort-based product

__global__ void __launch_bounds__(kThreads)
count_kernel(const uint32_t *__restrict__ occ, const uint32_t *__restrict__ occ_rd,
             const int *__restrict__ run_off, const int *__restrict__ run_len, int n_runs,
             uint32_t lo, uint32_t hi, uint64_t *__restrict__ npairs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += gridDim.x * blockDim.x)
        npairs[i] = xs::run_pairs(occ, occ_rd, (uint64_t)run_off[i], (uint32_t)run_len[i], lo, hi);
}

__global__ void __launch_bounds__(kThreads)
emit_kernel(const uint64_t *__restrict__ codes, const uint32_t *__restrict__ occ,
            const uint32_t *__restrict__ occ_rd, const uint32_t *__restrict__ fwd_bits,
            const uint64_t *__restrict__ occ_off, const uint32_t *__restrict__ read_len,
            const int *__restrict__ run_off, const int *__restrict__ run_len,
            const uint64_t *__restrict__ pair_end, int n_runs, uint32_t k, uint32_t stride,
            uint32_t nb, uint64_t *__restrict__ keys, xs::Cand *__restrict__ ent,
            uint32_t *__restrict__ idx)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += gridDim.x * blockDim.x) {
        const uint64_t e0 = i ? pair_end[i - 1] : 0;
        if (pair_end[i] == e0) continue;
        const uint64_t s = (uint64_t)run_off[i];
        xs::run_emit(occ, occ_rd, fwd_bits, occ_off, read_len, codes[s], s, (uint32_t)run_len[i],
                     k, stride, nb, e0, keys, ent, idx);
    }
}

__global__ void __launch_bounds__(kThreads)
gather_kernel(const xs::Cand *__restrict__ ent, const uint32_t *__restrict__ idx, uint64_t n,
              xs::Cand *__restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = ent[idx[i]];
}

__global__ void __launch_bounds__(kThreads)
out_kernel(const uint64_t *__restrict__ keys, const xs::Cand *__restrict__ agg, int n,
           uint32_t nb, uint32_t k, Pair *__restrict__ pairs, uint32_t *__restrict__ shared)
{
    const uint64_t mask = nb >= 32 ? 0xFFFFFFFFull : (1ull << nb) - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const xs::Cand c = agg[i];
        Pair p;
        p.a = (uint32_t)(keys[i] >> nb);
        p.b = (uint32_t)(keys[i] & mask) | (c.rc ? xs::kPairRC : 0u);
        p.seed_a = c.pa;
        p.seed_b = c.sb;
        p.seed_len = k;
        pairs[i] = p;
        shared[i] = c.shared;
    }
}

// ------------------------------------------------------ row-wise product

__global__ void __launch_bounds__(kThreads)
ucount_kernel(const uint32_t *__restrict__ occ, const uint32_t *__restrict__ occ_rd,
              const int *__restrict__ run_off, const int *__restrict__ run_len, int n_runs,
              uint32_t lo, uint32_t hi, uint32_t *__restrict__ ucnt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += gridDim.x * blockDim.x)
        ucnt[i] = xs::run_reads(occ, occ_rd, (uint64_t)run_off[i], (uint32_t)run_len[i], lo, hi);
}

// Column i of A (reliable run i) into members[col_end[i-1] .. col_end[i]),
// with each member's column id; counts each read's row length.
__global__ void __launch_bounds__(kThreads)
csc_kernel(const uint32_t *__restrict__ occ, const uint32_t *__restrict__ occ_rd,
           const uint32_t *__restrict__ fwd_bits, const uint64_t *__restrict__ occ_off,
           const int *__restrict__ run_off, const int *__restrict__ run_len,
           const uint32_t *__restrict__ col_end, int n_runs, uint32_t stride,
           uint64_t *__restrict__ members, uint32_t *__restrict__ col_of,
           uint32_t *__restrict__ row_cnt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += gridDim.x * blockDim.x) {
        const uint32_t c0 = i ? col_end[i - 1] : 0, c1 = col_end[i];
        if (c1 == c0) continue;
        xs::run_members(occ, occ_rd, fwd_bits, occ_off, (uint64_t)run_off[i], (uint32_t)run_len[i],
                        stride, members + c0);
        for (uint32_t j = c0; j < c1; ++j) {
            col_of[j] = (uint32_t)i;
            atomicAdd(&row_cnt[(uint32_t)(members[j] >> 32)], 1u);
        }
    }
}

// Row a of A: (column, position << 1 | forward) of a's reliable k-mers, in
// any order within the row.
__global__ void __launch_bounds__(kThreads)
csr_kernel(const uint64_t *__restrict__ members, const uint32_t *__restrict__ col_of, uint64_t nnz,
           const uint32_t *__restrict__ row_end, uint32_t *__restrict__ row_fill,
           uint32_t *__restrict__ row_col, uint32_t *__restrict__ row_pos)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = members[j];
        const uint32_t r = (uint32_t)(m >> 32);
        const uint32_t e = (r ? row_end[r - 1] : 0) + atomicAdd(&row_fill[r], 1u);
        row_col[e] = col_of[j];
        row_pos[e] = (uint32_t)(m & 0xFFFFFFFFu);
    }
}

// One block per read a: the partners b > a of a in a shared-memory table.
// Partners of a read kept in its staging area by the first pass; a read
// with more goes through the second pass.
constexpr uint32_t kStage = 256;

// Per-read staging of the first pass: partner id, 64-bit best seed and
// shared count of up to kStage partners of every read.
struct Stage {
    uint32_t *key;
    unsigned long long *best;
    uint32_t *cnt;
};

// WRITE = false (first pass, block a = read a): cand_cnt[a] = number of
// partners (0 and the overflow flag when the table is full); up to kStage
// partners go to a's staging area, a read with more is listed in big.
// WRITE = true (second pass, block i = read big[i]): the partners' records
// at cand_end[a-1] ..., in table order.
template <bool WRITE>
__global__ void __launch_bounds__(kThreads)
row_kernel(const uint32_t *__restrict__ row_end, const uint32_t *__restrict__ row_col,
           const uint32_t *__restrict__ row_pos, const uint32_t *__restrict__ col_end,
           const uint64_t *__restrict__ members, const uint32_t *__restrict__ read_len,
           uint32_t k, uint32_t nb, uint64_t *__restrict__ cand_cnt,
           const uint64_t *__restrict__ cand_end, uint32_t *__restrict__ overflow, Stage stage,
           uint32_t *__restrict__ big, uint32_t *__restrict__ n_big,
           uint64_t *__restrict__ rkey, unsigned long long *__restrict__ rbest,
           uint32_t *__restrict__ rshared, uint32_t *__restrict__ ridx)
{
    constexpr uint32_t kSlots = 1u << xs::kTableLg;
    __shared__ uint32_t tkey[kSlots], tcnt[kSlots];
    __shared__ unsigned long long tbest[kSlots];
    __shared__ uint32_t ovf, cursor;
    const uint32_t a = WRITE ? big[blockIdx.x] : blockIdx.x;
    const uint32_t e0 = a ? row_end[a - 1] : 0, e1 = row_end[a];
    if (e0 == e1) {  // a holds no reliable k-mer
        if (!WRITE && threadIdx.x == 0) cand_cnt[a] = 0;
        return;
    }
    for (uint32_t h = threadIdx.x; h < kSlots; h += blockDim.x) {
        tkey[h] = xs::kEmpty;
        tcnt[h] = 0;
        tbest[h] = ~0ull;
    }
    if (threadIdx.x == 0) {
        ovf = 0;
        cursor = 0;
    }
    __syncthreads();
    const xs::RowTable t{tkey, tcnt, tbest, xs::kTableLg};
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    // a warp per row entry, its lanes over the entry's column
    for (uint32_t e = e0 + warp; e < e1; e += n_warps) {
        if (*(volatile uint32_t *)&ovf) break;
        const uint32_t col = row_col[e], pw = row_pos[e];
        const uint32_t c0 = col ? col_end[col - 1] : 0, c1 = col_end[col];
        for (uint32_t j = c0 + lane; j < c1; j += 32)
            if (!xs::row_term(t, a, pw >> 1, (pw & 1u) != 0, members[j], read_len, k)) ovf = 1;
    }
    __syncthreads();
    if (ovf) {
        if (!WRITE && threadIdx.x == 0) {
            cand_cnt[a] = 0;
            atomicOr(overflow, 1u);
        }
        return;
    }
    if (!WRITE) {
        uint32_t n = 0;
        for (uint32_t h = threadIdx.x; h < kSlots; h += blockDim.x) n += tkey[h] != xs::kEmpty;
        n = __reduce_add_sync(0xFFFFFFFFu, n);
        if (lane == 0) atomicAdd(&cursor, n);
        __syncthreads();
        const uint32_t total = cursor;
        if (threadIdx.x == 0) {
            cand_cnt[a] = total;
            if (total > kStage) big[atomicAdd(n_big, 1u)] = a;
        }
        if (total > kStage) return;  // the second pass writes this read
        __syncthreads();
        if (threadIdx.x == 0) cursor = 0;
        __syncthreads();
        const uint64_t base = (uint64_t)a * kStage;
        for (uint32_t h = threadIdx.x; h < kSlots; h += blockDim.x) {
            if (tkey[h] == xs::kEmpty) continue;
            const uint64_t i = base + atomicAdd(&cursor, 1u);
            stage.key[i] = tkey[h];
            stage.best[i] = tbest[h];
            stage.cnt[i] = tcnt[h];
        }
    } else {
        const uint64_t base = a ? cand_end[a - 1] : 0;
        for (uint32_t h = threadIdx.x; h < kSlots; h += blockDim.x) {
            if (tkey[h] == xs::kEmpty) continue;
            const uint64_t i = base + atomicAdd(&cursor, 1u);
            rkey[i] = ((uint64_t)a << nb) | tkey[h];
            rbest[i] = tbest[h];
            rshared[i] = tcnt[h];
            ridx[i] = (uint32_t)i;
        }
    }
}

// The staged partners of every read with at most kStage of them, to their
// records at cand_end[a-1] ...; a warp per read.
__global__ void __launch_bounds__(kThreads)
stage_out_kernel(const uint64_t *__restrict__ cand_cnt, const uint64_t *__restrict__ cand_end,
                 Stage stage, uint32_t n_reads, uint32_t nb, uint64_t *__restrict__ rkey,
                 unsigned long long *__restrict__ rbest, uint32_t *__restrict__ rshared,
                 uint32_t *__restrict__ ridx)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t a = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_reads;
         a += warps) {
        const uint64_t n = cand_cnt[a];
        if (n == 0 || n > kStage) continue;
        const uint64_t base = a ? cand_end[a - 1] : 0;
        for (uint32_t j = lane; j < n; j += 32) {
            const uint64_t s = a * kStage + j, i = base + j;
            rkey[i] = (a << nb) | stage.key[s];
            rbest[i] = stage.best[s];
            rshared[i] = stage.cnt[s];
            ridx[i] = (uint32_t)i;
        }
    }
}

__global__ void __launch_bounds__(kThreads)
row_out_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx,
               const unsigned long long *__restrict__ best, const uint32_t *__restrict__ cnt,
               int n, uint32_t nb, uint32_t k, Pair *__restrict__ pairs,
               uint32_t *__restrict__ shared)
{
    const uint64_t mask = nb >= 32 ? 0xFFFFFFFFull : (1ull << nb) - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t j = idx[i];
        const uint64_t b = best[j];
        Pair p;
        p.a = (uint32_t)(keys[i] >> nb);
        p.b = (uint32_t)(keys[i] & mask) | ((b & 1u) ? xs::kPairRC : 0u);
        p.seed_a = (uint32_t)(b >> 32);
        p.seed_b = (uint32_t)(b & 0xFFFFFFFFu) >> 1;
        p.seed_len = k;
        pairs[i] = p;
        shared[i] = cnt[j];
    }
}

// ------------------------------------------------------------------ host

int grid_for(uint64_t n, int sm_count)
{
    const uint64_t blocks = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sm_count * 8;
    return (int)std::max<uint64_t>(1, std::min(blocks, cap));
}

// Stream-ordered device allocations of one call, released together.
struct Arena {
    cudaStream_t s;
    size_t budget, used = 0;
    std::vector<void *> held;
    int rc = XDROP_OK;
    std::string err;
    Arena(cudaStream_t st, size_t b) : s(st), budget(b) {}
    ~Arena()
    {
        for (void *p : held) cudaFreeAsync(p, s);
    }
    template <class T>
    bool get(T *&p, uint64_t count)
    {
        size_t bytes = std::max<size_t>((size_t)count * sizeof(T), 16);
        if (budget && used + bytes > budget) {
            err = "seed discovery tables exceed the device memory budget";
            rc = XDROP_ENOMEM;
            return false;
        }
        void *q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, bytes, s);
        if (e != cudaSuccess) {
            err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
            rc = e == cudaErrorMemoryAllocation ? XDROP_ENOMEM : XDROP_ECUDA;
            return false;
        }
        held.push_back(q);
        used += bytes;
        p = (T *)q;
        return true;
    }
    int cuda(cudaError_t e, const char *what)
    {
        if (e == cudaSuccess) return XDROP_OK;
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return rc = XDROP_ECUDA;
    }
};

#define XS_GET(ptr, count) \
    if (!ar.get(ptr, (count))) return ar.rc
#define XS_CK(call)                                         \
    do {                                                    \
        if (ar.cuda((call), #call) != XDROP_OK) return ar.rc; \
    } while (0)

// Input and front-step tables shared by both products.
struct Front {
    const uint32_t *packed, *read_len;
    const uint64_t *read_off;
    uint32_t n_reads, k, stride, lo, hi, nb;
    int sm_count;
    uint64_t n_occ = 0;
    uint64_t *occ_off = nullptr;
    const uint64_t *codes = nullptr;
    const uint32_t *occ = nullptr;
    uint32_t *occ_rd = nullptr, *fwd_bits = nullptr;
    int *run_off = nullptr, *run_len = nullptr;
    int n_runs = 0;
};

template <class T>
int read_back(Arena &ar, T *h, const T *d)
{
    XS_CK(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, ar.s));
    XS_CK(cudaStreamSynchronize(ar.s));
    return XDROP_OK;
}

int front(Arena &ar, Front &f, const std::vector<uint64_t> &occ_off)
{
    const int n = (int)f.n_occ;
    uint64_t *keys0, *keys1;
    uint32_t *occ0, *occ1;
    XS_GET(f.occ_off, f.n_reads + 1);
    XS_GET(keys0, f.n_occ);
    XS_GET(keys1, f.n_occ);
    XS_GET(occ0, f.n_occ);
    XS_GET(occ1, f.n_occ);
    XS_GET(f.occ_rd, f.n_occ);
    XS_GET(f.fwd_bits, (f.n_occ + 31) / 32);
    XS_CK(cudaMemcpyAsync(f.occ_off, occ_off.data(), (f.n_reads + 1) * sizeof(uint64_t),
                          cudaMemcpyHostToDevice, ar.s));
    kmer_kernel<<<grid_for(f.n_occ, f.sm_count), kThreads, 0, ar.s>>>(
        f.packed, f.read_off, f.occ_off, f.n_reads, f.n_occ, f.k, f.stride, keys0, occ0, f.occ_rd,
        f.fwd_bits);
    XS_CK(cudaGetLastError());
    // occurrences grouped by k-mer, stable: read, then position order
    cub::DoubleBuffer<uint64_t> dk(keys0, keys1);
    cub::DoubleBuffer<uint32_t> dv(occ0, occ1);
    char *tmp;
    size_t tmp_bytes = 0;
    XS_CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, dk, dv, n, 0, (int)(2 * f.k), ar.s));
    XS_GET(tmp, tmp_bytes);
    XS_CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, dk, dv, n, 0, (int)(2 * f.k), ar.s));
    f.codes = dk.Current();
    f.occ = dv.Current();
    // runs of length >= 2 (a k-mer seen once pairs no reads)
    int *d_nruns;
    XS_GET(f.run_off, f.n_occ / 2 + 1);
    XS_GET(f.run_len, f.n_occ / 2 + 1);
    XS_GET(d_nruns, 1);
    size_t rle_bytes = 0;
    char *rle_tmp;
    XS_CK(cub::DeviceRunLengthEncode::NonTrivialRuns(nullptr, rle_bytes, f.codes, f.run_off,
                                                     f.run_len, d_nruns, n, ar.s));
    XS_GET(rle_tmp, rle_bytes);
    XS_CK(cub::DeviceRunLengthEncode::NonTrivialRuns(rle_tmp, rle_bytes, f.codes, f.run_off,
                                                     f.run_len, d_nruns, n, ar.s));
    return read_back(ar, &f.n_runs, d_nruns);
}

int copy_out(Arena &ar, const Pair *d_pairs, const uint32_t *d_shared, int n_cand,
             std::vector<Pair> &out_pairs, std::vector<uint32_t> &out_shared)
{
    out_pairs.resize(n_cand);
    out_shared.resize(n_cand);
    XS_CK(cudaMemcpyAsync(out_pairs.data(), d_pairs, (size_t)n_cand * sizeof(Pair),
                          cudaMemcpyDeviceToHost, ar.s));
    XS_CK(cudaMemcpyAsync(out_shared.data(), d_shared, (size_t)n_cand * 4, cudaMemcpyDeviceToHost,
                          ar.s));
    return XDROP_OK;
}

int sort_product(Arena &ar, const Front &f, std::vector<Pair> &out_pairs,
                 std::vector<uint32_t> &out_shared)
{
    const int n_runs = f.n_runs;
    // pairs per reliable run and their output slots
    uint64_t *npairs, *pair_end;
    XS_GET(npairs, n_runs);
    XS_GET(pair_end, n_runs);
    count_kernel<<<grid_for(n_runs, f.sm_count), kThreads, 0, ar.s>>>(
        f.occ, f.occ_rd, f.run_off, f.run_len, n_runs, f.lo, f.hi, npairs);
    XS_CK(cudaGetLastError());
    size_t scan_bytes = 0;
    char *scan_tmp;
    XS_CK(cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, npairs, pair_end, n_runs, ar.s));
    XS_GET(scan_tmp, scan_bytes);
    XS_CK(cub::DeviceScan::InclusiveSum(scan_tmp, scan_bytes, npairs, pair_end, n_runs, ar.s));
    uint64_t n_ent = 0;
    if (int rc = read_back(ar, &n_ent, pair_end + (n_runs - 1))) return rc;
    if (n_ent == 0) return XDROP_OK;
    if (n_ent > kMaxItems) {
        ar.err = "more than 2^31 - 1 shared-k-mer entries; narrow the frequency window";
        return ar.rc = XDROP_ENOMEM;
    }
    // one entry per (read pair, shared reliable k-mer)
    uint64_t *ek0, *ek1;
    uint32_t *ei0, *ei1;
    xs::Cand *ent, *ent_sorted;
    XS_GET(ek0, n_ent);
    XS_GET(ek1, n_ent);
    XS_GET(ei0, n_ent);
    XS_GET(ei1, n_ent);
    XS_GET(ent, n_ent);
    XS_GET(ent_sorted, n_ent);
    emit_kernel<<<grid_for(n_runs, f.sm_count), kThreads, 0, ar.s>>>(
        f.codes, f.occ, f.occ_rd, f.fwd_bits, f.occ_off, f.read_len, f.run_off, f.run_len, pair_end,
        n_runs, f.k, f.stride, f.nb, ek0, ent, ei0);
    XS_CK(cudaGetLastError());
    // entries grouped by read pair, reduced to one candidate each
    const int ne = (int)n_ent;
    cub::DoubleBuffer<uint64_t> ek(ek0, ek1);
    cub::DoubleBuffer<uint32_t> ei(ei0, ei1);
    size_t sort_bytes = 0;
    char *sort_tmp;
    XS_CK(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, ek, ei, ne, 0, (int)(2 * f.nb), ar.s));
    XS_GET(sort_tmp, sort_bytes);
    XS_CK(cub::DeviceRadixSort::SortPairs(sort_tmp, sort_bytes, ek, ei, ne, 0, (int)(2 * f.nb), ar.s));
    gather_kernel<<<grid_for(n_ent, f.sm_count), kThreads, 0, ar.s>>>(ent, ei.Current(), n_ent,
                                                                      ent_sorted);
    XS_CK(cudaGetLastError());
    uint64_t *uniq;
    xs::Cand *agg;
    int *d_ncand;
    XS_GET(uniq, n_ent);
    XS_GET(agg, n_ent);
    XS_GET(d_ncand, 1);
    size_t red_bytes = 0;
    char *red_tmp;
    XS_CK(cub::DeviceReduce::ReduceByKey(nullptr, red_bytes, ek.Current(), uniq, ent_sorted, agg,
                                         d_ncand, xs::CandMerge(), ne, ar.s));
    XS_GET(red_tmp, red_bytes);
    XS_CK(cub::DeviceReduce::ReduceByKey(red_tmp, red_bytes, ek.Current(), uniq, ent_sorted, agg,
                                         d_ncand, xs::CandMerge(), ne, ar.s));
    int n_cand = 0;
    if (int rc = read_back(ar, &n_cand, d_ncand)) return rc;
    if (n_cand <= 0) return XDROP_OK;
    Pair *d_pairs;
    uint32_t *d_shared;
    XS_GET(d_pairs, n_cand);
    XS_GET(d_shared, n_cand);
    out_kernel<<<grid_for(n_cand, f.sm_count), kThreads, 0, ar.s>>>(uniq, agg, n_cand, f.nb, f.k,
                                                                     d_pairs, d_shared);
    XS_CK(cudaGetLastError());
    return copy_out(ar, d_pairs, d_shared, n_cand, out_pairs, out_shared);
}

// *done = false when some read's table overflowed (nothing written).
int row_product(Arena &ar, const Front &f, std::vector<Pair> &out_pairs,
                std::vector<uint32_t> &out_shared, bool *done, uint64_t *nonzeros)
{
    *done = false;
    const int n_runs = f.n_runs, n_reads = (int)f.n_reads;
    // columns: distinct reads per reliable run, scanned
    uint32_t *ucnt, *col_end;
    XS_GET(ucnt, n_runs);
    XS_GET(col_end, n_runs);
    ucount_kernel<<<grid_for(n_runs, f.sm_count), kThreads, 0, ar.s>>>(
        f.occ, f.occ_rd, f.run_off, f.run_len, n_runs, f.lo, f.hi, ucnt);
    XS_CK(cudaGetLastError());
    size_t bytes = 0;
    char *tmp;
    XS_CK(cub::DeviceScan::InclusiveSum(nullptr, bytes, ucnt, col_end, n_runs, ar.s));
    XS_GET(tmp, bytes);
    XS_CK(cub::DeviceScan::InclusiveSum(tmp, bytes, ucnt, col_end, n_runs, ar.s));
    uint32_t nnz = 0;
    if (int rc = read_back(ar, &nnz, col_end + (n_runs - 1))) return rc;
    *nonzeros = nnz;
    if (nnz == 0) {
        *done = true;
        return XDROP_OK;
    }
    uint64_t *members;
    uint32_t *col_of, *row_cnt, *row_end, *row_fill, *row_col, *row_pos;
    XS_GET(members, nnz);
    XS_GET(col_of, nnz);
    XS_GET(row_cnt, n_reads);
    XS_GET(row_end, n_reads);
    XS_GET(row_fill, n_reads);
    XS_GET(row_col, nnz);
    XS_GET(row_pos, nnz);
    XS_CK(cudaMemsetAsync(row_cnt, 0, (size_t)n_reads * 4, ar.s));
    XS_CK(cudaMemsetAsync(row_fill, 0, (size_t)n_reads * 4, ar.s));
    csc_kernel<<<grid_for(n_runs, f.sm_count), kThreads, 0, ar.s>>>(
        f.occ, f.occ_rd, f.fwd_bits, f.occ_off, f.run_off, f.run_len, col_end, n_runs, f.stride,
        members, col_of, row_cnt);
    XS_CK(cudaGetLastError());
    bytes = 0;
    XS_CK(cub::DeviceScan::InclusiveSum(nullptr, bytes, row_cnt, row_end, n_reads, ar.s));
    XS_GET(tmp, bytes);
    XS_CK(cub::DeviceScan::InclusiveSum(tmp, bytes, row_cnt, row_end, n_reads, ar.s));
    csr_kernel<<<grid_for(nnz, f.sm_count), kThreads, 0, ar.s>>>(members, col_of, nnz, row_end,
                                                                 row_fill, row_col, row_pos);
    XS_CK(cudaGetLastError());
    // each read's partners in one pass: counted, and staged when there are
    // at most kStage of them; reads with more are recomputed and written
    // by a second pass over those reads alone
    uint64_t *cand_cnt, *cand_end;
    uint32_t *flags, *big;  // flags[0]: table overflow, flags[1]: reads listed in big
    Stage stage;
    XS_GET(cand_cnt, n_reads);
    XS_GET(cand_end, n_reads);
    XS_GET(flags, 2);
    XS_GET(big, n_reads);
    XS_GET(stage.key, (uint64_t)n_reads * kStage);
    XS_GET(stage.best, (uint64_t)n_reads * kStage);
    XS_GET(stage.cnt, (uint64_t)n_reads * kStage);
    XS_CK(cudaMemsetAsync(flags, 0, 8, ar.s));
    row_kernel<false><<<n_reads, kThreads, 0, ar.s>>>(
        row_end, row_col, row_pos, col_end, members, f.read_len, f.k, f.nb, cand_cnt, nullptr,
        flags, stage, big, flags + 1, nullptr, nullptr, nullptr, nullptr);
    XS_CK(cudaGetLastError());
    bytes = 0;
    XS_CK(cub::DeviceScan::InclusiveSum(nullptr, bytes, cand_cnt, cand_end, n_reads, ar.s));
    XS_GET(tmp, bytes);
    XS_CK(cub::DeviceScan::InclusiveSum(tmp, bytes, cand_cnt, cand_end, n_reads, ar.s));
    uint32_t hflags[2] = {0, 0};
    uint64_t n_cand = 0;
    XS_CK(cudaMemcpyAsync(hflags, flags, 8, cudaMemcpyDeviceToHost, ar.s));
    if (int rc = read_back(ar, &n_cand, cand_end + (n_reads - 1))) return rc;
    const uint32_t ovf = hflags[0], n_big = hflags[1];
    if (ovf) return XDROP_OK;  // not done: the sort-based product takes over
    *done = true;
    if (n_cand == 0) return XDROP_OK;
    if (n_cand > kMaxItems) {
        ar.err = "more than 2^31 - 1 candidate pairs";
        return ar.rc = XDROP_ENOMEM;
    }
    uint64_t *rk0, *rk1;
    uint32_t *ri0, *ri1, *rshared;
    unsigned long long *rbest;
    XS_GET(rk0, n_cand);
    XS_GET(rk1, n_cand);
    XS_GET(ri0, n_cand);
    XS_GET(ri1, n_cand);
    XS_GET(rbest, n_cand);
    XS_GET(rshared, n_cand);
    stage_out_kernel<<<grid_for((uint64_t)n_reads * 32, f.sm_count), kThreads, 0, ar.s>>>(
        cand_cnt, cand_end, stage, (uint32_t)n_reads, f.nb, rk0, rbest, rshared, ri0);
    XS_CK(cudaGetLastError());
    if (n_big) {
        row_kernel<true><<<n_big, kThreads, 0, ar.s>>>(
            row_end, row_col, row_pos, col_end, members, f.read_len, f.k, f.nb, nullptr, cand_end,
            nullptr, stage, big, nullptr, rk0, rbest, rshared, ri0);
        XS_CK(cudaGetLastError());
    }
    // candidates in (a, b) order
    const int nc = (int)n_cand;
    cub::DoubleBuffer<uint64_t> rk(rk0, rk1);
    cub::DoubleBuffer<uint32_t> ri(ri0, ri1);
    bytes = 0;
    XS_CK(cub::DeviceRadixSort::SortPairs(nullptr, bytes, rk, ri, nc, 0, (int)(2 * f.nb), ar.s));
    XS_GET(tmp, bytes);
    XS_CK(cub::DeviceRadixSort::SortPairs(tmp, bytes, rk, ri, nc, 0, (int)(2 * f.nb), ar.s));
    Pair *d_pairs;
    uint32_t *d_shared;
    XS_GET(d_pairs, n_cand);
    XS_GET(d_shared, n_cand);
    row_out_kernel<<<grid_for(n_cand, f.sm_count), kThreads, 0, ar.s>>>(
        rk.Current(), ri.Current(), rbest, rshared, nc, f.nb, f.k, d_pairs, d_shared);
    XS_CK(cudaGetLastError());
    return copy_out(ar, d_pairs, d_shared, nc, out_pairs, out_shared);
}

}  // namespace

int find_candidates(cudaStream_t st, int sm_count, size_t budget, const uint32_t *packed,
                    const uint64_t *read_off, const uint32_t *read_len, uint32_t n_reads,
                    const uint32_t *h_len, uint32_t k, uint32_t stride, uint32_t lo, uint32_t hi,
                    uint32_t flags, std::vector<Pair> &out_pairs,
                    std::vector<uint32_t> &out_shared, SeedStats &stats, std::string &err)
{
    out_pairs.clear();
    out_shared.clear();
    stats = SeedStats{};
    std::vector<uint64_t> occ_off(n_reads + 1, 0);
    for (uint32_t r = 0; r < n_reads; ++r)
        occ_off[r + 1] = occ_off[r] + (h_len[r] >= k ? (h_len[r] - k) / stride + 1 : 0);
    stats.occurrences = occ_off[n_reads];
    if (stats.occurrences < 2) return XDROP_OK;
    if (stats.occurrences > kMaxItems) {
        err = "more than 2^31 - 1 k-mer occurrences; raise the stride";
        return XDROP_ENOMEM;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        err = "cudaEventCreate failed";
        return XDROP_ECUDA;
    }
    int rc = XDROP_OK;
    {
        Arena ar(st, budget);
        Front f;
        f.packed = packed;
        f.read_len = read_len;
        f.read_off = read_off;
        f.n_reads = n_reads;
        f.k = k;
        f.stride = stride;
        f.lo = lo;
        f.hi = hi;
        f.nb = xs::id_bits(n_reads);
        f.sm_count = sm_count;
        f.n_occ = stats.occurrences;
        rc = ar.cuda(cudaEventRecord(ev[0], st), "cudaEventRecord");
        if (!rc) rc = front(ar, f, occ_off);
        stats.runs = rc ? 0 : (uint64_t)std::max(f.n_runs, 0);
        bool done = rc != XDROP_OK || f.n_runs <= 0;
        const bool rows_ok = n_reads < kMaxItems;  // one block per read
        if (!done && !(flags & XDROP_SEEDS_SORT) && rows_ok) {
            rc = row_product(ar, f, out_pairs, out_shared, &done, &stats.nonzeros);
            if (done && !rc) stats.product = XDROP_SEEDS_ROWWISE;
        }
        if (!done && !rc) {
            rc = sort_product(ar, f, out_pairs, out_shared);
            if (!rc) stats.product = XDROP_SEEDS_SORT;
        }
        if (!rc) rc = ar.cuda(cudaEventRecord(ev[1], st), "cudaEventRecord");
        if (!rc) rc = ar.cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        if (!rc) {
            float ms = 0.f;
            rc = ar.cuda(cudaEventElapsedTime(&ms, ev[0], ev[1]), "cudaEventElapsedTime");
            stats.ms = ms;
        }
        if (rc) err = ar.err;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) {
        out_pairs.clear();
        out_shared.clear();
        return rc;
    }
    stats.candidates = out_pairs.size();
    return XDROP_OK;
}

#undef XS_GET
#undef XS_CK

}  // namespace xd
