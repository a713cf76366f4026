// Seed discovery on the device: reliable k-mers and candidate read pairs
// (the per-element steps and the readings are in xd_seeds.cuh).
//
// Pipeline, all on one stream, every intermediate table in HBM:
//   1. kmer_kernel: one thread per k-mer occurrence computes its canonical
//      code (3 word loads, a 2-bit-group reversal), its read (binary search
//      of the per-read occurrence offsets) and its strand (one warp ballot
//      per 32 occurrences).
//   2. a stable radix sort of (code, occurrence id) over the code's 2k bits:
//      each k-mer's occurrences become one run, in read and position order;
//   3. the runs of length >= 2 (run-length encoding);
//   4. count_kernel: one thread per run, the number of read pairs of a
//      reliable run; an inclusive scan gives each run its output slots;
//   5. emit_kernel: one thread per run writes its pairs (key a,b; Cand);
//   6. a stable radix sort of the pair keys, a gather of the Cands into
//      key order, and a reduce-by-key with xs::CandMerge;
//   7. out_kernel: one xdrop_pair and one shared count per candidate.
// The two sorts, the run-length encoding, the scan and the reduce-by-key
// are CUB library primitives; everything else is the kernels here.
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

int grid_for(uint64_t n, int sm_count)
{
    const uint64_t blocks = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sm_count * 8;
    return (int)std::max<uint64_t>(1, std::min(blocks, cap));
}

// Stream-ordered device allocations released together.
struct Arena {
    cudaStream_t s;
    size_t budget, used = 0;
    std::vector<void *> held;
    explicit Arena(cudaStream_t st, size_t b) : s(st), budget(b) {}
    ~Arena() { release(); }
    void release()
    {
        for (void *p : held) cudaFreeAsync(p, s);
        held.clear();
        used = 0;
    }
};

}  // namespace

int find_candidates(cudaStream_t st, int sm_count, size_t budget, const uint32_t *packed,
                    const uint64_t *read_off, const uint32_t *read_len, uint32_t n_reads,
                    const uint32_t *h_len, uint32_t k, uint32_t stride, uint32_t lo, uint32_t hi,
                    std::vector<Pair> &out_pairs, std::vector<uint32_t> &out_shared,
                    std::string &err)
{
    out_pairs.clear();
    out_shared.clear();
    std::vector<uint64_t> occ_off(n_reads + 1, 0);
    for (uint32_t r = 0; r < n_reads; ++r)
        occ_off[r + 1] = occ_off[r] + (h_len[r] >= k ? (h_len[r] - k) / stride + 1 : 0);
    const uint64_t n_occ = occ_off[n_reads];
    if (n_occ < 2) return XDROP_OK;
    if (n_occ > kMaxItems) {
        err = "more than 2^31 - 1 k-mer occurrences; raise the stride";
        return XDROP_ENOMEM;
    }
    Arena ar(st, budget);
    int rc = XDROP_OK;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        bytes = std::max<size_t>(bytes, 16);
        if (ar.budget && ar.used + bytes > ar.budget) {
            err = "seed discovery tables exceed the device memory budget";
            rc = XDROP_ENOMEM;
            return false;
        }
        cudaError_t e = cudaMallocAsync(p, bytes, ar.s);
        if (e != cudaSuccess) {
            err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
            rc = e == cudaErrorMemoryAllocation ? XDROP_ENOMEM : XDROP_ECUDA;
            return false;
        }
        ar.held.push_back(*p);
        ar.used += bytes;
        return true;
    };
#define XS_ALLOC(ptr, bytes) \
    if (!alloc((void **)&(ptr), (bytes))) return rc
#define XS_CK(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            err = std::string(#call ": ") + cudaGetErrorString(e_);   \
            return XDROP_ECUDA;                                       \
        }                                                             \
    } while (0)

    const int n = (int)n_occ;
    uint64_t *d_occ_off, *keys0, *keys1;
    uint32_t *occ0, *occ1, *occ_rd, *fwd_bits;
    XS_ALLOC(d_occ_off, (n_reads + 1) * sizeof(uint64_t));
    XS_ALLOC(keys0, n_occ * 8);
    XS_ALLOC(keys1, n_occ * 8);
    XS_ALLOC(occ0, n_occ * 4);
    XS_ALLOC(occ1, n_occ * 4);
    XS_ALLOC(occ_rd, n_occ * 4);
    XS_ALLOC(fwd_bits, (n_occ + 31) / 32 * 4);
    XS_CK(cudaMemcpyAsync(d_occ_off, occ_off.data(), (n_reads + 1) * sizeof(uint64_t),
                          cudaMemcpyHostToDevice, st));
    kmer_kernel<<<grid_for(n_occ, sm_count), kThreads, 0, st>>>(
        packed, read_off, d_occ_off, n_reads, n_occ, k, stride, keys0, occ0, occ_rd, fwd_bits);
    XS_CK(cudaGetLastError());

    // 2. occurrences grouped by k-mer, stable: read, then position order
    cub::DoubleBuffer<uint64_t> dk(keys0, keys1);
    cub::DoubleBuffer<uint32_t> dv(occ0, occ1);
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    XS_CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, dk, dv, n, 0, (int)(2 * k), st));
    XS_ALLOC(tmp, tmp_bytes);
    XS_CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, dk, dv, n, 0, (int)(2 * k), st));
    const uint64_t *codes = dk.Current();
    const uint32_t *occ = dv.Current();

    // 3. runs of length >= 2 (a k-mer seen once pairs no reads)
    int *run_off, *run_len, *d_nruns;
    XS_ALLOC(run_off, (n_occ / 2 + 1) * sizeof(int));
    XS_ALLOC(run_len, (n_occ / 2 + 1) * sizeof(int));
    XS_ALLOC(d_nruns, sizeof(int));
    size_t rle_bytes = 0;
    void *rle_tmp = nullptr;
    XS_CK(cub::DeviceRunLengthEncode::NonTrivialRuns(nullptr, rle_bytes, codes, run_off, run_len,
                                                     d_nruns, n, st));
    XS_ALLOC(rle_tmp, rle_bytes);
    XS_CK(cub::DeviceRunLengthEncode::NonTrivialRuns(rle_tmp, rle_bytes, codes, run_off, run_len,
                                                     d_nruns, n, st));
    int n_runs = 0;
    XS_CK(cudaMemcpyAsync(&n_runs, d_nruns, sizeof(int), cudaMemcpyDeviceToHost, st));
    XS_CK(cudaStreamSynchronize(st));
    if (n_runs <= 0) return XDROP_OK;

    // 4. pairs per reliable run and their output slots
    uint64_t *npairs, *pair_end;
    XS_ALLOC(npairs, (size_t)n_runs * 8);
    XS_ALLOC(pair_end, (size_t)n_runs * 8);
    count_kernel<<<grid_for(n_runs, sm_count), kThreads, 0, st>>>(occ, occ_rd, run_off, run_len,
                                                                   n_runs, lo, hi, npairs);
    XS_CK(cudaGetLastError());
    size_t scan_bytes = 0;
    void *scan_tmp = nullptr;
    XS_CK(cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, npairs, pair_end, n_runs, st));
    XS_ALLOC(scan_tmp, scan_bytes);
    XS_CK(cub::DeviceScan::InclusiveSum(scan_tmp, scan_bytes, npairs, pair_end, n_runs, st));
    uint64_t n_ent = 0;
    XS_CK(cudaMemcpyAsync(&n_ent, pair_end + (n_runs - 1), 8, cudaMemcpyDeviceToHost, st));
    XS_CK(cudaStreamSynchronize(st));
    if (n_ent == 0) return XDROP_OK;
    if (n_ent > kMaxItems) {
        err = "more than 2^31 - 1 shared-k-mer entries; narrow the frequency window";
        return XDROP_ENOMEM;
    }

    // 5. one entry per (read pair, shared reliable k-mer)
    const uint32_t nb = xs::id_bits(n_reads);
    uint64_t *ek0, *ek1;
    uint32_t *ei0, *ei1;
    xs::Cand *ent, *ent_sorted;
    XS_ALLOC(ek0, n_ent * 8);
    XS_ALLOC(ek1, n_ent * 8);
    XS_ALLOC(ei0, n_ent * 4);
    XS_ALLOC(ei1, n_ent * 4);
    XS_ALLOC(ent, n_ent * sizeof(xs::Cand));
    XS_ALLOC(ent_sorted, n_ent * sizeof(xs::Cand));
    emit_kernel<<<grid_for(n_runs, sm_count), kThreads, 0, st>>>(
        codes, occ, occ_rd, fwd_bits, d_occ_off, read_len, run_off, run_len, pair_end, n_runs, k,
        stride, nb, ek0, ent, ei0);
    XS_CK(cudaGetLastError());

    // 6. entries grouped by read pair, reduced to one candidate each
    const int ne = (int)n_ent;
    cub::DoubleBuffer<uint64_t> ek(ek0, ek1);
    cub::DoubleBuffer<uint32_t> ei(ei0, ei1);
    size_t sort2_bytes = 0;
    void *sort2_tmp = nullptr;
    XS_CK(cub::DeviceRadixSort::SortPairs(nullptr, sort2_bytes, ek, ei, ne, 0, (int)(2 * nb), st));
    XS_ALLOC(sort2_tmp, sort2_bytes);
    XS_CK(cub::DeviceRadixSort::SortPairs(sort2_tmp, sort2_bytes, ek, ei, ne, 0, (int)(2 * nb), st));
    gather_kernel<<<grid_for(n_ent, sm_count), kThreads, 0, st>>>(ent, ei.Current(), n_ent,
                                                                   ent_sorted);
    XS_CK(cudaGetLastError());
    uint64_t *uniq;
    xs::Cand *agg;
    int *d_ncand;
    XS_ALLOC(uniq, n_ent * 8);
    XS_ALLOC(agg, n_ent * sizeof(xs::Cand));
    XS_ALLOC(d_ncand, sizeof(int));
    size_t red_bytes = 0;
    void *red_tmp = nullptr;
    XS_CK(cub::DeviceReduce::ReduceByKey(nullptr, red_bytes, ek.Current(), uniq, ent_sorted, agg,
                                         d_ncand, xs::CandMerge(), ne, st));
    XS_ALLOC(red_tmp, red_bytes);
    XS_CK(cub::DeviceReduce::ReduceByKey(red_tmp, red_bytes, ek.Current(), uniq, ent_sorted, agg,
                                         d_ncand, xs::CandMerge(), ne, st));
    int n_cand = 0;
    XS_CK(cudaMemcpyAsync(&n_cand, d_ncand, sizeof(int), cudaMemcpyDeviceToHost, st));
    XS_CK(cudaStreamSynchronize(st));
    if (n_cand <= 0) return XDROP_OK;

    // 7. pair records
    Pair *d_pairs;
    uint32_t *d_shared;
    XS_ALLOC(d_pairs, (size_t)n_cand * sizeof(Pair));
    XS_ALLOC(d_shared, (size_t)n_cand * 4);
    out_kernel<<<grid_for(n_cand, sm_count), kThreads, 0, st>>>(uniq, agg, n_cand, nb, k, d_pairs,
                                                                 d_shared);
    XS_CK(cudaGetLastError());
    out_pairs.resize(n_cand);
    out_shared.resize(n_cand);
    XS_CK(cudaMemcpyAsync(out_pairs.data(), d_pairs, (size_t)n_cand * sizeof(Pair),
                          cudaMemcpyDeviceToHost, st));
    XS_CK(cudaMemcpyAsync(out_shared.data(), d_shared, (size_t)n_cand * 4, cudaMemcpyDeviceToHost,
                          st));
    XS_CK(cudaStreamSynchronize(st));
#undef XS_ALLOC
#undef XS_CK
    return XDROP_OK;
}

}  // namespace xd
