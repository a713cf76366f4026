// Host runtime of the C ABI declared in include/xdrop.h.
//
// A context owns one CUDA stream, a device job descriptor, scratch (task
// order, bin counters, spill lists, the unbounded tier's diagonals) and,
// in batched mode, one instantiated CUDA graph of the whole launch
// sequence.  Kernels read their job descriptor from device memory, so the
// graph is replayed unchanged for every submit (and every chunk of a
// large submit); it is re-captured only when scratch has to grow.
//
// Plain mode is the paper's baseline scheme (Section "Baseline": the work
// is split into batches of 10,000 and each is fed to the GPU in turn): one
// launch of the 32-lane tile per 10,000-pair sub-batch, in submit order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/xdrop.h"
#include "xd_launch.h"
#include "xd_seeds.cuh"
#include "xd_serve.h"

using namespace xd;

static_assert(sizeof(xdrop_pair) == sizeof(Pair), "pair layout");
static_assert(sizeof(xdrop_result) == 28, "result layout");
static_assert(sizeof(xdrop_scoring) == sizeof(Scoring), "scoring layout");

namespace {

thread_local std::string g_err = "";

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(XDROP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

constexpr uint64_t kSubBatchPairs = 10000;  // plain mode (Section "Baseline")
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Counter block layout (uint32 words) in device memory.
enum : int {
    C_HIST = 0,          // NBINS
    C_OFFS = 32,         // NBINS
    C_NVALID = 64,
    C_COUNTER = 65,
    C_SPILL0 = 66,       // spill counts of tiers 0..2
    C_SPILL1 = 67,
    C_SPILL2 = 68,
    C_NBAD = 69,
    C_MAXLEN = 70,
    C_WORDS = 72
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct Ticket {
    uint64_t id = 0;
    bool device_submit = false;
    size_t n_pairs = 0;
    xdrop_result *out = nullptr;  // caller's results (host submit)
    void *d_mem = nullptr;        // inputs + results (host submit)
    size_t d_bytes = 0;
    void *h_pinned = nullptr;     // results staging + counters + job
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr, ev_done = nullptr;
    uint32_t launches = 0, graph_replays = 0;
    uint32_t *h_ctrs = nullptr;   // copy of the counter block at the end
    Job *h_job = nullptr;
    xdrop_result *h_out = nullptr;
};

}  // namespace

struct xdrop_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    uint32_t mode = XDROP_MODE_BATCHED;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::unordered_map<uint64_t, Ticket *> tickets;
    uint64_t next_id = 1;
    size_t used = 0;  // device bytes held (scratch + tickets)

    Job *d_job = nullptr;
    uint32_t *d_ctrs = nullptr;
    DevBuf order, spill[3], wide;
    DevBuf plain_ctl;  // plain mode: task count and work counter per sub-batch
    size_t cap_tasks = 0;
    int64_t wide_per_cta = 0;
    int wide_grid = 0;

    // cached max read length of the last device submit
    const uint32_t *maxlen_ptr = nullptr;
    uint32_t maxlen_n = 0, maxlen_val = 0;

    Tile tile0 = {8, 8};
    int tile0_bps = 0;            // resident blocks per SM of tile0
    Tile forced = {0, 0};         // xdrop_set_tile
    // tuned first tile per (scoring, length bucket of the job)
    std::map<std::tuple<int, int, int, int, int>, Tile> tuned;
    uint64_t scratch_version = 0; // bumped whenever a scratch buffer moves
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev_main0 = nullptr, ev_main1 = nullptr;  // recorded inside the graph
    Tile graph_tile = {0, 0};
    uint64_t graph_version = ~0ull;

    xdrop_stats last = {};

    // resident reads (xdrop_load_reads) and the serving loop
    DevBuf r_packed, r_off, r_len;
    std::vector<uint64_t> h_off;
    std::vector<uint32_t> h_len;
    uint64_t r_words = 0;
    uint32_t r_n = 0, r_maxlen = 0;
    bool have_reads = false;
    uint64_t reads_gen = 0;  // bumped by every xdrop_load_reads
    xd::Server *srv = nullptr;
    uint64_t serve_idle_ns = 0;  // xdrop_set_serve_idle (0: the default)

    // the last seed discovery result (xdrop_find_candidates)
    std::vector<Pair> cand_pairs;
    std::vector<uint32_t> cand_shared;
    std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, uint32_t> cand_params;
    uint64_t cand_gen = 0;  // reads_gen it was computed on; 0: none
    xd::SeedStats seed_stats;
};

constexpr uint64_t kServeTicket = 1ull << 63;

namespace {

int dev_alloc(xdrop_ctx *c, DevBuf &b, size_t bytes)
{
    if (b.cap >= bytes) return XDROP_OK;
    size_t nb = std::max(bytes, b.cap + b.cap / 2);
    // In serving mode the budget bounds the requests in flight instead.
    if (c->budget && c->mode != XDROP_MODE_SERVE && c->used - b.cap + nb > c->budget) {
        nb = bytes;
        if (c->used - b.cap + nb > c->budget)
            return fail(c->tickets.empty() ? XDROP_ENOMEM : XDROP_EBUSY,
                        "device memory budget exceeded (%zu bytes needed)", nb);
    }
    if (b.p) {
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaFree(b.p));
        c->used -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    CK(cudaMalloc(&b.p, nb));
    b.cap = nb;
    c->used += nb;
    c->scratch_version += 1;
    return XDROP_OK;
}

// Scratch for n_tasks tasks and the unbounded tier for reads up to maxlen.
int ensure_scratch(xdrop_ctx *c, size_t n_tasks, uint32_t maxlen)
{
    size_t tasks = std::max<size_t>(n_tasks, 1024);
    int rc;
    if ((rc = dev_alloc(c, c->order, tasks * 4))) return rc;
    for (auto &s : c->spill)
        if ((rc = dev_alloc(c, s, tasks * 4))) return rc;
    c->cap_tasks = std::min(c->order.cap, std::min(c->spill[0].cap,
                            std::min(c->spill[1].cap, c->spill[2].cap))) / 4;
    int64_t per = (int64_t)3 * ((int64_t)maxlen + 1);
    per = (per + 63) / 64 * 64;
    if (per > c->wide_per_cta) {
        if ((rc = dev_alloc(c, c->wide, (size_t)per * 4 * c->wide_grid))) return rc;
        c->wide_per_cta = per;
    }
    return XDROP_OK;
}

int validate_scoring(const xdrop_scoring *s)
{
    if (!s) return fail(XDROP_EINVAL, "scoring is NULL");
    if (s->match <= 0) return fail(XDROP_EINVAL, "match must be > 0 (got %d)", s->match);
    if (s->mismatch > 0) return fail(XDROP_EINVAL, "mismatch must be <= 0 (got %d)", s->mismatch);
    if (s->gap >= 0) return fail(XDROP_EINVAL, "gap must be < 0 (got %d)", s->gap);
    if (s->x < 0 || (int64_t)s->x >= SCORE_LIMIT)
        return fail(XDROP_EINVAL, "x must be in [0, 2^25) (got %d)", s->x);
    if (s->match >= SCORE_LIMIT || -(int64_t)s->mismatch >= SCORE_LIMIT || -(int64_t)s->gap >= SCORE_LIMIT)
        return fail(XDROP_EINVAL, "score magnitude too large");
    return XDROP_OK;
}

Spill spill_of(xdrop_ctx *c, int k)
{
    return Spill{(uint32_t *)c->spill[k].p, c->d_ctrs + C_SPILL0 + k};
}

Tile next_tile_after(Tile t)
{
    // The 128-wide tile for narrower first tiers, then 512.  Its overflow
    // tier is 32 lanes x 4 cells: the few extensions that reach it run one
    // per warp, and with half the cells per lane a diagonal takes half as
    // long, so the tier (which ends when its longest extension does) is
    // shorter than with 16 lanes x 8 cells.
    if (t.width() < 128) return Tile{32, 4};
    return Tile{32, 16};
}

// Enqueue the batched launch sequence (graph body) with first tile t0.
int enqueue_batched(xdrop_ctx *c, Tile t0, int bps, bool main_events, uint32_t *launches)
{
    cudaStream_t s = c->stream;
    uint32_t *ctr = c->d_ctrs;
    CK(cudaMemsetAsync(ctr, 0, C_NBAD * 4, s));  // keep NBAD / MAXLEN
    const int bgrid = c->sm_count * 4;
    CK(launch_binning(c->d_job, 0, bgrid, ctr + C_HIST, ctr + C_OFFS, ctr + C_NVALID,
                      (uint32_t *)c->order.p, s));
    if (bps <= 0) return fail(XDROP_ECUDA, "tile %dx%d not available", t0.lanes, t0.c);
    // External record nodes, so the events are really recorded on replay.
    if (main_events) CK(cudaEventRecordWithFlags(c->ev_main0, s, cudaEventRecordExternal));
    CK(launch_persistent(t0, c->sm_count * bps, c->d_job, (uint32_t *)c->order.p,
                         ctr + C_NVALID, ctr + C_COUNTER, spill_of(c, 0), s));
    if (main_events) CK(cudaEventRecordWithFlags(c->ev_main1, s, cudaEventRecordExternal));
    int n = 4;
    Tile t1 = next_tile_after(t0);
    int k = 0;
    if (t1.width() < 512) {
        CK(launch_spill(t1, false, c->sm_count * 4, c->d_job, spill_of(c, 0), spill_of(c, 1), s));
        k = 1;
        ++n;
    }
    CK(launch_spill(Tile{32, 16}, false, c->sm_count * 2, c->d_job, spill_of(c, k),
                    spill_of(c, k + 1), s));
    CK(launch_wide(false, c->wide_grid, c->d_job, spill_of(c, k + 1), (int32_t *)c->wide.p,
                   c->wide_per_cta, s));
    n += 2;
    if (launches) *launches = n;
    return XDROP_OK;
}

// Candidate first tiles for autotuning (all persistent instantiations);
// the packed 16-bit ones only for scorings they hold exactly.
const Tile kTuneTiles[] = {{4, 16}, {8, 8}, {16, 4}, {8, 16}, {16, 8}, {32, 4}};
const Tile kPackedTiles[] = {{4, 8, true},  {2, 16, true}, {4, 16, true}, {8, 8, true},
                             {2, 32, true}, {8, 16, true}, {16, 8, true}, {4, 32, true}};

// The first tile for a submit: the forced one (unpacked when the scoring
// does not fit 16 bits) or the tuned one for this scoring.
int pick_tile(xdrop_ctx *c, Ticket *tk, const Job &job, Tile *out);

// Time the whole batched sequence for every candidate first tile on a
// sample of `job`, pick the fastest.  Synchronous.
int autotune(xdrop_ctx *c, Ticket *tk, const Job &job, Tile *best)
{
    cudaStream_t s = c->stream;
    // Scorings that fit 16 bits choose among the packed tiles only (each is
    // faster than the 32-bit tile of its shape), on a third of the job so
    // the end of the sample, where few extensions are left, does not decide
    // between tiles of different concurrency; other scorings time the
    // 32-bit tiles on an eighth.  The sample is stratified and random (one
    // pair out of every block of 3 or 8, seeded), so it has the job's
    // length mix even when the input is sorted or clustered.
    //
    // The sample and its results live in the job's own result buffer
    // (48 bytes per sampled pair, at most 16 of the 28 bytes per pair there),
    // so tuning needs no memory beyond the submit's; the buffer is zeroed
    // afterwards, before validation writes the status words.
    const bool packed = packed_scoring_ok(job.sc);
    const uint32_t stride = job.n_pairs <= 3 * 4096 ? 1u : (packed ? 3u : 8u);
    const uint64_t m = (job.n_pairs + stride - 1) / stride;
    Job js = job;
    if (stride > 1) {
        Pair *sp = (Pair *)job.out;
        int32_t *so = job.out + m * (sizeof(Pair) / 4);
        CK(launch_sample_pairs(job.pairs, job.n_pairs, stride, 0x5eed1234u, sp, m, s));
        js.pairs = sp;
        js.out = so;
        js.n_pairs = m;
    }
    CK(cudaStreamSynchronize(s));
    *tk->h_job = js;
    CK(cudaMemcpyAsync(c->d_job, tk->h_job, sizeof(Job), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    *best = Tile{0, 0};
    std::vector<Tile> cands;
    if (packed) cands.assign(std::begin(kPackedTiles), std::end(kPackedTiles));
    else cands.assign(std::begin(kTuneTiles), std::end(kTuneTiles));
    for (const Tile &t : cands) {
        if (t.packed && !packed_tile_ok(t, job.sc)) continue;
        const int bps = persistent_blocks_per_sm(t);
        if (bps <= 0) continue;
        float tmin = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, s));
            int rc = enqueue_batched(c, t, bps, false, nullptr);
            if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tmin = std::min(tmin, ms);
        }
        if (tmin < best_ms) { best_ms = tmin; *best = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the full job for the real run, with a clean result buffer
    *tk->h_job = job;
    CK(cudaMemcpyAsync(c->d_job, tk->h_job, sizeof(Job), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(job.out, 0, job.n_pairs * sizeof(xdrop_result), s));
    CK(cudaStreamSynchronize(s));
    return best->lanes ? XDROP_OK : fail(XDROP_ECUDA, "no tile could be timed");
}

// Length bucket of a job (the tuning key beside the scoring): the length
// bin ceil(log2(max(m, n) + 1)) holding the median of the job's work, each
// task weighted by 2^bin (about its length), from a device histogram read
// back synchronously.  Workloads of different length mixes tune apart.
int length_bucket(xdrop_ctx *c, Ticket *tk, int *bucket)
{
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->d_ctrs + C_HIST, 0, 32 * 4, s));
    CK(launch_length_hist(c->d_job, c->sm_count * 4, c->d_ctrs + C_HIST, s));
    CK(cudaMemcpyAsync(tk->h_ctrs, c->d_ctrs + C_HIST, 32 * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double total = 0, run = 0;
    for (int b = 0; b < 32; ++b) total += (double)tk->h_ctrs[b] * std::ldexp(1.0, b);
    *bucket = 0;
    for (int b = 0; b < 32; ++b) {
        run += (double)tk->h_ctrs[b] * std::ldexp(1.0, b);
        if (run * 2 >= total && total > 0) {
            *bucket = b;
            break;
        }
    }
    return XDROP_OK;
}

int pick_tile(xdrop_ctx *c, Ticket *tk, const Job &job, Tile *out)
{
    Tile t = c->forced;
    if (t.lanes) {
        *out = usable_tile(t, job.sc);
        return XDROP_OK;
    }
    int bucket = 0;
    if (int rc = length_bucket(c, tk, &bucket)) return rc;
    auto key = std::make_tuple(job.sc.match, job.sc.mismatch, job.sc.gap, job.sc.x, bucket);
    auto it = c->tuned.find(key);
    if (it != c->tuned.end()) {
        *out = it->second;
        return XDROP_OK;
    }
    int rc = autotune(c, tk, job, &t);
    if (rc) return rc;
    c->tuned[key] = t;
    *out = t;
    return XDROP_OK;
}

int run_batched(xdrop_ctx *c, Ticket *tk)
{
    if (!c->gexec || c->graph_version != c->scratch_version ||
        !c->graph_tile.same(c->tile0)) {
        c->tile0_bps = persistent_blocks_per_sm(c->tile0);
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        uint32_t launches = 0;
        int rc = enqueue_batched(c, c->tile0, c->tile0_bps, true, &launches);
        cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return fail(XDROP_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(XDROP_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        c->graph_version = c->scratch_version;
        c->graph_tile = c->tile0;
        c->last.launches = launches;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    tk->graph_replays += 1;
    tk->launches += c->last.launches;
    return XDROP_OK;
}

// Plain form (Section "Method", Baseline: batches of 10,000 alignments, each
// sent to the GPU on its own): one launch of the first band tile per
// 10,000-pair sub-batch, in pair order, with a grid sized to the
// sub-batch; no length binning, no graph, no autotuning.  The tile is the
// forced one (xdrop_set_tile), else packed 4x16, so that it can run the
// very tile and arithmetic of the batched form.  Overflowing extensions go
// through the same wider tiers afterwards.
int run_plain(xdrop_ctx *c, Ticket *tk, const Job &job)
{
    cudaStream_t s = c->stream;
    const uint64_t n_pairs = job.n_pairs;
    CK(cudaMemsetAsync(c->d_ctrs, 0, C_NBAD * 4, s));
    const Tile t0 = usable_tile(c->forced.lanes ? c->forced : Tile{4, 16, true}, job.sc);
    c->tile0 = t0;
    const int bps = persistent_blocks_per_sm(t0);
    if (bps <= 0) return fail(XDROP_ECUDA, "tile %dx%d not available", t0.lanes, t0.c);
    const uint64_t n_sub = (n_pairs + kSubBatchPairs - 1) / kSubBatchPairs;
    int rc;
    if ((rc = dev_alloc(c, c->plain_ctl, n_sub * 8))) return rc;
    uint32_t *order = (uint32_t *)c->order.p, *ctl = (uint32_t *)c->plain_ctl.p;
    CK(launch_plain_setup(n_pairs, kSubBatchPairs, order, ctl, s));
    const uint64_t groups_per_block = (uint64_t)persistent_block_threads(t0) / t0.lanes;
    for (uint64_t k = 0; k < n_sub; ++k) {
        const uint64_t p0 = k * kSubBatchPairs, np = std::min(kSubBatchPairs, n_pairs - p0);
        const uint64_t blocks = (2 * np + groups_per_block - 1) / groups_per_block;
        const int grid = (int)std::min<uint64_t>(blocks, (uint64_t)c->sm_count * bps);
        CK(launch_persistent(t0, grid, c->d_job, order + 2 * p0, ctl + 2 * k, ctl + 2 * k + 1,
                             spill_of(c, 0), s));
    }
    tk->launches += (uint32_t)(1 + n_sub);
    Tile t1 = next_tile_after(t0);
    int k = 0;
    if (t1.width() < 512) {
        CK(launch_spill(t1, false, c->sm_count * 4, c->d_job, spill_of(c, 0), spill_of(c, 1), s));
        k = 1;
        tk->launches += 1;
    }
    CK(launch_spill(Tile{32, 16}, false, c->sm_count * 2, c->d_job, spill_of(c, k),
                    spill_of(c, k + 1), s));
    CK(launch_wide(false, c->wide_grid, c->d_job, spill_of(c, k + 1), (int32_t *)c->wide.p,
                   c->wide_per_cta, s));
    tk->launches += 2;
    return XDROP_OK;
}

void free_ticket(xdrop_ctx *c, Ticket *tk)
{
    if (tk->ev_begin) cudaEventDestroy(tk->ev_begin);
    if (tk->ev_end) cudaEventDestroy(tk->ev_end);
    if (tk->ev_done) cudaEventDestroy(tk->ev_done);
    if (tk->d_mem) {
        cudaFree(tk->d_mem);
        c->used -= tk->d_bytes;
    }
    if (tk->h_pinned) cudaFreeHost(tk->h_pinned);
    delete tk;
}

// Common tail of both submit flavours: descriptor, launches, copies back.
int launch_ticket(xdrop_ctx *c, Ticket *tk, const Job &job, uint32_t maxlen)
{
    cudaStream_t s = c->stream;
    int rc;
    if ((rc = ensure_scratch(c, 2 * job.n_pairs, maxlen))) return rc;
    *tk->h_job = job;
    CK(cudaMemcpyAsync(c->d_job, tk->h_job, sizeof(Job), cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(tk->ev_begin, s));
    // the tile first: autotuning uses the result buffer as scratch, and
    // validation then writes every status word
    if (job.n_pairs && c->mode != XDROP_MODE_PLAIN) {
        if ((rc = pick_tile(c, tk, job, &c->tile0))) return rc;
    }
    if (tk->device_submit) {
        CK(cudaMemsetAsync(c->d_ctrs + C_NBAD, 0, 4, s));
        CK(launch_validate(c->d_job, job.n_pairs, c->d_ctrs + C_NBAD, s));
        tk->launches += 1;
    }
    if (job.n_pairs) {
        if (c->mode == XDROP_MODE_PLAIN) rc = run_plain(c, tk, job);
        else rc = run_batched(c, tk);
        if (rc) return rc;
    }
    CK(cudaEventRecord(tk->ev_end, s));
    CK(cudaMemcpyAsync(tk->h_ctrs, c->d_ctrs, C_WORDS * 4, cudaMemcpyDeviceToHost, s));
    if (!tk->device_submit && tk->n_pairs)
        CK(cudaMemcpyAsync(tk->h_out, job.out, tk->n_pairs * sizeof(xdrop_result),
                           cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(tk->ev_done, s));
    return XDROP_OK;
}

// Batched mode over resident reads when the pair table does not fit the
// device memory budget: the pairs stream through in chunks of `chunk`
// pairs (host -> device, one replay of the same CUDA graph, results back),
// all in stream order on the context's stream.  tk->h_job has one pinned
// Job slot per chunk, so every chunk's descriptor copy has its own source.
int launch_ticket_chunked(xdrop_ctx *c, Ticket *tk, const xdrop_pair *h_pairs, size_t n_pairs,
                          size_t chunk, const Job &base, char *d_pairs, char *d_out,
                          uint32_t maxlen)
{
    cudaStream_t s = c->stream;
    int rc;
    if ((rc = ensure_scratch(c, 2 * chunk, maxlen))) return rc;
    CK(cudaEventRecord(tk->ev_begin, s));
    size_t k = 0;
    for (size_t p0 = 0; p0 < n_pairs; p0 += chunk, ++k) {
        const size_t np = std::min(chunk, n_pairs - p0);
        CK(cudaMemcpyAsync(d_pairs, h_pairs + p0, np * sizeof(xdrop_pair), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(d_out, 0, np * sizeof(xdrop_result), s));
        Job job = base;
        job.pairs = (const Pair *)d_pairs;
        job.n_pairs = np;
        job.out = (int32_t *)d_out;
        tk->h_job[k] = job;
        CK(cudaMemcpyAsync(c->d_job, &tk->h_job[k], sizeof(Job), cudaMemcpyHostToDevice, s));
        if (k == 0) {  // first tile: as for an unchunked submit
            if ((rc = pick_tile(c, tk, job, &c->tile0))) return rc;
        }
        if ((rc = run_batched(c, tk))) return rc;
        CK(cudaMemcpyAsync(tk->h_out + p0, d_out, np * sizeof(xdrop_result), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(tk->ev_end, s));
    CK(cudaMemcpyAsync(tk->h_ctrs, c->d_ctrs, C_WORDS * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(tk->ev_done, s));
    return XDROP_OK;
}

int new_ticket(xdrop_ctx *c, size_t n_pairs, bool device_submit, Ticket **out, size_t n_jobs = 1)
{
    Ticket *tk = new Ticket();
    tk->device_submit = device_submit;
    tk->n_pairs = n_pairs;
    size_t pin = align_up(sizeof(Job) * std::max<size_t>(n_jobs, 1)) + align_up(C_WORDS * 4) +
                 (device_submit ? 0 : align_up(n_pairs * sizeof(xdrop_result)));
    cudaError_t e = cudaHostAlloc(&tk->h_pinned, pin, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreate(&tk->ev_begin);
    if (e == cudaSuccess) e = cudaEventCreate(&tk->ev_end);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&tk->ev_done, cudaEventBlockingSync);
    if (e != cudaSuccess) {
        free_ticket(c, tk);
        return fail(XDROP_ECUDA, "ticket setup: %s", cudaGetErrorString(e));
    }
    char *p = (char *)tk->h_pinned;
    tk->h_job = (Job *)p;
    p += align_up(sizeof(Job) * std::max<size_t>(n_jobs, 1));
    tk->h_ctrs = (uint32_t *)p;
    p += align_up(C_WORDS * 4);
    tk->h_out = device_submit ? nullptr : (xdrop_result *)p;
    *out = tk;
    return XDROP_OK;
}

}  // namespace

extern "C" {

int xdrop_init(xdrop_ctx **out, int device, size_t budget, uint32_t flags)
{
    if (!out) return fail(XDROP_EINVAL, "out is NULL");
    *out = nullptr;
    if (flags > XDROP_MODE_SERVE) return fail(XDROP_EINVAL, "unknown flags 0x%x", flags);
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(XDROP_EINVAL, "no CUDA device %d", device);
    CK(cudaSetDevice(device));
    xdrop_ctx *c = new xdrop_ctx();
    c->device = device;
    c->budget = budget;
    c->mode = flags;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_job, sizeof(Job));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ctrs, C_WORDS * 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_ctrs, 0, C_WORDS * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_main0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_main1);
    if (e != cudaSuccess) {
        xdrop_free(c);
        return fail(XDROP_ECUDA, "init: %s", cudaGetErrorString(e));
    }
    c->used = sizeof(Job) + C_WORDS * 4;
    c->wide_grid = 2 * c->sm_count;
    *out = c;
    return XDROP_OK;
}

int xdrop_submit(xdrop_ctx *c, const uint32_t *packed, const uint64_t *read_off,
                 const uint32_t *read_len, uint32_t n_reads, const xdrop_pair *pairs,
                 size_t n_pairs, const xdrop_scoring *s, xdrop_result *out, xdrop_ticket *t)
{
    if (!c || !t) return fail(XDROP_EINVAL, "context or ticket pointer is NULL");
    int rc = validate_scoring(s);
    if (rc) return rc;
    if (n_pairs && (!pairs || !out || !read_off || !read_len || !packed))
        return fail(XDROP_EINVAL, "NULL input array");
    if (2 * (uint64_t)n_pairs >= ((uint64_t)1 << 32))
        return fail(XDROP_EINVAL, "too many pairs in one submit");
    // Host-side validation of every read and pair.
    uint64_t n_words = 0;
    uint32_t maxlen = 0;
    for (uint32_t r = 0; r < n_reads; ++r) {
        if (read_off[r] & 15) return fail(XDROP_EINVAL, "read %u offset not a multiple of 16", r);
        if ((int64_t)read_len[r] >= LEN_LIMIT) return fail(XDROP_EINVAL, "read %u too long", r);
        n_words = std::max<uint64_t>(n_words, (read_off[r] + read_len[r] + 15) / 16);
        maxlen = std::max(maxlen, read_len[r]);
    }
    if (n_words * 16 >= ((uint64_t)1 << 32)) return fail(XDROP_EINVAL, "packed buffer too large");
    const Scoring sc{s->match, s->mismatch, s->gap, s->x};
    bool any_rc = false;  // reverse-strand pairs: store the reverse complements too
    for (size_t p = 0; p < n_pairs; ++p) {
        const Pair &pr = *(const Pair *)&pairs[p];
        if (!pair_ok(pr, n_reads, read_len, read_off, (int64_t)n_words, sc, true))
            return fail(XDROP_EINVAL, "pair %zu is invalid (read id, seed or length limit)", p);
        any_rc |= (pr.b & kPairRC) != 0;
    }
    const uint64_t pk_words = any_rc ? 2 * n_words : n_words;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    Ticket *tk = nullptr;
    if ((rc = new_ticket(c, n_pairs, false, &tk))) return rc;
    tk->out = out;
    // One device allocation for the inputs and results of this ticket.
    size_t o_packed = 0, o_off = align_up(std::max<uint64_t>(pk_words, 1) * 4);
    size_t o_len = o_off + align_up((size_t)std::max(n_reads, 1u) * 8);
    size_t o_pairs = o_len + align_up((size_t)std::max(n_reads, 1u) * 4);
    size_t o_out = o_pairs + align_up(std::max<size_t>(n_pairs, 1) * sizeof(xdrop_pair));
    size_t bytes = o_out + align_up(std::max<size_t>(n_pairs, 1) * sizeof(xdrop_result));
    if (c->budget && c->used + bytes > c->budget) {
        free_ticket(c, tk);
        return fail(c->tickets.empty() ? XDROP_ENOMEM : XDROP_EBUSY,
                    "device memory budget exceeded (%zu bytes needed)", bytes);
    }
    cudaError_t e = cudaMalloc(&tk->d_mem, bytes);
    if (e != cudaSuccess) {
        free_ticket(c, tk);
        return fail(XDROP_ECUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    tk->d_bytes = bytes;
    c->used += bytes;
    char *d = (char *)tk->d_mem;
    cudaStream_t st = c->stream;
    e = cudaSuccess;
    if (n_words) e = cudaMemcpyAsync(d + o_packed, packed, n_words * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_reads)
        e = cudaMemcpyAsync(d + o_off, read_off, (size_t)n_reads * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_reads)
        e = cudaMemcpyAsync(d + o_len, read_len, (size_t)n_reads * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pairs)
        e = cudaMemcpyAsync(d + o_pairs, pairs, n_pairs * sizeof(xdrop_pair),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pairs)
        e = cudaMemsetAsync(d + o_out, 0, n_pairs * sizeof(xdrop_result), st);
    if (e == cudaSuccess && any_rc) {
        e = launch_revcomp((const uint32_t *)(d + o_packed), (int64_t)n_words,
                           (const uint64_t *)(d + o_off), (const uint32_t *)(d + o_len), n_reads,
                           (uint32_t *)(d + o_packed) + n_words, st);
        if (e == cudaSuccess) tk->launches += 1;
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_ticket(c, tk);
        return fail(XDROP_ECUDA, "input copy: %s", cudaGetErrorString(e));
    }
    Job job{};
    job.packed = (const uint32_t *)(d + o_packed);
    job.n_words = (int64_t)std::max<uint64_t>(pk_words, 1);
    job.rc_off = any_rc ? (int64_t)(16 * n_words) : 0;
    job.read_off = (const uint64_t *)(d + o_off);
    job.read_len = (const uint32_t *)(d + o_len);
    job.n_reads = n_reads;
    job.pairs = (const Pair *)(d + o_pairs);
    job.n_pairs = n_pairs;
    job.sc = sc;
    job.out = (int32_t *)(d + o_out);
    job.cells = nullptr;
    if ((rc = launch_ticket(c, tk, job, maxlen))) {
        cudaStreamSynchronize(st);
        free_ticket(c, tk);
        return rc;
    }
    tk->id = c->next_id++;
    c->tickets[tk->id] = tk;
    *t = tk->id;
    return XDROP_OK;
}

int xdrop_submit_device(xdrop_ctx *c, const uint32_t *packed, uint64_t n_words,
                        const uint64_t *read_off, const uint32_t *read_len, uint32_t n_reads,
                        const xdrop_pair *pairs, size_t n_pairs, const xdrop_scoring *s,
                        xdrop_result *out, xdrop_ticket *t)
{
    if (!c || !t) return fail(XDROP_EINVAL, "context or ticket pointer is NULL");
    int rc = validate_scoring(s);
    if (rc) return rc;
    if (n_pairs && (!pairs || !out || !read_off || !read_len || !packed || !n_words))
        return fail(XDROP_EINVAL, "NULL input array");
    if (2 * (uint64_t)n_pairs >= ((uint64_t)1 << 32))
        return fail(XDROP_EINVAL, "too many pairs in one submit");
    if (n_words * 16 >= ((uint64_t)1 << 32)) return fail(XDROP_EINVAL, "packed buffer too large");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    // Largest read (sizes the unbounded tier); cached per read_len array.
    uint32_t maxlen = c->maxlen_val;
    if (n_pairs && (read_len != c->maxlen_ptr || n_reads != c->maxlen_n)) {
        CK(cudaMemsetAsync(c->d_ctrs + C_MAXLEN, 0, 4, c->stream));
        CK(launch_max_len(read_len, n_reads, c->d_ctrs + C_MAXLEN, c->stream));
        CK(cudaMemcpyAsync(&maxlen, c->d_ctrs + C_MAXLEN, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->maxlen_ptr = read_len;
        c->maxlen_n = n_reads;
        c->maxlen_val = maxlen;
    }
    Ticket *tk = nullptr;
    if ((rc = new_ticket(c, n_pairs, true, &tk))) return rc;
    Job job{};
    job.packed = packed;
    job.n_words = (int64_t)n_words;
    job.read_off = read_off;
    job.read_len = read_len;
    job.n_reads = n_reads;
    job.pairs = (const Pair *)pairs;
    job.n_pairs = n_pairs;
    job.sc = Scoring{s->match, s->mismatch, s->gap, s->x};
    job.out = (int32_t *)out;
    job.cells = nullptr;
    if ((rc = launch_ticket(c, tk, job, maxlen))) {
        cudaStreamSynchronize(c->stream);
        free_ticket(c, tk);
        return rc;
    }
    tk->id = c->next_id++;
    c->tickets[tk->id] = tk;
    *t = tk->id;
    return XDROP_OK;
}

int xdrop_sync(xdrop_ctx *c, xdrop_ticket t, int64_t timeout_ns)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    if (t & kServeTicket) {
        if (!c->srv) return fail(XDROP_EINVAL, "unknown ticket %llu", (unsigned long long)t);
        std::string err;
        const int rc = xd::server_sync(c->srv, t & ~kServeTicket, timeout_ns, err);
        return rc ? fail(rc, "%s", err.c_str()) : XDROP_OK;
    }
    Ticket *tk = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->tickets.find(t);
        if (it == c->tickets.end()) return fail(XDROP_EINVAL, "unknown ticket %llu", (unsigned long long)t);
        tk = it->second;
    }
    CK(cudaSetDevice(c->device));
    if (timeout_ns < 0) {
        CK(cudaEventSynchronize(tk->ev_done));
    } else {
        auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            cudaError_t q = cudaEventQuery(tk->ev_done);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return fail(XDROP_ECUDA, "sync: %s", cudaGetErrorString(q));
            auto el = std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ns) return fail(XDROP_ETIMEDOUT, "ticket %llu not done", (unsigned long long)t);
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->tickets.find(t);
    if (it == c->tickets.end()) return fail(XDROP_EINVAL, "ticket %llu already synced", (unsigned long long)t);
    c->tickets.erase(it);
    if (!tk->device_submit && tk->n_pairs)
        memcpy(tk->out, tk->h_out, tk->n_pairs * sizeof(xdrop_result));
    float ms = 0.f, ms_main = 0.f;
    if (cudaEventElapsedTime(&ms, tk->ev_begin, tk->ev_end) != cudaSuccess) ms = 0.f;
    if (tk->graph_replays && cudaEventElapsedTime(&ms_main, c->ev_main0, c->ev_main1) != cudaSuccess)
        ms_main = 0.f;
    (void)cudaGetLastError();  // a failed timing query must not leak into later checks
    xdrop_stats st = {};
    st.kernel_ms = ms;
    st.main_kernel_ms = ms_main;
    st.tasks = 2 * (uint64_t)tk->n_pairs;
    st.overflow_tasks = tk->h_ctrs[C_SPILL0];
    st.wide_tasks = next_tile_after(c->tile0).width() >= 512 ? tk->h_ctrs[C_SPILL1]
                                                              : tk->h_ctrs[C_SPILL2];
    st.launches = tk->launches;
    st.graph_replays = tk->graph_replays;
    st.tile_lanes = c->tile0.lanes;
    st.tile_cells = c->tile0.c | (c->tile0.packed ? XDROP_TILE_PACKED16 : 0);
    c->last = st;
    const uint32_t nbad = tk->device_submit ? tk->h_ctrs[C_NBAD] : 0;
    free_ticket(c, tk);
    if (nbad) return fail(XDROP_EINVAL, "%u pairs failed validation (status set)", nbad);
    return XDROP_OK;
}

void xdrop_free(xdrop_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->srv) xd::server_destroy(c->srv);
    cudaFree(c->r_packed.p);
    cudaFree(c->r_off.p);
    cudaFree(c->r_len.p);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &kv : c->tickets) free_ticket(c, kv.second);
    c->tickets.clear();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->ev_main0) cudaEventDestroy(c->ev_main0);
    if (c->ev_main1) cudaEventDestroy(c->ev_main1);
    cudaFree(c->order.p);
    cudaFree(c->plain_ctl.p);
    for (auto &s : c->spill) cudaFree(s.p);
    cudaFree(c->wide.p);
    cudaFree(c->d_job);
    cudaFree(c->d_ctrs);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *xdrop_last_error(xdrop_ctx *c)
{
    (void)c;
    return g_err.c_str();
}

void *xdrop_stream(xdrop_ctx *c) { return c ? (void *)c->stream : nullptr; }

int xdrop_get_stats(xdrop_ctx *c, xdrop_stats *st)
{
    if (!c || !st) return fail(XDROP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    *st = c->last;
    st->device_bytes = c->used;
    return XDROP_OK;
}

int xdrop_load_reads(xdrop_ctx *c, const uint32_t *packed, const uint64_t *read_off,
                     const uint32_t *read_len, uint32_t n_reads)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    if (n_reads && (!packed || !read_off || !read_len)) return fail(XDROP_EINVAL, "NULL input array");
    uint64_t n_words = 0;
    uint32_t maxlen = 0;
    for (uint32_t r = 0; r < n_reads; ++r) {
        if (read_off[r] & 15) return fail(XDROP_EINVAL, "read %u offset not a multiple of 16", r);
        if ((int64_t)read_len[r] >= LEN_LIMIT) return fail(XDROP_EINVAL, "read %u too long", r);
        n_words = std::max<uint64_t>(n_words, (read_off[r] + read_len[r] + 15) / 16);
        maxlen = std::max(maxlen, read_len[r]);
    }
    if (n_words * 16 >= ((uint64_t)1 << 32)) return fail(XDROP_EINVAL, "packed buffer too large");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    if (c->srv) {  // waits for the serving requests in flight
        xd::server_destroy(c->srv);
        c->srv = nullptr;
    }
    CK(cudaStreamSynchronize(c->stream));
    int rc;
    const uint64_t nw = std::max<uint64_t>(n_words, 1);
    // the reads, then their reverse complements (reverse-strand pairs)
    if ((rc = dev_alloc(c, c->r_packed, 2 * nw * 4))) return rc;
    if ((rc = dev_alloc(c, c->r_off, std::max<size_t>(n_reads, 1) * 8))) return rc;
    if ((rc = dev_alloc(c, c->r_len, std::max<size_t>(n_reads, 1) * 4))) return rc;
    if (n_words) CK(cudaMemcpy(c->r_packed.p, packed, n_words * 4, cudaMemcpyHostToDevice));
    if (n_reads) {
        CK(cudaMemcpy(c->r_off.p, read_off, (size_t)n_reads * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->r_len.p, read_len, (size_t)n_reads * 4, cudaMemcpyHostToDevice));
        CK(launch_revcomp((const uint32_t *)c->r_packed.p, (int64_t)nw, (const uint64_t *)c->r_off.p,
                          (const uint32_t *)c->r_len.p, n_reads, (uint32_t *)c->r_packed.p + nw,
                          c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->h_off.assign(read_off, read_off + n_reads);
    c->h_len.assign(read_len, read_len + n_reads);
    c->r_words = nw;
    c->r_n = n_reads;
    c->r_maxlen = maxlen;
    c->have_reads = true;
    ++c->reads_gen;
    if ((rc = ensure_scratch(c, 0, maxlen))) return rc;
    if (c->mode == XDROP_MODE_SERVE) {
        xd::ResidentReads rr;
        rr.packed = (const uint32_t *)c->r_packed.p;
        rr.n_words = (int64_t)(2 * nw);
        rr.rc_off = (int64_t)(16 * nw);
        rr.read_off = (const uint64_t *)c->r_off.p;
        rr.read_len = (const uint32_t *)c->r_len.p;
        rr.n_reads = n_reads;
        std::string err;
        // Packed 4x16 unless a tile was forced; requests whose scoring does
        // not fit 16 bits run on the serving kernel's 32-bit second tier.
        const Tile t = c->forced.lanes ? c->forced : Tile{4, 16, true};
        c->srv = xd::server_create(c->device, c->sm_count, c->budget, t, rr, c->h_len.data(),
                                   (int32_t *)c->wide.p, c->wide_per_cta, c->wide_grid,
                                   c->serve_idle_ns, err);
        if (!c->srv) return fail(XDROP_ECUDA, "%s", err.c_str());
    }
    return XDROP_OK;
}

int xdrop_submit_pairs(xdrop_ctx *c, const xdrop_pair *pairs, size_t n_pairs,
                       const xdrop_scoring *s, xdrop_result *out, xdrop_ticket *t)
{
    if (!c || !t) return fail(XDROP_EINVAL, "context or ticket pointer is NULL");
    int rc = validate_scoring(s);
    if (rc) return rc;
    if (n_pairs && (!pairs || !out)) return fail(XDROP_EINVAL, "NULL input array");
    if (2 * (uint64_t)n_pairs >= ((uint64_t)1 << 32))
        return fail(XDROP_EINVAL, "too many pairs in one submit");
    const Scoring sc{s->match, s->mismatch, s->gap, s->x};
    xd::Server *srv = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->have_reads) return fail(XDROP_EINVAL, "no resident reads (xdrop_load_reads)");
        for (size_t p = 0; p < n_pairs; ++p) {
            const Pair &pr = *(const Pair *)&pairs[p];
            if (!pair_ok(pr, c->r_n, c->h_len.data(), c->h_off.data(), (int64_t)c->r_words, sc, true))
                return fail(XDROP_EINVAL, "pair %zu is invalid (read id, seed or length limit)", p);
        }
        srv = c->srv;
    }
    if (srv) {
        std::string err;
        uint64_t id = 0;
        rc = xd::server_submit(srv, pairs, n_pairs, sc, out, &id, err);
        if (rc) return fail(rc, "%s", err.c_str());
        *t = id | kServeTicket;
        return XDROP_OK;
    }
    // not serving: an ordinary ticket over the resident reads, streamed in
    // chunks when the pair table does not fit the device memory budget
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    const size_t per_pair = sizeof(xdrop_pair) + sizeof(xdrop_result) + 2 * 4 * 4;  // + task scratch
    size_t chunk = std::max<size_t>(n_pairs, 1);
    if (c->budget && c->mode != XDROP_MODE_PLAIN) {
        const size_t scratch_now = c->order.cap + c->spill[0].cap + c->spill[1].cap + c->spill[2].cap;
        const size_t fixed = c->used - scratch_now + 4 * kAlign;
        if (c->budget <= fixed + 1024 * per_pair)
            return fail(c->tickets.empty() ? XDROP_ENOMEM : XDROP_EBUSY,
                        "device memory budget too small for resident reads plus a chunk");
        if (!c->tickets.empty() && c->budget < c->used + chunk * per_pair)
            return fail(XDROP_EBUSY, "device memory budget taken by work in flight");
        const size_t fit = (c->budget - fixed) / per_pair;
        if (fit < chunk) {
            chunk = fit;
            // scratch sized for this chunk must not stay larger from before
            for (DevBuf *b : {&c->order, &c->spill[0], &c->spill[1], &c->spill[2]}) {
                if (b->cap > 2 * chunk * 4) {
                    CK(cudaStreamSynchronize(c->stream));
                    cudaFree(b->p);
                    c->used -= b->cap;
                    b->p = nullptr;
                    b->cap = 0;
                    c->scratch_version += 1;
                }
            }
        }
    }
    const size_t n_chunks = (std::max<size_t>(n_pairs, 1) + chunk - 1) / chunk;
    Ticket *tk = nullptr;
    if ((rc = new_ticket(c, n_pairs, false, &tk, n_chunks))) return rc;
    tk->out = out;
    const size_t o_out = align_up(chunk * sizeof(xdrop_pair));
    const size_t bytes = o_out + align_up(chunk * sizeof(xdrop_result));
    if (c->budget && c->mode == XDROP_MODE_PLAIN && c->used + bytes > c->budget) {
        free_ticket(c, tk);
        return fail(c->tickets.empty() ? XDROP_ENOMEM : XDROP_EBUSY,
                    "device memory budget exceeded (%zu bytes needed)", bytes);
    }
    cudaError_t e = cudaMalloc(&tk->d_mem, bytes);
    if (e != cudaSuccess) {
        free_ticket(c, tk);
        return fail(XDROP_ECUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    tk->d_bytes = bytes;
    c->used += bytes;
    char *d = (char *)tk->d_mem;
    if (n_chunks > 1) {
        Job base{};
        base.packed = (const uint32_t *)c->r_packed.p;
        base.n_words = (int64_t)(2 * c->r_words);
        base.rc_off = (int64_t)(16 * c->r_words);
        base.read_off = (const uint64_t *)c->r_off.p;
        base.read_len = (const uint32_t *)c->r_len.p;
        base.n_reads = c->r_n;
        base.sc = sc;
        if ((rc = launch_ticket_chunked(c, tk, pairs, n_pairs, chunk, base, d, d + o_out,
                                        c->r_maxlen))) {
            cudaStreamSynchronize(c->stream);
            free_ticket(c, tk);
            return rc;
        }
        tk->id = c->next_id++;
        c->tickets[tk->id] = tk;
        *t = tk->id;
        return XDROP_OK;
    }
    if (n_pairs) e = cudaMemcpyAsync(d, pairs, n_pairs * sizeof(xdrop_pair), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_pairs)
        e = cudaMemsetAsync(d + o_out, 0, n_pairs * sizeof(xdrop_result), c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        free_ticket(c, tk);
        return fail(XDROP_ECUDA, "input copy: %s", cudaGetErrorString(e));
    }
    Job job{};
    job.packed = (const uint32_t *)c->r_packed.p;
    job.n_words = (int64_t)(2 * c->r_words);
    job.rc_off = (int64_t)(16 * c->r_words);
    job.read_off = (const uint64_t *)c->r_off.p;
    job.read_len = (const uint32_t *)c->r_len.p;
    job.n_reads = c->r_n;
    job.pairs = (const Pair *)d;
    job.n_pairs = n_pairs;
    job.sc = sc;
    job.out = (int32_t *)(d + o_out);
    if ((rc = launch_ticket(c, tk, job, c->r_maxlen))) {
        cudaStreamSynchronize(c->stream);
        free_ticket(c, tk);
        return rc;
    }
    tk->id = c->next_id++;
    c->tickets[tk->id] = tk;
    *t = tk->id;
    return XDROP_OK;
}

int xdrop_get_serve_stats(xdrop_ctx *c, xdrop_serve_stats *st)
{
    if (!c || !st) return fail(XDROP_EINVAL, "NULL argument");
    memset(st, 0, sizeof(*st));
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->srv) {
        const xd::ServerStats s = xd::server_stats(c->srv);
        st->requests_done = s.requests_done;
        st->wide_passes = s.wide_passes;
        st->relaunches = s.relaunches;
        st->max_in_flight = s.max_in_flight;
        st->admission_waits = s.admission_waits;
        st->published = s.published;
        st->consumed = s.consumed;
        st->spill_reserved = s.spill_reserved;
        st->spill_taken = s.spill_taken;
        st->ring_warps = s.ring_warps;
        st->idle_exits = s.idle_exits;
        st->help_sessions = s.help_sessions;
        st->surplus_counts = s.surplus_counts;
    }
    return XDROP_OK;
}

int xdrop_set_serve_idle(xdrop_ctx *c, uint64_t idle_ns)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    c->serve_idle_ns = idle_ns;
    if (c->srv) xd::server_set_idle_ns(c->srv, idle_ns);
    return XDROP_OK;
}

int xdrop_find_candidates(xdrop_ctx *c, const xdrop_kmer_params *p, xdrop_pair *pairs,
                          uint32_t *shared, size_t cap, size_t *n)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    if (!p || !n || (cap && !pairs)) return fail(XDROP_EINVAL, "NULL argument");
    if (p->k < 1 || p->k > xs::kMaxK || p->stride < 1 || p->lo < 1 || p->lo > p->hi ||
        p->hi > xs::kMaxHi ||
        (p->flags & ~XDROP_SEEDS_SORT))
        return fail(XDROP_EINVAL,
                    "k-mer parameters out of range (k %u, stride %u, lo %u, hi %u, flags %u)", p->k,
                    p->stride, p->lo, p->hi, p->flags);
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->have_reads) return fail(XDROP_EINVAL, "no resident reads (xdrop_load_reads)");
    CK(cudaSetDevice(c->device));
    const auto key = std::make_tuple(p->k, p->stride, p->lo, p->hi, p->flags);
    if (c->cand_gen != c->reads_gen || c->cand_params != key) {
        c->cand_gen = 0;
        const size_t left = c->budget ? (c->budget > c->used ? c->budget - c->used : 1) : 0;
        std::string err;
        const int rc = find_candidates(c->stream, c->sm_count, left, (const uint32_t *)c->r_packed.p,
                                       (const uint64_t *)c->r_off.p, (const uint32_t *)c->r_len.p,
                                       c->r_n, c->h_len.data(), p->k, p->stride, p->lo, p->hi,
                                       p->flags, c->cand_pairs, c->cand_shared, c->seed_stats,
                                       err);
        if (rc) return fail(rc, "%s", err.c_str());
        c->cand_params = key;
        c->cand_gen = c->reads_gen;
    }
    const size_t total = c->cand_pairs.size(), m = std::min(cap, total);
    if (m) {
        memcpy(pairs, c->cand_pairs.data(), m * sizeof(xdrop_pair));
        if (shared) memcpy(shared, c->cand_shared.data(), m * sizeof(uint32_t));
    }
    *n = total;
    return XDROP_OK;
}

int xdrop_accept_device(xdrop_ctx *c, const xdrop_pair *pairs, const xdrop_result *results,
                        size_t n, const uint32_t *read_len, uint32_t n_reads,
                        const xdrop_accept_params *p, uint8_t *accept)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    if (!p) return fail(XDROP_EINVAL, "NULL parameters");
    if (p->error_e4 > 10000 || p->delta_e4 > 10000)
        return fail(XDROP_EINVAL, "error_e4 and delta_e4 must be at most 10000");
    if (n == 0) return XDROP_OK;
    if (!pairs || !results || !read_len || !accept) return fail(XDROP_EINVAL, "NULL array");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    CK(launch_accept((const Pair *)pairs, (const int32_t *)results, read_len, n_reads, n,
                     p->match, p->mismatch, p->error_e4, p->delta_e4, accept, c->stream));
    return XDROP_OK;
}

int xdrop_get_seed_stats(xdrop_ctx *c, xdrop_seed_stats *st)
{
    if (!c || !st) return fail(XDROP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    memset(st, 0, sizeof *st);
    st->ms = c->seed_stats.ms;
    st->occurrences = c->seed_stats.occurrences;
    st->runs = c->seed_stats.runs;
    st->candidates = c->seed_stats.candidates;
    st->product = c->seed_stats.product;
    st->pad = 0;
    st->nonzeros = c->seed_stats.nonzeros;
    return XDROP_OK;
}

int xdrop_best_seeds_device(xdrop_ctx *c, const xdrop_pair *pairs, const xdrop_result *results,
                            size_t n, int32_t match, uint32_t *best)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    if (n == 0) return XDROP_OK;
    if (!pairs || !results || !best) return fail(XDROP_EINVAL, "NULL array");
    if ((uint64_t)n >= ((uint64_t)1 << 31)) return fail(XDROP_EINVAL, "too many records");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    CK(launch_best_seeds((const Pair *)pairs, (const int32_t *)results, n, match, best, c->stream));
    return XDROP_OK;
}

int xdrop_set_tile(xdrop_ctx *c, int lanes, int cells)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (lanes == 0) {
        c->forced = Tile{0, 0};
        return XDROP_OK;
    }
    const bool packed = (cells & XDROP_TILE_PACKED16) != 0;
    cells &= ~XDROP_TILE_PACKED16;
    if (packed) {
        for (const Tile &t : kPackedTiles)
            if (t.lanes == lanes && t.c == cells) {
                c->forced = t;
                return XDROP_OK;
            }
    } else {
        for (const Tile &t : kTuneTiles)
            if (t.lanes == lanes && t.c == cells) {
                c->forced = t;
                return XDROP_OK;
            }
    }
    return fail(XDROP_EINVAL, "no %dx%d%s tile", lanes, cells, packed ? " packed" : "");
}

int xdrop_last_spills(xdrop_ctx *c, uint32_t *dst, size_t cap, size_t *n)
{
    if (!c || !n || (cap && !dst)) return fail(XDROP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    uint32_t cnt = 0;
    CK(cudaMemcpy(&cnt, c->d_ctrs + C_SPILL0, 4, cudaMemcpyDeviceToHost));
    *n = cnt;
    size_t k = std::min<size_t>(cap, cnt);
    if (k) CK(cudaMemcpy(dst, c->spill[0].p, k * 4, cudaMemcpyDeviceToHost));
    return XDROP_OK;
}

int xdrop_count_cells_device(xdrop_ctx *c, const uint32_t *packed, uint64_t n_words,
                             const uint64_t *read_off, const uint32_t *read_len,
                             uint32_t n_reads, const xdrop_pair *pairs, size_t n_pairs,
                             const xdrop_scoring *s, int64_t *cells)
{
    if (!c) return fail(XDROP_EINVAL, "context is NULL");
    int rc = validate_scoring(s);
    if (rc) return rc;
    if (n_pairs == 0) return XDROP_OK;
    if (!pairs || !cells || !read_off || !read_len || !packed || !n_words)
        return fail(XDROP_EINVAL, "NULL input array");
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    CK(cudaMemsetAsync(c->d_ctrs + C_MAXLEN, 0, 4, st));
    CK(launch_max_len(read_len, n_reads, c->d_ctrs + C_MAXLEN, st));
    uint32_t maxlen = 0;
    CK(cudaMemcpyAsync(&maxlen, c->d_ctrs + C_MAXLEN, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((rc = ensure_scratch(c, 2 * n_pairs, maxlen))) return rc;
    Job job{};
    job.packed = packed;
    job.n_words = (int64_t)n_words;
    job.read_off = read_off;
    job.read_len = read_len;
    job.n_reads = n_reads;
    job.pairs = (const Pair *)pairs;
    job.n_pairs = n_pairs;
    job.sc = Scoring{s->match, s->mismatch, s->gap, s->x};
    job.out = nullptr;
    job.cells = cells;
    CK(cudaMemcpyAsync(c->d_job, &job, sizeof(Job), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->d_ctrs, 0, C_NBAD * 4, st));
    CK(cudaMemsetAsync(cells, 0, 2 * n_pairs * 8, st));
    for (uint64_t t0 = 0; t0 < 2 * n_pairs; t0 += (1u << 24)) {
        uint32_t nt = (uint32_t)std::min<uint64_t>(1u << 24, 2 * n_pairs - t0);
        CK(launch_window(Tile{32, 16}, true, c->d_job, (uint32_t)t0, nt, spill_of(c, 0), st));
    }
    CK(launch_wide(true, c->wide_grid, c->d_job, spill_of(c, 0), (int32_t *)c->wide.p,
                   c->wide_per_cta, st));
    CK(cudaStreamSynchronize(st));
    return XDROP_OK;
}

}  // extern "C"
