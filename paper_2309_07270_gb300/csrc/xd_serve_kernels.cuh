// Device side of the serving mode: the control block, the ring and
// spill-queue task sources, and the serving kernels of both first-tier
// forms (32-bit and packed 16-bit).
#pragma once
#include "xd_device.cuh"
#include "xd_lockstep16.cuh"

namespace xd {

// Control block of the serving kernel (device memory).  The host-written,
// read-mostly words share one line; each device-hot counter has its own.
struct ServeCtl {
    unsigned long long published;   // ring entries the host has published (host writes)
    unsigned long long idle_ns;     // a waiting warp leaves after this long (hang guard)
    unsigned int stop;              // host: leave once idle
    unsigned int yield;             // host: take no more tasks, leave when drained
    unsigned int ring_alive;        // warps still running (host sets)
    unsigned int abort;             // host: leave now, abandoning tasks (teardown)
    unsigned int idle_exits;        // first-tier warps that left on the idle bound
    alignas(128) unsigned long long consumed;    // ring entries taken (device CAS)
    alignas(128) unsigned long long spill_tail;  // second-tier queue: entries reserved
    alignas(128) unsigned long long spill_head;  // second-tier queue: entries taken
    alignas(128) unsigned int helpers;           // warps registered to serve the queue
    unsigned int help_sessions;                  // registrations, over all launches
    unsigned int surplus_counts;                 // extensions counted past their request's total
};

// ---------------------------------------------------------------------------
// Serving: a persistent kernel fed by a device ring of tasks that the host
// keeps appending to while the kernel runs (continuous batching).  Ring
// entry = slot << 24 | task; slot names the request's device Job.
//
// Every warp starts on the first-tier tile and ring tasks.  A task whose
// band outgrows that tile goes to a device spill queue, served by the next
// wider tile.  No warp is set aside for it: a ring warp that sees a backlog
// registers as a helper (at most one per kTasksPerHelper queued entries,
// and one as soon as there is any), lets its groups finish their ring
// tasks, serves the queue, and goes back to the ring once the queue has
// stayed empty for kHelpLingerNs.  A task too wide for the second tier is
// listed in its request (Job::spill_list, counted in ctr[1]) for the host's
// unbounded pass.
//
// Ring entries are claimed in chunks of kChunk when the backlog is deep
// (one CAS on `consumed`), their entries read before the CAS (see
// RingSrc), and what the claiming warp does not need at once goes to a
// shared-memory queue of its block, from which the block's warps take
// theirs.  A warp registers as a helper, or leaves for good, only after it
// found its own buffer and its block's queue empty, and a registered helper
// takes no more ring tasks (else a block that keeps refilling its queue
// would keep its helpers on the ring).  Only a warp that is not a helper
// moves entries into the queue, and it takes from the queue before it can
// register or leave, so the queue is always drained by a warp still on the
// ring.  The number of helpers is capped (ServeArgs::max_helpers) so that a
// burst of overflow cannot take every warp off the first tier.
//
// Every wait is bounded: ring warps leave after an idle limit (or on stop /
// yield), helpers once the queue stays empty; a queue entry that never
// appears sets the error word.
// ---------------------------------------------------------------------------
constexpr uint32_t kSpillQueueMask = (1u << 16) - 1;
constexpr int kEntrySpinLimit = 1 << 20;

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct ServeArgs {
    ServeCtl *ctl;
    const uint32_t *ring;
    uint32_t ring_mask;
    uint32_t *spq;             // spill queue, entry + 1 (0 = empty)
    const Job *slot_jobs;
    uint32_t *done;            // mapped host: per slot tag and wide count; [2*64] error word
    uint32_t n_slots;
    uint32_t max_helpers;      // most warps registered to serve the second tier at once
    uint32_t one;              // 1 (the packed loop's FMA-pipe adds, see fma_add)
};

// Count a finished task; the last one of a request publishes it.
__device__ __forceinline__ void serve_count(const ServeArgs &a, const Job *gj, const Job &J)
{
    __threadfence();
    const uint32_t f = atomicAdd(&J.ctr[0], 1u) + 1u;
    if ((uint64_t)f > 2 * J.n_pairs) atomicAdd(&a.ctl->surplus_counts, 1u);  // must stay 0
    if ((uint64_t)f == 2 * J.n_pairs) {
        const size_t sl = (size_t)(gj - a.slot_jobs);
        volatile uint32_t *d = a.done;
        d[2 * sl + 1] = *(volatile const uint32_t *)&J.ctr[1];
        __threadfence_system();
        d[2 * sl] = J.tag;
    }
}

// A task the second tier cannot hold: listed for the host's unbounded pass.
__device__ __forceinline__ void serve_list_wide(const ServeArgs &a, const Job *gj, const Job &J,
                                                uint32_t task)
{
    const uint32_t k = atomicAdd(&J.ctr[1], 1u);
    J.spill_list[k] = task;
    serve_count(a, gj, J);
}

constexpr unsigned long long kTasksPerHelper = 2;   // queued second-tier entries per helper warp
constexpr unsigned long long kHelpLingerNs = 100000;  // a helper leaves after this long with no task
constexpr unsigned long long kDeepBacklog = 16384;   // ring positions: claim chunks above this
constexpr int kChunk = 64;                           // ring entries per claim with a deep backlog

// The block's queue of ring entries in shared memory.  Control word:
// generation << 32 | filling << 31 | first << 16 | count.  A warp that claimed
// a chunk moves the entries it does not need now into an empty queue (taking
// it with the filling bit, writing the entries, then publishing a new
// generation); a warp takes entries by copying them first and then CASing
// the word, which succeeds only if no refill came between (the generation).
constexpr unsigned long long kQCount = 0xFFFFull;
constexpr unsigned long long kQFill = 1ull << 31;
struct BlockQueue {
    unsigned long long ctl;
    uint32_t ent[kChunk];
};

// Fetch state of one warp, kept by its lane 0 in shared memory (the band
// loops' registers hold none of it), and the warp's own entries.
struct WarpFetch {
    unsigned long long idle_since;  // first poll that found nothing (0: none)
    int own_head, own_n;            // entries of `ent` not yet handed out
    int backoff;                    // loop turns before the next poll
    int level;                      // backoff doubling level
    unsigned int helper;            // registered in ctl->helpers: finish the ring tasks, then help
    uint32_t ent[kChunk];
};

__device__ __forceinline__ void reset_fetch(WarpFetch *w, bool keep_helper)
{
    w->idle_since = 0;
    w->own_head = 0;
    w->own_n = 0;
    w->backoff = 0;
    w->level = 0;
    if (!keep_helper) w->helper = 0;
}

// Lane 0: move up to `want` entries of the block queue into the warp's own
// buffer.  Returns how many, 0 if the queue is empty (or being filled), or
// -1 if it still holds entries after losing every CAS race (the caller then
// decides nothing this turn, so no warp leaves the ring loop while its
// block's queue holds tasks).
__device__ __forceinline__ int take_block(BlockQueue *q, WarpFetch *w, int want)
{
    unsigned long long c = *(volatile unsigned long long *)&q->ctl;
    for (int tries = 0; tries < 16; ++tries) {
        const int cnt = (int)(c & kQCount);
        if (cnt == 0 || (c & kQFill)) return 0;
        const int first = (int)((c >> 16) & 0x7FFF);
        const int k = cnt < want ? cnt : want;
        __threadfence_block();
        for (int i = 0; i < k; ++i) w->ent[i] = ((volatile uint32_t *)q->ent)[first + i];
        const unsigned long long nc = (c & ~0x7FFFFFFFull) |
                                      ((unsigned long long)(first + k) << 16) |
                                      (unsigned long long)(cnt - k);
        const unsigned long long got = atomicCAS(&q->ctl, c, nc);
        if (got == c) {
            w->own_head = 0;
            w->own_n = k;
            return k;
        }
        c = got;
    }
    return -1;
}

// First-tier task source of a serving warp.
//
// Ring reuse.  The host reuses a ring slot once the tasks of requests that
// are done (a count, completed) leave room: position p + ring size is
// published only when p < completed.  completed never exceeds the device's
// claim counter `consumed`, so the entry of a position that is not claimed
// yet cannot be overwritten.  A warp therefore reads the entries of a chunk
// BEFORE its CAS on `consumed`: if the CAS succeeds, no one had claimed the
// chunk, and the entries read are the chunk's.  Buffers and the block queue
// hold entries, never positions, so a claimed task survives its slot's reuse.
struct RingSrc {
    static constexpr bool kCanAbort = true;  // teardown may stop the loop
    ServeArgs a;
    BlockQueue *bq;        // the block's queue (shared memory)
    WarpFetch *w;          // this warp's fetch state (lane 0 only) and entries
    bool leaving = false;  // stop, yield or the idle bound (not a switch to the second tier)

    // Register this warp as a second-tier helper if the backlog wants one
    // more (leader).
    __device__ __forceinline__ bool try_help(unsigned long long backlog)
    {
        unsigned long long need = (backlog + kTasksPerHelper - 1) / kTasksPerHelper;
        if (need > a.max_helpers) need = a.max_helpers;
        unsigned int h = *(volatile unsigned int *)&a.ctl->helpers;
        for (int tries = 0; tries < 4 && (unsigned long long)h < need; ++tries) {
            const unsigned int got = atomicCAS(&a.ctl->helpers, h, h + 1u);
            if (got == h) {
                atomicAdd(&a.ctl->help_sessions, 1u);
                w->helper = 1u;
                return true;
            }
            h = got;
        }
        return false;
    }

    // Warp-level fetch (see BatchSrc), run by every lane.  Lane 0 decides;
    // entries come from the warp's own buffer, the block queue, or a chunk
    // claimed by one CAS on `consumed` whose entries the whole warp reads
    // first.  A lost CAS race is retried; only an empty ring starts the
    // back-off.
    __device__ __forceinline__ int fetch_warp(unsigned needm, int lane, int gbase, unsigned gm,
                                              bool need, uint32_t &task, const Job *&gj)
    {
        enum { kNone = 0, kGrant = 1, kClaim = 2 };
        int status = 0;  // 1 granted, 0 none, -1 leave, -2 help the second tier
        int act = kNone;
        bool polled = false;  // lane 0 read the ring's published and claimed ends
        unsigned long long cons = 0, pub = 0;
        const int want = __popc(needm);
        if (lane == 0) {
            int kb = 0;
            if (w->own_n > 0) {
                act = kGrant;  // the warp's own entries first: no other warp can take them
            } else if (w->helper) {
                // registered: take no more ring tasks; the warp's groups finish
                // theirs and the warp serves the second tier
                status = -2;
            } else if ((kb = take_block(bq, w, want)) != 0) {
                if (kb > 0) act = kGrant;
            } else if (w->backoff > 0) {
                --w->backoff;
            } else {
                volatile ServeCtl *v = a.ctl;
                const unsigned long long backlog =
                    *(volatile unsigned long long *)&a.ctl->spill_tail -
                    *(volatile unsigned long long *)&a.ctl->spill_head;
                if (v->yield) {
                    status = -1;
                } else if (backlog > 0 && try_help(backlog)) {
                    status = -2;
                } else {
                    pub = v->published;
                    cons = *(volatile unsigned long long *)&a.ctl->consumed;
                    polled = true;
                    if (cons < pub) act = kClaim;
                }
            }
        }
        act = __shfl_sync(FULL, act, 0);
        // claim: read the chunk's entries, then CAS (see the struct comment)
        for (int tries = 0; tries < 4 && act == kClaim; ++tries) {
            cons = __shfl_sync(FULL, cons, 0);
            pub = __shfl_sync(FULL, pub, 0);
            const unsigned long long chunk =
                (pub - cons > kDeepBacklog) ? (unsigned long long)kChunk : (unsigned long long)want;
            const int kk = (int)((pub - cons < chunk) ? pub - cons : chunk);
            for (int i = lane; i < kk; i += 32)
                w->ent[i] = *(volatile const uint32_t *)&a.ring[(cons + (unsigned long long)i) &
                                                                a.ring_mask];
            __syncwarp();
            if (lane == 0) {
                const unsigned long long got =
                    atomicCAS(&a.ctl->consumed, cons, cons + (unsigned long long)kk);
                if (got == cons) {
                    w->own_head = 0;
                    w->own_n = kk;
                    act = kGrant;
                } else if (got >= pub) {
                    act = kNone;  // the rest was claimed meanwhile
                    cons = got;
                } else {
                    cons = got;
                }
            }
            act = __shfl_sync(FULL, act, 0);
        }
        int k = 0, first = 0;
        if (lane == 0) {
            if (act == kClaim) act = kNone;  // out of tries: again at the next turn
            if (act == kGrant) {
                status = 1;
                k = w->own_n < want ? w->own_n : want;
                first = w->own_head;
                w->own_head += k;
                w->own_n -= k;
                w->idle_since = 0;  // a task from any source ends an idle spell
                w->level = 0;
            } else if (status == 0 && polled && cons >= pub) {
                // nothing published to take
                volatile ServeCtl *v = a.ctl;
                const unsigned long long now = globaltimer_ns();
                if (w->idle_since == 0) w->idle_since = now;
                if (v->stop) {
                    status = -1;
                } else if (now - w->idle_since > v->idle_ns) {
                    status = -1;  // hang guard: counted for the host
                    atomicAdd(&a.ctl->idle_exits, 1u);
                }
                w->backoff = 1 << w->level;
                if (w->level < 6) ++w->level;
            }
        }
        // every lane takes part in the broadcasts before any lane returns
        status = __shfl_sync(FULL, status, 0);
        k = __shfl_sync(FULL, k, 0);
        first = __shfl_sync(FULL, first, 0);
        // with a deep backlog, offer the rest of a fresh chunk to the block
        if (status == 1) offer_rest(lane);
        if (status == -1) leaving = true;
        if (!need) return 0;
        if (status < 0) return -1;
        if (status == 0) return 0;
        const int rank = __popc(needm & ((1u << gbase) - 1u));
        if (rank >= k) return 0;
        const uint32_t entry = ((volatile uint32_t *)w->ent)[first + rank];
        task = entry & 0xffffffu;
        gj = &a.slot_jobs[entry >> 24];
        return 1;
    }

    // Move the warp's remaining own entries into the block queue if it is
    // empty (all lanes; lane 0 decides).  Entries handed out in this call
    // are read by their groups before the warp's next fetch, and the moved
    // ones lie after them in `ent`, so nothing in use is overwritten.
    __device__ __forceinline__ void offer_rest(int lane)
    {
        int n = 0, from = 0;
        unsigned long long gen = 0;
        if (lane == 0 && w->own_n > 0 && !w->helper) {  // a helper serves its own entries
            const unsigned long long c = *(volatile unsigned long long *)&bq->ctl;
            if ((c & kQCount) == 0 && !(c & kQFill) &&
                atomicCAS(&bq->ctl, c, (c & ~0xFFFFFFFFull) | kQFill) == c) {
                n = w->own_n;
                from = w->own_head;
                gen = c >> 32;
                w->own_n = 0;
            }
        }
        n = __shfl_sync(FULL, n, 0);
        if (n == 0) return;
        from = __shfl_sync(FULL, from, 0);
        for (int i = lane; i < n; i += 32) bq->ent[i] = w->ent[from + i];
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            *(volatile unsigned long long *)&bq->ctl = ((gen + 1ull) << 32) | (unsigned long long)n;
        }
        __syncwarp();
    }

    __device__ __forceinline__ void idle() { __nanosleep(2000); }
    __device__ __forceinline__ bool aborted() const
    {
        return *(volatile const unsigned int *)&a.ctl->abort != 0u;
    }
    __device__ __forceinline__ Ext open(const Job *gj, uint32_t task, Scoring &sc)
    {
        const Job J = ldcg_job(gj);
        sc = J.sc;
        return decode_cg(J, task);
    }
    __device__ __forceinline__ void retire(const Job *gj, uint32_t task, bool overflow, int32_t T,
                                           int32_t bi, int32_t bj)
    {
        const Job J = ldcg_job(gj);
        if (!overflow) {
            store_result_cg(J, task, T, bi, bj);
            serve_count(a, gj, J);
            return;
        }
        // Hand the task to the second tier (not counted yet).  Reserve a
        // queue position only while the queue has room; the slot's previous
        // occupant (one lap earlier) has been taken, and its taker clears
        // the slot right after reading it.
        volatile ServeCtl *v = a.ctl;
        unsigned long long t = v->spill_tail;
        for (int tries = 0; tries < 8; ++tries) {
            if (t - v->spill_head > kSpillQueueMask) break;  // full
            const unsigned long long got = atomicCAS(&a.ctl->spill_tail, t, t + 1);
            if (got == t) {
                volatile uint32_t *slot = (volatile uint32_t *)&a.spq[t & kSpillQueueMask];
                bool free_slot = false;
                for (int spin = 0; spin < kEntrySpinLimit; ++spin) {
                    if (*slot == 0u) { free_slot = true; break; }
                    __nanosleep(64);
                }
                if (!free_slot) {
                    volatile uint32_t *d = a.done;
                    d[2 * a.n_slots] = 1u;  // error word: the slot never drained
                    __threadfence_system();
                }
                *slot = (((uint32_t)(gj - a.slot_jobs) << 24) | task) + 1u;
                return;
            }
            t = got;
        }
        serve_list_wide(a, gj, J, task);  // queue full or contended: the host's pass
    }
};

// Second-tier task source of a helper warp.  Every queued entry's producer
// goes on fetching after it pushed, so it sees the backlog and registers as
// a helper unless enough are registered already: a queued entry always has
// a helper that has not left yet.
struct SpillSrc {
    static constexpr bool kCanAbort = true;  // teardown may stop the loop
    ServeArgs a;
    WarpFetch *w;  // this warp's fetch state (lane 0 only; reset before the loop)
    bool failed = false;

    __device__ __forceinline__ int fetch_warp(unsigned needm, int lane, int gbase, unsigned gm,
                                              bool need, uint32_t &task, const Job *&gj)
    {
        int status = 0;  // 1 granted k positions, 0 none, -1 leave
        int k = 0;
        unsigned long long base = 0;
        if (lane == 0) {
            if (w->backoff > 0) {
                --w->backoff;
            } else {
                volatile ServeCtl *v = a.ctl;
                const unsigned long long tail = *(volatile unsigned long long *)&a.ctl->spill_tail;
                unsigned long long head = *(volatile unsigned long long *)&a.ctl->spill_head;
                const unsigned long long want = (unsigned long long)__popc(needm);
                for (int tries = 0; tries < 4 && head < tail; ++tries) {
                    const unsigned long long kk = (tail - head < want) ? tail - head : want;
                    const unsigned long long got = atomicCAS(&a.ctl->spill_head, head, head + kk);
                    if (got == head) {
                        base = head;
                        k = (int)kk;
                        status = 1;
                        break;
                    }
                    head = got;
                }
                if (status == 1) {
                    w->level = 0;
                    w->idle_since = 0;
                } else if (head >= tail) {
                    // An empty queue: linger a little (more overflow is
                    // likely soon), then go back to the ring.
                    const unsigned long long now = globaltimer_ns();
                    if (w->idle_since == 0) w->idle_since = now;
                    if (v->yield || v->stop || now - w->idle_since > kHelpLingerNs) status = -1;
                    w->backoff = 1 << w->level;
                    if (w->level < 4) ++w->level;
                }
            }
        }
        // every lane takes part in the broadcasts before any lane returns
        status = __shfl_sync(FULL, status, 0);
        k = __shfl_sync(FULL, k, 0);
        base = __shfl_sync(FULL, base, 0);
        if (!need) return 0;
        if (status < 0) return -1;
        if (status == 0) return 0;
        const int rank = __popc(needm & ((1u << gbase) - 1u));
        if (rank >= k) return 0;
        // Each granted position's entry is written right after its producer
        // reserved it.  The group leader waits for it (bounded), takes it and
        // clears the slot, then hands it to its group.
        uint32_t val = 0;
        if (lane == gbase) {
            volatile uint32_t *slot = (volatile uint32_t *)&a.spq[(base + rank) & kSpillQueueMask];
            for (int spin = 0; spin < kEntrySpinLimit; ++spin) {
                val = *slot;
                if (val) break;
                __nanosleep(64);
            }
            if (val) {
                *slot = 0u;
            } else {
                volatile uint32_t *d = a.done;
                d[2 * a.n_slots] = 1u;  // error word: an entry never appeared
                __threadfence_system();
            }
        }
        val = __shfl_sync(gm, val, gbase);
        if (val == 0) {
            failed = true;
            return -1;
        }
        const uint32_t entry = val - 1u;
        task = entry & 0xffffffu;
        gj = &a.slot_jobs[entry >> 24];
        return 1;
    }
    __device__ __forceinline__ void idle() { __nanosleep(2000); }
    __device__ __forceinline__ bool aborted() const
    {
        return *(volatile const unsigned int *)&a.ctl->abort != 0u;
    }
    __device__ __forceinline__ Ext open(const Job *gj, uint32_t task, Scoring &sc)
    {
        const Job J = ldcg_job(gj);
        sc = J.sc;
        return decode_cg(J, task);
    }
    __device__ __forceinline__ void retire(const Job *gj, uint32_t task, bool overflow, int32_t T,
                                           int32_t bi, int32_t bj)
    {
        const Job J = ldcg_job(gj);
        if (overflow) {
            serve_list_wide(a, gj, J, task);
        } else {
            store_result_cg(J, task, T, bi, bj);
            serve_count(a, gj, J);
        }
    }
};

// The warp loop of both serving kernels: the first-tier loop FIRST on ring
// tasks, and when the warp registered as a helper, the second-tier loop
// SECOND on the spill queue, then back to the ring.
template <class FirstLoop, class SecondLoop>
__device__ __forceinline__ void serve_warp(const ServeArgs &a, FirstLoop first, SecondLoop second)
{
    __shared__ BlockQueue s_bq;       // the block's ring entries
    __shared__ WarpFetch s_fetch[8];  // 256 threads: 8 warps
    WarpFetch *wf = &s_fetch[threadIdx.x >> 5];
    const bool lead = (threadIdx.x & 31) == 0;
    if (threadIdx.x == 0) s_bq.ctl = 0ull;
    __syncthreads();
    for (;;) {
        if (lead) reset_fetch(wf, false);
        __syncwarp();
        RingSrc src{a, &s_bq, wf};
        first(src);
        if (__any_sync(FULL, src.leaving || src.aborted())) {
            if (lead && wf->helper) atomicSub(&a.ctl->helpers, 1u);
            break;
        }
        if (lead) reset_fetch(wf, true);
        __syncwarp();
        SpillSrc help{a, wf};
        second(help);
        if (lead) atomicSub(&a.ctl->helpers, 1u);
        if (__any_sync(FULL, help.failed || help.aborted())) break;
    }
    __threadfence();  // this warp's queue pushes before it counts itself out
    if ((threadIdx.x & 31) == 0) atomicSub(&a.ctl->ring_alive, 1u);
}

template <int L1, int C1, int L2, int C2>
__global__ void __launch_bounds__(256)
serve_kernel(ServeArgs a, const uint32_t *pk, int64_t nw)
{
    serve_warp(a, [&](RingSrc &src) { lockstep_loop<L1, C1>(src, pk, nw); },
               [&](SpillSrc &src) { lockstep_loop<L2, C2>(src, pk, nw); });
}

// Warps of a serving grid (all start on the first tier).
__host__ __device__ inline uint32_t serve_warps(int grid) { return (uint32_t)grid * 8u; }

// Serving form: the ring loop runs the packed tile, the second tier (helper
// warps) the 32-bit tile L2 x C2, which also takes every task whose scoring
// does not fit 16 bits.  Same protocol as serve_kernel.
template <int L1, int C2a, int L2, int C2>
__global__ void __launch_bounds__(256, 2)
serve16_kernel(ServeArgs a, const uint32_t *pk, int64_t nw)
{
    serve_warp(a, [&](RingSrc &src) { lockstep16_loop<L1, C2a>(src, pk, nw, a.one); },
               [&](SpillSrc &src) { lockstep_loop<L2, C2>(src, pk, nw); });
}

}  // namespace xd
