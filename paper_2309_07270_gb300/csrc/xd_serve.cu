// Serving runtime: continuous batching of alignment requests from many
// producer threads on one GPU.
//
// One persistent serving kernel (the lockstep band kernel with a ring task
// source) runs while there is work.  Producers submit requests of read
// pairs against reads resident on the device; a worker thread admits a
// request when a slot is free, its buffers fit the device arena (memory
// admission) and the task ring has room, copies its pairs to the device and
// publishes its extensions into the ring.  Requests admitted while others
// run are picked up by the running kernel, so their work overlaps on the
// device.  Groups that finish the last task of a request write its tag (and
// its spill count) into mapped host memory; the worker then copies its
// results back and wakes the producer.
//
// Extensions whose band outgrows the serving tile go to a second-tier
// queue inside the kernel (a wider tile).  The few that outgrow that too are
// listed per request; once the request's other extensions are done the
// worker runs the 512-slot and unbounded tiers on them on a side stream.
// The serving kernel is launched a couple of blocks short of full
// occupancy, so that pass finds room beside it.  Every wait in the kernel
// is bounded (idle guard) and the host can make it leave at once (abort).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "xd_serve_kernels.cuh"
#include "xd_serve.h"
#include "xdrop.h"

namespace xd {
namespace {

constexpr int kSlots = 64;                    // requests admitted at once
constexpr uint32_t kRingBits = 21;            // task ring: 2 Mi entries
constexpr uint64_t kRing = 1ull << kRingBits;
constexpr size_t kAlign = 256;
constexpr size_t kHostPool = (size_t)512 << 20;  // pinned staging
// The host stops the serving kernel once nothing has been queued or in
// flight for kHostIdleS; kIdleNs only bounds a group's wait if that never
// happens (hang guard), so groups do not drop out during ordinary lulls.
constexpr unsigned long long kIdleNs = 5ull * 1000 * 1000 * 1000;
constexpr double kHostIdleS = 0.05;
constexpr double kShutdownWaitS = 60.0;       // bound on draining at context free
constexpr double kKernelExitWaitS = 30.0;     // bound on the kernel's exit at free

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, cap) (offsets only).
class Arena {
public:
    explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t cap() const { return cap_; }

private:
    size_t cap_, used_ = 0;
    std::map<size_t, size_t> free_;
};

enum ReqState { QUEUED, ADMITTED, SPILLED, COPYING, DONE };

struct Req {
    uint64_t id = 0;
    size_t n = 0;
    Scoring sc{};
    xdrop_result *out = nullptr;
    std::vector<xdrop_pair> pairs;
    ReqState state = QUEUED;
    int rc = 0;
    std::string err;
    int slot = -1;
    size_t dev_off = 0, dev_bytes = 0, host_off = 0, host_bytes = 0;
    // offsets inside the device / host areas
    size_t d_pairs = 0, d_out = 0, d_spill = 0, d_spill2 = 0, d_ctr = 0;
    size_t h_pairs = 0, h_out = 0, h_ring = 0, h_job = 0, h_pub = 0;
    cudaEvent_t ev = nullptr;
};

}  // namespace

class Server {
public:
    int device = 0, sm_count = 0;
    Tile tile{4, 16};
    int grid = 0;
    ResidentReads rr;
    std::vector<uint32_t> rr_len_host;  // read lengths (task ordering)
    int32_t *wide_scratch = nullptr;  // the server's own unbounded-tier scratch
    int32_t *own_wide = nullptr;
    int64_t wide_per_cta = 0;
    int wide_grid = 0;

    cudaStream_t s_kernel = nullptr, s_copy = nullptr, s_side = nullptr;
    ServeCtl *d_ctl = nullptr;
    uint32_t *d_ring = nullptr;
    uint32_t *d_spq = nullptr;      // second-tier queue
    Job *d_jobs = nullptr;
    char *d_arena = nullptr;
    char *h_pool = nullptr;         // pinned staging
    volatile uint32_t *h_done = nullptr;  // mapped: tag, spill count per slot
    uint32_t *d_done = nullptr;     // device view of h_done
    uint32_t *h_flags = nullptr;    // pinned constants: [0] = 0, [1] = 1
    ServeCtl *h_ctl_init = nullptr; // pinned
    ServeCtl *h_ctl_snap = nullptr; // pinned
    Arena dev_arena{0}, host_arena{0};

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    Req *slots[kSlots] = {};
    uint64_t next_id = 1;
    uint64_t published = 0, completed_tasks = 0;
    bool kernel_running = false;
    bool stop_sent = false;
    std::chrono::steady_clock::time_point last_busy = std::chrono::steady_clock::now();
    bool shutdown = false;
    std::chrono::steady_clock::time_point shutdown_at;
    std::string fatal;
    ServerStats stats;
    std::thread worker;

    void run();
    bool admit(Req *r);
    void complete_kernel_part(Req *r);
    void finish_copy(Req *r);
    void handle_spills(std::vector<Req *> &sp);
    cudaError_t ensure_kernel();
    bool wait_kernel_exit(double secs);
    void fail_all(const std::string &msg);
};

namespace {

cudaError_t set_flag(Server *s, unsigned int *field, int value, cudaStream_t st)
{
    return cudaMemcpyAsync(field, &s->h_flags[value ? 1 : 0], sizeof(unsigned int),
                           cudaMemcpyHostToDevice, st);
}

}  // namespace

bool Server::wait_kernel_exit(double secs)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(s_kernel);
        if (q != cudaErrorNotReady) return true;
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > secs)
            return false;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

cudaError_t Server::ensure_kernel()
{
    if (kernel_running) {
        cudaError_t q = cudaStreamQuery(s_kernel);
        if (q == cudaErrorNotReady) return cudaSuccess;
        if (q != cudaSuccess) return q;
        kernel_running = false;
    }
    h_ctl_init->ring_alive = serve_warps(grid);
    cudaError_t e = cudaMemcpyAsync(&d_ctl->ring_alive, &h_ctl_init->ring_alive, sizeof(unsigned int),
                                    cudaMemcpyHostToDevice, s_kernel);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&d_ctl->idle_ns, &h_ctl_init->idle_ns, sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, s_kernel);
    if (e == cudaSuccess) e = set_flag(this, &d_ctl->stop, 0, s_kernel);
    if (e == cudaSuccess) e = set_flag(this, &d_ctl->abort, 0, s_kernel);
    stop_sent = false;
    ServeArgs a;
    a.ctl = d_ctl;
    a.ring = d_ring;
    a.ring_mask = (uint32_t)(kRing - 1);
    a.spq = d_spq;
    a.slot_jobs = d_jobs;
    a.done = d_done;
    a.n_slots = kSlots;
    a.max_helpers = std::max<uint32_t>(1u, serve_warps(grid) / 4);  // a quarter of the warps
    a.one = 1u;
    if (e == cudaSuccess) e = launch_serve(tile, grid, a, rr.packed, rr.n_words, s_kernel);
    if (e == cudaSuccess) {
        kernel_running = true;
        stats.relaunches += 1;
    }
    return e;
}

bool Server::admit(Req *r)
{
    int slot = -1;
    for (int k = 0; k < kSlots; ++k)
        if (!slots[k]) { slot = k; break; }
    if (slot < 0) return false;
    const uint64_t tasks = 2 * (uint64_t)r->n;
    if (published + tasks - completed_tasks > kRing) return false;
    // device: pairs, results, spill lists, counters
    r->d_pairs = 0;
    r->d_out = align_up(r->n * sizeof(xdrop_pair));
    r->d_spill = r->d_out + align_up(r->n * sizeof(xdrop_result));
    r->d_spill2 = r->d_spill + align_up(tasks * 4);
    r->d_ctr = r->d_spill2 + align_up(tasks * 4);
    r->dev_bytes = r->d_ctr + kAlign;
    // host staging: pairs, results, ring entries, job, published value
    r->h_pairs = 0;
    r->h_out = align_up(r->n * sizeof(xdrop_pair));
    r->h_ring = r->h_out + align_up(r->n * sizeof(xdrop_result));
    r->h_job = r->h_ring + align_up(tasks * 4);
    r->h_pub = r->h_job + align_up(sizeof(Job));
    r->host_bytes = r->h_pub + kAlign;
    if (!dev_arena.alloc(r->dev_bytes, &r->dev_off)) {
        stats.admission_waits += 1;
        return false;
    }
    if (!host_arena.alloc(r->host_bytes, &r->host_off)) {
        dev_arena.release(r->dev_off, r->dev_bytes);
        stats.admission_waits += 1;
        return false;
    }
    char *d = d_arena + r->dev_off;
    char *h = h_pool + r->host_off;
    // Clear the slot's done word before anything of this request can reach
    // the device: a small request may finish (and the kernel write its tag)
    // before this thread runs again after queueing the copies below.
    h_done[2 * slot] = 0;
    h_done[2 * slot + 1] = 0;
    memcpy(h + r->h_pairs, r->pairs.data(), r->n * sizeof(xdrop_pair));
    // Ring entries longest extension first (the batched form's order), so
    // the lockstep groups of a warp run extensions of similar length.
    uint32_t *ring_stage = (uint32_t *)(h + r->h_ring);
    {
        std::vector<std::pair<uint32_t, uint32_t>> key(tasks);
        for (uint64_t t = 0; t < tasks; ++t) {
            const xdrop_pair &p = r->pairs[t >> 1];
            uint32_t m, n;
            if (t & 1) {
                m = rr_len_host[p.a] - p.seed_a - p.seed_len;
                n = rr_len_host[p.b & ~kPairRC] - p.seed_b - p.seed_len;
            } else {
                m = p.seed_a;
                n = p.seed_b;
            }
            key[t] = {std::max(m, n), (uint32_t)t};
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<uint32_t, uint32_t> &x,
                            const std::pair<uint32_t, uint32_t> &y) { return x.first > y.first; });
        for (uint64_t t = 0; t < tasks; ++t)
            ring_stage[t] = ((uint32_t)slot << 24) | key[t].second;
    }
    Job *job = (Job *)(h + r->h_job);
    job->packed = rr.packed;
    job->n_words = rr.n_words;
    job->rc_off = rr.rc_off;
    job->read_off = rr.read_off;
    job->read_len = rr.read_len;
    job->n_reads = rr.n_reads;
    job->pairs = (const Pair *)(d + r->d_pairs);
    job->n_pairs = r->n;
    job->sc = r->sc;
    job->out = (int32_t *)(d + r->d_out);
    job->cells = nullptr;
    job->ctr = (uint32_t *)(d + r->d_ctr);
    job->spill_list = (uint32_t *)(d + r->d_spill);
    job->tag = (uint32_t)r->id;
    const uint64_t first = published;
    published += tasks;
    *(unsigned long long *)(h + r->h_pub) = published;

    cudaError_t e = cudaMemcpyAsync(d + r->d_pairs, h + r->h_pairs, r->n * sizeof(xdrop_pair),
                                    cudaMemcpyHostToDevice, s_copy);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + r->d_out, 0, r->n * sizeof(xdrop_result), s_copy);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + r->d_ctr, 0, kAlign, s_copy);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_jobs + slot, job, sizeof(Job), cudaMemcpyHostToDevice, s_copy);
    // ring entries, wrapping at the end of the ring
    const uint64_t pos = first & (kRing - 1);
    const uint64_t n1 = std::min<uint64_t>(tasks, kRing - pos);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ring + pos, ring_stage, n1 * 4, cudaMemcpyHostToDevice, s_copy);
    if (e == cudaSuccess && tasks > n1)
        e = cudaMemcpyAsync(d_ring, ring_stage + n1, (tasks - n1) * 4, cudaMemcpyHostToDevice,
                            s_copy);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&d_ctl->published, h + r->h_pub, sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, s_copy);
    if (e != cudaSuccess) {
        fatal = std::string("serve admission: ") + cudaGetErrorString(e);
        return false;
    }
    slots[slot] = r;
    r->slot = slot;
    r->state = ADMITTED;
    r->pairs.clear();
    r->pairs.shrink_to_fit();
    size_t inflight = 0;
    for (auto *q : slots) inflight += q != nullptr;
    stats.max_in_flight = std::max<uint64_t>(stats.max_in_flight, inflight);
    return true;
}

void Server::finish_copy(Req *r)
{
    char *h = h_pool + r->host_off;
    if (r->n) memcpy(r->out, h + r->h_out, r->n * sizeof(xdrop_result));
    dev_arena.release(r->dev_off, r->dev_bytes);
    host_arena.release(r->host_off, r->host_bytes);
    slots[r->slot] = nullptr;
    completed_tasks += 2 * (uint64_t)r->n;
    r->state = DONE;
    stats.requests_done += 1;
}

void Server::complete_kernel_part(Req *r)
{
    char *d = d_arena + r->dev_off;
    char *h = h_pool + r->host_off;
    cudaError_t e = cudaMemcpyAsync(h + r->h_out, d + r->d_out, r->n * sizeof(xdrop_result),
                                    cudaMemcpyDeviceToHost, s_copy);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, s_copy);
    if (e != cudaSuccess) fatal = std::string("serve copy-back: ") + cudaGetErrorString(e);
    r->state = COPYING;
}

void Server::handle_spills(std::vector<Req *> &sp)
{
    // Wider tiers for the extensions both in-kernel tiers could not hold,
    // on the side stream (the serving kernel leaves room for it).
    cudaError_t e = cudaSuccess;
    for (Req *r : sp) {
        char *d = d_arena + r->dev_off;
        uint32_t *ctr = (uint32_t *)(d + r->d_ctr);
        Spill in{(uint32_t *)(d + r->d_spill), ctr + 1};
        Spill out{(uint32_t *)(d + r->d_spill2), ctr + 2};
        if (e == cudaSuccess)
            e = launch_spill(Tile{32, 16}, false, 2 * sm_count, d_jobs + r->slot, in, out, s_side);
        if (e == cudaSuccess)
            e = launch_wide(false, wide_grid, d_jobs + r->slot, out, wide_scratch, wide_per_cta, s_side);
        if (e == cudaSuccess) {
            char *h = h_pool + r->host_off;
            e = cudaMemcpyAsync(h + r->h_out, d + r->d_out, r->n * sizeof(xdrop_result),
                                cudaMemcpyDeviceToHost, s_side);
        }
        if (e == cudaSuccess) e = cudaEventRecord(r->ev, s_side);
        r->state = COPYING;
        stats.wide_passes += 1;
    }
    if (e != cudaSuccess) fatal = std::string("serve wide pass: ") + cudaGetErrorString(e);
}

void Server::fail_all(const std::string &msg)
{
    if (kernel_running) set_flag(this, &d_ctl->abort, 1, s_copy);
    for (auto &kv : reqs) {
        Req *r = kv.second;
        if (r->state != DONE) {
            r->rc = XDROP_ECUDA;
            r->err = msg;
            r->state = DONE;
        }
    }
    queue.clear();
    for (auto &sl : slots) sl = nullptr;  // buffers stay with the failed device state
}

void Server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progress = false;
        if (!fatal.empty()) {
            fail_all(fatal);
            cv.notify_all();
        }
        if (h_done[2 * kSlots] && fatal.empty())
            fatal = "serving kernel: a second-tier queue entry never appeared";
        // completions
        std::vector<Req *> spilled;
        for (int k = 0; k < kSlots; ++k) {
            Req *r = slots[k];
            if (!r) continue;
            if (r->state == ADMITTED && h_done[2 * k] == (uint32_t)r->id) {
                if (h_done[2 * k + 1]) {
                    r->state = SPILLED;
                    spilled.push_back(r);
                } else {
                    complete_kernel_part(r);
                }
                progress = true;
            }
            if (r->state == COPYING) {
                cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaSuccess) {
                    finish_copy(r);
                    progress = true;
                } else if (q != cudaErrorNotReady) {
                    fatal = std::string("serve event: ") + cudaGetErrorString(q);
                }
            }
        }
        if (!spilled.empty() && fatal.empty()) handle_spills(spilled);
        if (progress) cv.notify_all();
        // Work after an idle stop: the kernel had nothing in flight and is
        // leaving; wait for it so the next launch starts with every group.
        if (stop_sent && kernel_running && !queue.empty() && fatal.empty()) {
            if (!wait_kernel_exit(5.0)) {
                set_flag(this, &d_ctl->abort, 1, s_copy);
                if (!wait_kernel_exit(kKernelExitWaitS)) fatal = "serve stop: the kernel did not leave";
            }
            kernel_running = false;
        }
        // admission, in arrival order
        bool published_any = false;
        while (!queue.empty() && fatal.empty()) {
            if (!admit(queue.front())) break;
            queue.pop_front();
            published_any = true;
            progress = true;
        }
        bool any_admitted = false;
        for (auto *r : slots) any_admitted |= (r && r->state == ADMITTED);
        if ((published_any || any_admitted) && fatal.empty()) {
            cudaError_t e = ensure_kernel();
            if (e != cudaSuccess) fatal = std::string("serve kernel launch: ") + cudaGetErrorString(e);
        }
        bool busy = !queue.empty();
        for (auto *r : slots) busy |= r != nullptr;
        if (shutdown && !busy) break;
        if (shutdown && std::chrono::duration<double>(std::chrono::steady_clock::now() -
                                                      shutdown_at).count() > kShutdownWaitS) {
            fail_all("context freed with requests still in flight");
            cv.notify_all();
            break;
        }
        const auto now = std::chrono::steady_clock::now();
        if (busy) {
            last_busy = now;
        } else if (kernel_running && !stop_sent &&
                   std::chrono::duration<double>(now - last_busy).count() > kHostIdleS) {
            // idle: let the serving kernel's groups leave together
            if (set_flag(this, &d_ctl->stop, 1, s_copy) == cudaSuccess) stop_sent = true;
        }
        if (!progress) {
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(10));
                lk.lock();
            } else {
                cv.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

Server *server_create(int device, int sm_count, size_t device_budget, Tile tile,
                      const ResidentReads &rr, const uint32_t *read_len_host,
                      int32_t *wide_scratch, int64_t wide_per_cta, int wide_grid,
                      uint64_t idle_ns, std::string &err)
{
    cudaSetDevice(device);
    Server *s = new Server();
    s->device = device;
    s->sm_count = sm_count;
    s->tile = tile;
    s->rr = rr;
    s->rr_len_host.assign(read_len_host, read_len_host + rr.n_reads);
    (void)wide_scratch;
    s->wide_per_cta = wide_per_cta;
    s->wide_grid = wide_grid;
    const int bps = serve_blocks_per_sm(tile);
    if (bps <= 0) {
        err = "serving tile not available";
        delete s;
        return nullptr;
    }
    s->grid = std::max(1, bps * sm_count - 2);  // room for the side-stream pass
    const size_t arena = device_budget ? device_budget : ((size_t)1 << 30);
    s->dev_arena = Arena(arena);
    s->host_arena = Arena(kHostPool);
    cudaError_t e = cudaStreamCreateWithFlags(&s->s_kernel, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctl, sizeof(ServeCtl));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ring, kRing * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_spq, (kSpillQueueMask + 1) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->d_spq, 0, (kSpillQueueMask + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_jobs, kSlots * sizeof(Job));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, arena);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_pool, kHostPool, cudaHostAllocDefault);
    void *hd = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(&hd, (2 * kSlots + 2) * 4, cudaHostAllocMapped);
    if (e == cudaSuccess) {
        s->h_done = (volatile uint32_t *)hd;
        e = cudaHostGetDevicePointer((void **)&s->d_done, hd, 0);
    }
    if (e == cudaSuccess && wide_per_cta > 0)
        e = cudaMalloc(&s->own_wide, (size_t)wide_per_cta * 4 * wide_grid);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_flags, 2 * 4, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_ctl_init, sizeof(ServeCtl), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_ctl_snap, sizeof(ServeCtl), cudaHostAllocDefault);
    if (e == cudaSuccess) {
        for (int k = 0; k < 2 * kSlots + 2; ++k) s->h_done[k] = 0;
        s->wide_scratch = s->own_wide;
        s->h_flags[0] = 0;
        s->h_flags[1] = 1;
        memset(s->h_ctl_init, 0, sizeof(ServeCtl));
        s->h_ctl_init->idle_ns = idle_ns ? idle_ns : kIdleNs;
        e = cudaMemcpy(s->d_ctl, s->h_ctl_init, sizeof(ServeCtl), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        err = std::string("serve setup: ") + cudaGetErrorString(e);
        server_destroy(s);
        return nullptr;
    }
    s->worker = std::thread([s] { s->run(); });
    return s;
}

int server_submit(Server *s, const xdrop_pair *pairs, size_t n_pairs, const Scoring &sc,
                  xdrop_result *out, uint64_t *ticket, std::string &err)
{
    if (2 * (uint64_t)n_pairs > kRing) {
        err = "request larger than the serving task ring";
        return XDROP_EINVAL;
    }
    {
        const uint64_t tasks = 2 * (uint64_t)n_pairs;
        const size_t dev = align_up(n_pairs * sizeof(xdrop_pair)) +
                           align_up(n_pairs * sizeof(xdrop_result)) + 2 * align_up(tasks * 4) +
                           kAlign;
        const size_t host = align_up(n_pairs * sizeof(xdrop_pair)) +
                            align_up(n_pairs * sizeof(xdrop_result)) + align_up(tasks * 4) +
                            align_up(sizeof(Job)) + kAlign;
        if (dev > s->dev_arena.cap() || host > s->host_arena.cap()) {
            err = "request does not fit the serving memory budget even alone";
            return XDROP_ENOMEM;
        }
    }
    Req *r = new Req();
    r->n = n_pairs;
    r->sc = sc;
    r->out = out;
    r->pairs.assign(pairs, pairs + n_pairs);
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete r;
        err = "event creation failed";
        return XDROP_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->fatal.empty()) {
            cudaEventDestroy(r->ev);
            delete r;
            err = s->fatal;
            return XDROP_ECUDA;
        }
        r->id = s->next_id++;
        if (n_pairs == 0) r->state = DONE;
        else s->queue.push_back(r);
        s->reqs[r->id] = r;
        *ticket = r->id;
    }
    s->cv.notify_all();
    return XDROP_OK;
}

bool server_owns(Server *s, uint64_t ticket)
{
    std::lock_guard<std::mutex> lk(s->mu);
    return s->reqs.count(ticket) != 0;
}

int server_sync(Server *s, uint64_t ticket, int64_t timeout_ns, std::string &err)
{
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        err = "unknown serving ticket";
        return XDROP_EINVAL;
    }
    Req *r = it->second;
    auto pred = [r] { return r->state == DONE; };
    if (timeout_ns < 0) {
        s->cv.wait(lk, pred);
    } else if (!s->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
        err = "serving request not done";
        if (r->state == ADMITTED) {
            // what the device has: finished extensions and the slot's done word
            uint32_t ctr[2] = {0, 0};
            const char *d = s->d_arena + r->dev_off;
            if (cudaMemcpyAsync(ctr, d + r->d_ctr, sizeof(ctr), cudaMemcpyDeviceToHost,
                                s->s_copy) == cudaSuccess &&
                cudaStreamSynchronize(s->s_copy) == cudaSuccess) {
                err += ": " + std::to_string(ctr[0]) + " of " + std::to_string(2 * r->n) +
                       " extensions finished on the device, " + std::to_string(ctr[1]) +
                       " listed for the wide pass; done word " +
                       std::to_string(s->h_done[2 * r->slot]) + ", tag " + std::to_string(r->id);
            }
            ServeCtl c{};
            if (cudaMemcpyAsync(s->h_ctl_snap, s->d_ctl, sizeof(ServeCtl), cudaMemcpyDeviceToHost,
                                s->s_copy) == cudaSuccess &&
                cudaStreamSynchronize(s->s_copy) == cudaSuccess) {
                c = *s->h_ctl_snap;
                err += "; surplus counts " + std::to_string(c.surplus_counts);
            }
        }
        return XDROP_ETIMEDOUT;
    }
    const int rc = r->rc;
    if (rc) err = r->err;
    s->reqs.erase(it);
    cudaEventDestroy(r->ev);
    delete r;
    return rc;
}

ServerStats server_stats(Server *s)
{
    std::lock_guard<std::mutex> lk(s->mu);
    ServerStats st = s->stats;
    // live counters of the control block (a small copy on the copy stream)
    ServeCtl c{};
    if (cudaMemcpyAsync(s->h_ctl_snap, s->d_ctl, sizeof(ServeCtl), cudaMemcpyDeviceToHost,
                        s->s_copy) == cudaSuccess &&
        cudaStreamSynchronize(s->s_copy) == cudaSuccess) {
        c = *s->h_ctl_snap;
        st.published = c.published;
        st.consumed = c.consumed;
        st.spill_reserved = c.spill_tail;
        st.spill_taken = c.spill_head;
        st.ring_warps = c.ring_alive;
        st.idle_exits = c.idle_exits;
        st.help_sessions = c.help_sessions;
        st.surplus_counts = c.surplus_counts;
    }
    return st;
}

void server_set_idle_ns(Server *s, uint64_t idle_ns)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->h_ctl_init->idle_ns = idle_ns ? idle_ns : kIdleNs;
}

void server_destroy(Server *s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->shutdown = true;
            s->shutdown_at = std::chrono::steady_clock::now();
        }
        s->cv.notify_all();
        s->worker.join();
    }
    cudaSetDevice(s->device);
    if (s->d_ctl && s->kernel_running) {
        // stop and yield: groups take no new task and leave; then, if the
        // kernel is still there after a few seconds, abort it (tasks are
        // abandoned; nothing is in flight by then unless a request failed).
        set_flag(s, &s->d_ctl->stop, 1, s->s_copy);
        set_flag(s, &s->d_ctl->yield, 1, s->s_copy);
        cudaStreamSynchronize(s->s_copy);
        auto wait_exit = [s](double secs) {
            auto t0 = std::chrono::steady_clock::now();
            while (cudaStreamQuery(s->s_kernel) == cudaErrorNotReady &&
                   std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() < secs)
                std::this_thread::sleep_for(std::chrono::milliseconds(1));
        };
        wait_exit(5.0);
        if (cudaStreamQuery(s->s_kernel) == cudaErrorNotReady) {
            set_flag(s, &s->d_ctl->abort, 1, s->s_copy);
            cudaStreamSynchronize(s->s_copy);
            wait_exit(kKernelExitWaitS);
        }
        cudaStreamSynchronize(s->s_side);
        if (cudaStreamQuery(s->s_kernel) == cudaErrorNotReady) {
            // The kernel did not leave: keep its memory (it may still touch
            // it) and give up on freeing the rest of the server.
            return;
        }
    }
    for (auto &kv : s->reqs) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    if (s->s_kernel) cudaStreamDestroy(s->s_kernel);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    if (s->s_side) cudaStreamDestroy(s->s_side);
    cudaFree(s->d_ctl);
    cudaFree(s->d_ring);
    cudaFree(s->d_spq);
    cudaFree(s->d_jobs);
    cudaFree(s->d_arena);
    if (s->h_pool) cudaFreeHost(s->h_pool);
    if (s->h_done) cudaFreeHost((void *)s->h_done);
    cudaFree(s->own_wide);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->h_ctl_init) cudaFreeHost(s->h_ctl_init);
    if (s->h_ctl_snap) cudaFreeHost(s->h_ctl_snap);
    delete s;
}

}  // namespace xd
