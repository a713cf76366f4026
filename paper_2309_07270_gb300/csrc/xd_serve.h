// Serving runtime (continuous batching on one GPU): internal interface
// between the C ABI layer and xd_serve.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "xd_launch.h"
#include "xdrop.h"

namespace xd {

// Reads resident on the device (shared by every request).
struct ResidentReads {
    const uint32_t *packed = nullptr;  // device: the reads, then their reverse complements
    int64_t n_words = 0;               // words of the whole buffer
    int64_t rc_off = 0;                // bases from a read to its reverse complement
    const uint64_t *read_off = nullptr;  // device
    const uint32_t *read_len = nullptr;  // device
    uint32_t n_reads = 0;
};

struct ServerStats {
    uint64_t requests_done = 0;
    uint64_t wide_passes = 0;   // requests that ran the side-stream wider tiers
    uint64_t relaunches = 0;    // serving kernel launches
    uint64_t max_in_flight = 0; // admitted requests at once
    uint64_t admission_waits = 0;
    uint64_t published = 0, consumed = 0, spill_reserved = 0, spill_taken = 0, ring_warps = 0;
    uint64_t idle_exits = 0;    // first-tier warps that left on the idle bound (all launches)
    uint64_t help_sessions = 0; // warps that registered to serve the second tier (all launches)
    uint64_t surplus_counts = 0; // extensions counted past their request's total (stays 0)
};

class Server;

// device_budget: bytes of device arena for request buffers (pairs, results,
// spill lists); tile: the lockstep tile of the serving kernel; wide_scratch
// and wide_per_cta: the context's unbounded-tier scratch.
Server *server_create(int device, int sm_count, size_t device_budget, Tile tile,
                      const ResidentReads &rr, const uint32_t *read_len_host,
                      int32_t *wide_scratch, int64_t wide_per_cta, int wide_grid,
                      uint64_t idle_ns, std::string &err);
// Copies the pairs; returns 0 or an XDROP_* error.
int server_submit(Server *s, const xdrop_pair *pairs, size_t n_pairs, const Scoring &sc,
                  xdrop_result *out, uint64_t *ticket, std::string &err);
// 0, XDROP_ETIMEDOUT, XDROP_EINVAL (unknown ticket) or the request's error.
int server_sync(Server *s, uint64_t ticket, int64_t timeout_ns, std::string &err);
bool server_owns(Server *s, uint64_t ticket);
ServerStats server_stats(Server *s);
// Bound of a serving group's wait for work (hang guard), from the next
// kernel launch on; 0 restores the default.
void server_set_idle_ns(Server *s, uint64_t idle_ns);
void server_destroy(Server *s);

// Serving kernel launchers (tile families; the second tier follows from
// the first: 64-slot tiles pair with 16x8, 128-slot tiles with 32x16).
struct ServeArgs;
cudaError_t launch_serve(Tile t, int grid, const ServeArgs &a, const uint32_t *pk, int64_t nw,
                         cudaStream_t s);
int serve_blocks_per_sm(Tile t);

}  // namespace xd
