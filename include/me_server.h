/* Request server over the matrix-element library: continuous batching of
 * matrix-element and cross-section requests on one GPU.
 *
 * Each request is one xsec_step of include/me.h for a named process (Eq. 4:
 * |M|^2 at on-device phase-space points, Monte Carlo weights and sums), with
 * its own seed and counter offset.  Requests arrive at any time; the server
 *   - keeps every process it has seen created and resident on the device
 *     (compiled program and colour matrix stay in device memory);
 *   - admits requests first-in first-out while the device memory they need
 *     (|M|^2 and momentum arrays, per-chunk partial sums) fits in the budget
 *     beside the slot workspaces; a request bigger than the budget is refused;
 *   - launches a chunk as one CUDA graph per slot and process (the phase-space
 *     and |M|^2 kernels, captured at the first use and instantiated once; a
 *     chunk rewrites the kernels' per-chunk arguments in the executable graph),
 *     falling back to direct launches if a graph cannot be made;
 *   - splits every admitted request into chunks of a per-process size chosen
 *     by a timing autotuner (the smallest chunk whose time per point is within
 *     15 % of the best one), and keeps n_slots CUDA streams busy with chunks
 *     taken round-robin from all admitted requests, so that requests that
 *     arrive while others run start on the next free slot and overlap with
 *     them on the device;
 *   - sums each request's per-block partials in a fixed order, so a request's
 *     results do not depend on what else runs: alone or in a mix, |M|^2 and
 *     the sums are bit-identical.
 * Persistent mode (config.persistent = 1).  Instead of one graph launch per chunk,
 * each slot becomes a lane that runs one persistent kernel for one process at a
 * time (launched as a captured CUDA graph: claim-counter reset and kernel).  The
 * kernel's blocks claim items -- tiles of admitted requests -- from a queue in
 * page-locked host memory that the scheduler keeps filling while the kernel runs:
 * requests of that process that arrive meanwhile join the running kernel, their
 * tiles interleaved round-robin with the others' a little ahead of the blocks'
 * claims.  The block finishing a request's last tile sums its tile partials in tile
 * order and publishes the sums; the scheduler closes the queue when it has nothing
 * left to publish and the kernel ends.  A lane's kernel takes the SMs' resident
 * blocks divided by the number of lanes running.  The tile size (points per item)
 * and the resident blocks per SM come from an autotuner per process.  A block that
 * waits spin_limit_us for an item fails the lane (ME_ERR_TIMEOUT) rather than hang.
 * One scheduler thread owns all device work; the entry points may be called
 * from any host thread.  Latencies are host-clock times in ms since
 * me_server_create.  The paper has no serving layer: this interface is the
 * request loop built around its Monte Carlo step.
 */
#ifndef ME_SERVER_H
#define ME_SERVER_H

#include "me.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct me_server_s* me_server;

typedef struct {
  uint64_t mem_cap_bytes; /* device memory budget of the slot workspaces and the admitted
                             requests' buffers (0: 40 GiB) */
  int32_t n_slots;        /* CUDA streams with a chunk in flight at once, 1..16 (0: 4) */
  int32_t max_requests;   /* requests admitted at once, 1..65536 (0: 4096) */
  int32_t persistent;     /* 1: persistent lanes (below) for every process that has a persistent
                             kernel; the others (all-gluon processes) keep the chunk launches */
  int32_t spin_limit_us;  /* persistent lanes: longest a block of the kernel waits for its next
                             item (about 1 us per poll) before it gives up, 1..10^7 (0: 500000);
                             requests it leaves unfinished fail with ME_ERR_TIMEOUT */
  int32_t inject_feeder_stall; /* failure injection for tests: 1 = the scheduler never publishes
                             items to a running lane nor closes it, so its kernel's waits run out */
  int32_t pad_;
} me_server_config;

typedef struct {
  const char* process;     /* process string as for me_create (copied at submit) */
  int32_t precision;       /* ME_FP64 or ME_MIXED */
  int32_t want_me2;        /* keep |M|^2 of every accepted point for me_server_wait */
  int32_t want_momenta;    /* keep the momenta, SoA [n_ext][4][n], for me_server_wait */
  int32_t pad_;
  uint64_t seed;           /* Philox key of the request */
  uint64_t counter_offset; /* point i of the request uses counter offset + i (as xsec_step) */
  int64_t n;               /* accepted points, >= 1 */
  me_kin kin;              /* generator and cuts, as for xsec_step */
} me_request;

typedef struct {
  int32_t done;        /* 1 once the request's device work is complete */
  int32_t status;      /* me_status of the request: ME_OK, ME_ERR_TIMEOUT (a point exhausted its
                          redraws), ME_ERR_CUDA, ME_ERR_OOM */
  me_xsec_acc acc;     /* Monte Carlo sums of this request alone (as one xsec_step) */
  double t_submit_ms;  /* me_server_submit returned */
  double t_admit_ms;   /* buffers allocated within the budget */
  double t_start_ms;   /* first chunk launched */
  double t_done_ms;    /* device work observed complete by the scheduler */
  int64_t chunk;       /* points per launch used for this request */
} me_request_result;

typedef struct {
  uint64_t mem_cap_bytes;
  uint64_t bytes_in_use;   /* slot workspaces + admitted requests */
  uint64_t bytes_peak;
  int64_t submitted, admitted, completed, waiting, active;
  int64_t points_done;     /* accepted points of completed requests */
  int64_t launches;        /* chunk launches (each: phase-space and |M|^2 kernels) */
  int64_t graph_launches;  /* of those, launched as the slot's instantiated CUDA graph of the step */
  int64_t lane_launches;   /* persistent mode: persistent kernels started (each a graph launch) */
  int64_t lane_items;      /* persistent mode: tiles published to running kernels */
  int64_t lane_timeouts;   /* persistent mode: kernels that ended because a wait ran out */
} me_server_stats;

/* Start a server on the caller's current CUDA device.  cfg may be NULL (defaults). */
me_status me_server_create(const me_server_config* cfg, me_server* out);

/* Create the process (if new) and run the chunk autotuner for it now, on the
 * calling thread, so that the first request does not pay for it.  kin: the
 * generator and cuts to tune with.  *chunk (may be NULL) receives the choice:
 * points per launch (chunk mode), or points per tile (persistent mode). */
me_status me_server_warm(me_server s, const char* process, int32_t precision, const me_kin* kin, int64_t* chunk);

/* Queue a request; returns at once with a ticket.  Argument errors (unknown
 * process, bad kin, n < 1, a request larger than the whole budget) are
 * returned here and queue nothing. */
me_status me_server_submit(me_server s, const me_request* r, int64_t* ticket);

/* Non-blocking state of a request (res->done = 0 while it runs). */
me_status me_server_poll(me_server s, int64_t ticket, me_request_result* res);

/* Wait up to timeout_s seconds (< 0: no limit) for a request.  On completion:
 * copies |M|^2 into me2_host (n doubles) and the momenta into momenta_host
 * (n_ext*4*n doubles) where requested at submit and the pointer is not NULL,
 * releases the request's device memory and retires the ticket.  On timeout
 * returns ME_ERR_TIMEOUT and the request stays queued or running. */
me_status me_server_wait(me_server s, int64_t ticket, double timeout_s, me_request_result* res, double* me2_host,
                         double* momenta_host);

me_status me_server_get_stats(me_server s, me_server_stats* st);

/* Stop: waits for the device work in flight, then frees everything.  Tickets
 * not yet waited for are dropped. */
void me_server_destroy(me_server s);

#ifdef __cplusplus
}
#endif

#endif /* ME_SERVER_H */
