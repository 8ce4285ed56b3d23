/*
 * ms_server.h -- step server of the batched rigid-body step (libmsim.so).
 *
 * Serves many clients at once, the way a training or evaluation service
 * drives the paper's GPU-parallel environments (Sec. "GPU Parallelized
 * Simulation and Rendering": thousands of envs stepped together with
 * heterogeneous contents, Sec. "Heterogeneous GPU Simulation").  A client
 * opens a session owning 1..1024 envs of any scene type; the session's state
 * stays resident on the device for its whole life.  Sessions are admitted
 * against an HBM budget.  Each step request advances one session by one
 * step with fresh drive targets; a worker thread merges the pending
 * requests (at most one per session, none of a session whose previous step
 * is still running) into one launch of the batched kernel over the union of
 * their envs, keeps up to max_inflight such launches running at once on
 * their own streams, and stamps every request with its host arrival and
 * completion times.  The comparison mode launches one ms_step per request
 * instead (with the same number of launches in flight).
 *
 * ms_server_create sets the release threshold of the device's default
 * memory pool (a per-process setting) to its maximum, so that memory freed
 * by closed sessions is kept for the next session instead of being returned
 * to the driver at every synchronisation.
 *
 * All functions return ms_status (include/ms.h) and are thread-safe.
 */
#ifndef MS_SERVER_H
#define MS_SERVER_H

#include "ms.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_server ms_server;

typedef struct {
    int32_t merge;              /* 1: merge pending requests into one launch; 0: one launch per request */
    int32_t max_requests;       /* at most this many requests per merged launch (<= 0: no limit) */
    double coalesce_us;         /* after the first pending request, wait up to this long for more */
    int32_t max_inflight;       /* launches running at once, 1..64 (0: 16) */
} ms_server_options;

typedef struct {
    uint64_t ticket;
    uint64_t session;
    int32_t done;               /* 1 when the step has completed */
    int32_t status;             /* MS_OK, or the session's first device status error */
    double t_arrive;            /* seconds, host monotonic clock (ms_server_now) */
    double t_done;
    double latency;             /* t_done - t_arrive */
    int32_t launch_envs;        /* envs stepped by the launch that served it */
} ms_request_result;

typedef struct {
    uint64_t sessions_open, sessions_admitted, sessions_rejected;
    uint64_t requests_done, launches, env_steps;
    size_t hbm_used, hbm_budget;
    double p50, p99, mean;      /* request latency (s) over the completed requests */
    double busy_s;              /* time the worker spent with a launch in flight */
    uint64_t graph_captures;    /* launches that captured and instantiated a new graph */
    double launch_p50, launch_p99, launch_max;  /* host time (s) of one launch: staging to completion */
    double queue_p50, queue_p99;                /* request arrival to the start of its launch (s) */
    double stage_p99, stage_max;                /* host time (s) to stage and enqueue one launch */
} ms_server_stats;

/* Create a server on the current device.  hbm_budget_bytes bounds the
 * device memory of all open sessions together.  opt may be NULL (merge,
 * no limit, no coalescing wait, 4 launches in flight).  MS_ERR_INVALID_ARG
 * for max_inflight outside 0..64. */
ms_status ms_server_create(size_t hbm_budget_bytes, const ms_server_options* opt, ms_server** out);

/* Open a session of n_envs envs (flat tables as ms_create_batch_flat).
 * Returns MS_ERR_NOT_ADMITTED (nothing allocated) when the session's
 * estimated bytes do not fit in the remaining budget. */
ms_status ms_server_open(ms_server* s, const ms_body_desc* bodies, const int32_t* body_off,
                         const ms_joint_desc* joints, const int32_t* joint_off, int n_envs,
                         const ms_sim_params* p, uint64_t* session);

/* Close a session after its pending requests completed; frees its memory. */
ms_status ms_server_close(ms_server* s, uint64_t session);

/* Queue one step of the session.  actions: host float [n_envs][A] drive
 * targets (A = the session's max joints per env; NaN keeps a target) or
 * NULL; copied before returning.  *ticket identifies the request. */
ms_status ms_server_submit(ms_server* s, uint64_t session, const float* actions, uint64_t* ticket);

/* Result of a request; MS_ERR_BUSY while it is pending, MS_ERR_NOT_FOUND
 * for an unknown ticket.  A completed result is kept until read once. */
ms_status ms_server_poll(ms_server* s, uint64_t ticket, ms_request_result* out);

/* Block until every queued request has completed. */
ms_status ms_server_drain(ms_server* s);

/* Copy a session's state, float [n_bodies][13], to host memory. */
ms_status ms_server_copy_state(ms_server* s, uint64_t session, float* dst);

ms_status ms_server_stats_get(ms_server* s, ms_server_stats* out);

/* Clear the latency record and counters (not the sessions). */
ms_status ms_server_reset_stats(ms_server* s);

/* Stop the worker, close every session, free the server.  NULL accepted. */
ms_status ms_server_destroy(ms_server* s);

/* The host clock the server stamps requests with (seconds). */
double ms_server_now(void);

#ifdef __cplusplus
}
#endif
#endif
