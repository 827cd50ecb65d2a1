/* Native client of the serving engine and of the batch calls (load
 * generator): replays a stream of requests against salt_serve_submit /
 * salt_serve_poll from two native threads, or runs the same requests as
 * plain per-request batch calls. The paper has no counterpart: these are the
 * measured side of the serving comparison (continuous batching against one
 * launch per request), written over the public C ABI of salt.h only, so the
 * figures contain no interpreter overhead.
 *
 * libsalt_client.so links libsalt_b300.so; every pointer below is HOST
 * memory unless stated otherwise. Calls return SALT_* status codes. */
#ifndef SALT_CLIENT_H
#define SALT_CLIENT_H

#include "salt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Outcome of a replay. Latency here is the client's: from the request's
 * scheduled arrival (its submission when arrivals are not given) to the
 * return of salt_serve_poll with its results. */
typedef struct {
    double wall_s;        /* first submission to the last result */
    double submit_s;      /* first to last submission */
    int64_t completed;    /* requests whose poll returned SALT_OK */
    double p50_ms, p99_ms;
} salt_replay_stats;

/* Replay n requests against ctx's serving engine: one thread submits
 * request i at arrival_s[i] seconds after the start (all at once when
 * arrival_s is NULL; arrivals nondecreasing), another sweeps the oldest
 * outstanding requests (up to 32 at a time) with non-blocking polls, backing
 * off 20 us after a sweep that finds nothing, and takes each result when it is
 * ready. Results go to chi2_out[i] (HOST float64 [n_par]) and
 * grad_out[i] (HOST float32 [n_par][5], requests with want_grad) when those
 * arrays and entries are non-NULL, else to a scratch buffer. lat_ms
 * (nullable, [n]) receives each request's client latency. Returns the first
 * failing submission's or poll's status (the remaining requests are still
 * drained), SALT_ERR_INVALID for bad arguments. */
int salt_client_replay(salt_ctx *ctx, const salt_request *reqs, int32_t n, const double *arrival_s,
                       double *const *chi2_out, float *const *grad_out, double *lat_ms, salt_replay_stats *out);

/* Outcome of the plain per-request loop. */
typedef struct {
    double wall_s;        /* the requests run, back to back */
    int64_t completed;    /* requests run before the time limit */
    double p50_ms, p99_ms;
} salt_plain_stats;

/* The same requests without batching, each on its own, in order: before the
 * clock starts, every request's inputs are packed once into pinned host
 * memory (at most pack_bytes; later requests are left out) and device buffers
 * for the largest request are allocated; then per request one host-to-device
 * copy into those buffers, salt_chi2 or salt_chi2_grad on a one-supernova
 * batch without a plan, one device-to-host copy of its results and a stream
 * synchronisation. Stops after time_limit_s seconds. lat_ms (nullable, [n])
 * receives each run request's latency. */
int salt_client_plain(salt_ctx *ctx, const salt_request *reqs, int32_t n, double time_limit_s, size_t pack_bytes,
                      double *lat_ms, salt_plain_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* SALT_CLIENT_H */
