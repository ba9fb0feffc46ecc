/*
 * hpmxp_serve.h -- request executor of libhpmxp.so: many independent dense
 * systems (the serving workload: sizes from a few hundred to several thousand,
 * one to eight right-hand sides each) solved concurrently on one GPU.
 *
 * Each request runs the method of section "Algorithmic Framework" unchanged:
 * generation (section "Matrix Generation") when the caller passes no matrix,
 * low-precision LU without pivoting, fp64 GMRES-IR to the HPL threshold.  The
 * executor adds only scheduling: requests are admitted in arrival order
 * whenever their device memory fits in one caller-provided arena (admission
 * by HBM footprint), and `workers` host threads, each with its own CUDA
 * stream, run the admitted requests side by side so that the small kernels of
 * different systems overlap on the GPU.  A request's arithmetic does not
 * depend on what else runs: its x is bit-for-bit the x of the same request
 * run alone.
 *
 * Memory: the arena is caller-owned device memory, kept by the executor until
 * hpmxp_executor_destroy returns.  The executor sub-allocates it on the host
 * (first fit, 256-byte aligned blocks, freed blocks coalesce) and never
 * allocates device memory itself; it creates one CUDA stream per worker.
 */
#ifndef HPMXP_SERVE_H_
#define HPMXP_SERVE_H_

#include "hpmxp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpmxp_executor hpmxp_executor;   /* opaque */

typedef struct {
  int64_t id;            /* caller's tag, returned in the completion */
  int64_t n;             /* 1 <= n <= 131072 */
  int64_t nrhs;          /* 1..8 */
  int32_t prec;          /* hpmxp_prec of the factors */
  int32_t nb;            /* Schur-update depth 128/256/512, or 0: 128 for n < 4096, else 256 */
  const double* A;       /* device, n x n, lda >= n; NULL together with b: generate both */
  int64_t lda;
  const double* b;       /* device, n x nrhs, ldb >= n */
  int64_t ldb;
  double* x;             /* device out, n x nrhs, ldx >= n; NULL: x is kept only in the arena
                            while the request runs (the completion still reports the outcome) */
  int64_t ldx;
  uint64_t seed;         /* generator arguments, used when A and b are NULL */
  double margin;
  int32_t diag_mode;
  int32_t reserved;
  hpmxp_ir_params params;
} hpmxp_request;

typedef struct {
  int64_t id;
  int32_t status;        /* hpmxp_status: the factorization's breakdown, else the solve's outcome */
  int32_t nrhs;
  hpmxp_ir_info info[8]; /* per right-hand side (first nrhs entries) */
  double t_submit;       /* seconds on the executor's clock (hpmxp_executor_clock) */
  double t_start;        /* admitted: its memory was reserved and a worker took it */
  double t_done;
} hpmxp_completion;

/* Arena bytes one request needs (0 for an invalid request). */
size_t hpmxp_request_footprint(const hpmxp_request* r);

/* Starts `workers` (1..64) threads on `device`, each with its own stream.
 * arena: device memory of arena_bytes bytes, 256-byte aligned, owned by the
 * caller, not touched by anyone else until destroy returns. */
hpmxp_status hpmxp_executor_create(int device, int workers, void* arena, size_t arena_bytes,
                                   hpmxp_executor** out);

/* The same executor in batch mode: each worker takes the request at the head
 * of the queue and the ones queued right after it (up to max_batch, 1..256,
 * in arrival order, as many as fit the arena together) and runs them as one
 * batch through hpmxp_factor_batched and hpmxp_solve_ir_batched (grouped
 * kernels, lockstep refinement); requests in HPMXP_BF16 / HPMXP_FP16 with nb 0
 * or 128 (batches use depth 128) and equal refinement parameters share a
 * batch, any other runs alone.  Every request of a batch completes when the
 * batch does; max_batch = 1 is the plain executor. */
hpmxp_status hpmxp_executor_create_batched(int device, int workers, int max_batch, void* arena, size_t arena_bytes,
                                           hpmxp_executor** out);

/* Queues a copy of *r and returns at once.  HPMXP_EINVAL: bad request;
 * HPMXP_ENOMEM: its footprint exceeds the whole arena (it could never run).
 * Caller buffers named by the request must stay valid until its completion. */
hpmxp_status hpmxp_executor_submit(hpmxp_executor* ex, const hpmxp_request* r);

/* Moves up to `max` completions (in completion order) to `out`; waits up to
 * timeout_ms milliseconds for the first one (0: do not wait).  Returns how
 * many were written. */
int hpmxp_executor_poll(hpmxp_executor* ex, hpmxp_completion* out, int max, int timeout_ms);

/* Requests submitted and not yet returned by poll. */
int64_t hpmxp_executor_outstanding(hpmxp_executor* ex);

/* Seconds since the executor was created (the clock of the completions). */
double hpmxp_executor_clock(hpmxp_executor* ex);

/* Runs every queued request to completion, stops the workers, destroys their
 * streams and frees the executor (not the arena).  Completions not yet polled
 * are dropped. */
hpmxp_status hpmxp_executor_destroy(hpmxp_executor* ex);

#ifdef __cplusplus
}
#endif

#endif /* HPMXP_SERVE_H_ */
