/*
 * hpmxp.h -- C interface of the HPL-MxP solver library (libhpmxp.so).
 *
 * The library solves A x = b for a dense n x n system to the fp64 accuracy
 * HPL demands, by a low-precision LU factorization without pivoting followed
 * by fp64 GMRES-based iterative refinement (Dongarra & Luszczek, "HPL-MxP
 * Benchmark: Mixed-Precision Algorithms, Iterative Refinement, and Scalable
 * Data Generation", arXiv 2509.19618, section "Algorithmic Framework").  It
 * runs on one GB300 GPU (sm_103a).
 *
 * Conventions shared by every entry point:
 *  - Every array argument is DEVICE memory owned by the caller.  The library
 *    never allocates, frees or retains caller memory; scratch space is passed
 *    in as `ws` / `ws_bytes` (size from the matching *_workspace function,
 *    256-byte aligned).  Host-side outputs are marked "host".
 *  - Matrices are column major with an explicit leading dimension.
 *  - Every call is ordered on the caller's CUDA stream (`stream`, a
 *    cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 *    that return host values synchronize that stream before returning.
 *  - Every call returns an hpmxp_status and never aborts, exits or traps.
 *    HPMXP_EINVAL leaves every output untouched.  Device waits inside the
 *    library's kernels are bounded; a wait that runs out returns
 *    HPMXP_ETIMEOUT and leaves the outputs unspecified.
 *  - The library is thread compatible: concurrent calls must use distinct
 *    workspaces.
 */
#ifndef HPMXP_H_
#define HPMXP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPMXP_OK = 0,
  HPMXP_EINVAL = 1,      /* bad argument (size, leading dimension, alignment, NULL) */
  HPMXP_ENOMEM = 2,      /* workspace too small */
  HPMXP_ECUDA = 3,       /* a CUDA runtime/driver call failed */
  HPMXP_ENOCONV = 4,     /* refinement needed more than max_iters iterations */
  HPMXP_EBREAKDOWN = 5,  /* zero or non-finite pivot, or non-finite value in the refinement */
  HPMXP_ETIMEOUT = 6,    /* a bounded device-side wait ran out */
  HPMXP_EINVALID = 7     /* final scaled residual >= the acceptance threshold */
} hpmxp_status;

/* Low-precision format of the factorization (section "Algorithmic Framework":
 * the factors must be at least FP16-accurate; BF16 has FP32's exponent range).
 * HPMXP_FP8_E4M3 keeps BF16 factors and runs only the trailing-matrix (Schur)
 * update on OCP E4M3 operands with fp32 per-128x128-tile scales.
 * HPMXP_BF16_TRAIL32 / HPMXP_FP16_TRAIL32 follow Fig. 1 with a 32-bit trailing
 * matrix: the Schur updates (16-bit operands, fp32 accumulation) are
 * accumulated into an fp32 copy of the matrix, and a block column / row is
 * rounded to the 16-bit format only once, when it becomes the panel; the
 * factors are BF16 / FP16 as with HPMXP_BF16 / HPMXP_FP16, which the solve
 * accepts for them too. */
typedef enum {
  HPMXP_BF16 = 0,
  HPMXP_FP16 = 1,
  HPMXP_FP8_E4M3 = 2,
  HPMXP_BF16_TRAIL32 = 3,
  HPMXP_FP16_TRAIL32 = 4
} hpmxp_prec;

/* Diagonal of the generated matrix (section "Matrix Generation" and the
 * diagonal-scaling discussion of section "Experimental Results"). */
typedef enum {
  HPMXP_DIAG_DOMINANT = 0, /* a_ii = sum_{j!=i} |a_ij| + margin: strictly row diagonally dominant */
  HPMXP_DIAG_SQRTN = 1,    /* a_ii = r_ii + sign(r_ii) c sqrt(n) with c = margin: the sqrt(n) scaling the
                              paper recommends (c = 1), and its 5/8 sqrt(n) curve (c = 0.625) */
  HPMXP_DIAG_NONE = 2,     /* raw uniform entries, no diagonal scaling */
  HPMXP_DIAG_DEPARTURE = 3 /* a_ii = rho sum_{j!=i} |a_ij| with rho = margin > 0: a controlled departure
                              from diagonal dominance (rho < 1), weak dominance at rho = 1 */
} hpmxp_diag;

/* Human-readable name of a status code (static storage; never NULL). */
const char* hpmxp_status_string(hpmxp_status s);

/* Library version as major*10000 + minor*100 + patch. */
int hpmxp_version(void);

/* ------------------------------------------------------------------------ */
/* Generation (section "Matrix Generation": a scalable generator for which any
 * entry is computable independently; the matrix admits LU without pivoting).
 *
 * Entries come from the 64-bit LCG s' = 6364136223846793005 s +
 * 1442695040888963407 (mod 2^64) seeded with `seed`; draw t uses the state
 * after t+1 steps, reached by skip-ahead.  The top 52 bits u of a state give
 * the value (2u + 1 - 2^52) 2^-53, uniform in (-0.5, 0.5) and never 0.
 * Entry A(i,j) is draw i + j*n, b(i,r) is draw n*n + i + r*n.  The diagonal is
 * then replaced as `diag_mode` says; for DOMINANT and DEPARTURE the
 * off-diagonal magnitudes are summed exactly in 128-bit integer arithmetic and
 * a_ii = fl(fl(S_i) 2^-53 + margin) (DOMINANT) or fl(fl(S_i) 2^-53 margin)
 * (DEPARTURE); SQRTN gives fl(r_ii + sign(r_ii) fl(margin fl(sqrt(n)))); so the
 * result is bit-for-bit reproducible.  DEPARTURE needs margin > 0.
 *
 *   n        1 <= n <= 131072
 *   A        out, n x n fp64, column major, lda >= n
 *   b        out, n x nrhs fp64, ldb >= n (may be NULL when nrhs == 0)
 *   ws       scratch of hpmxp_generate_workspace(n) bytes
 * Generation is not part of the timed solve (section "Algorithmic Framework",
 * figure-of-merit paragraph). */
size_t hpmxp_generate_workspace(int64_t n);
hpmxp_status hpmxp_generate(int64_t n, uint64_t seed, double margin, int diag_mode, double* A,
                            int64_t lda, double* b, int64_t ldb, int64_t nrhs, void* ws,
                            size_t ws_bytes, void* stream);

/* hpmxp_generate without a workspace argument, for callers that cannot hand
 * the library scratch memory: a program whose device memory is all held by
 * its own pool (a caching allocator, or a solver that sized A, LU and the
 * solve workspace to fill HBM), or one that must not call cudaMalloc/cudaFree
 * around generation because those calls synchronize the device.  The paper
 * has no counterpart: this is a convenience of this library.
 *
 * Same arguments, output and bit-for-bit result as hpmxp_generate.  The 16 n
 * bytes of 128-bit row sums live in a fixed 2 MiB array inside libhpmxp.so,
 * which every GPU that loads the library holds until the process exits; this
 * call allocates nothing.  The array is cleared on `stream` at the start of
 * every call.
 *
 *   n > 131072   HPMXP_ENOMEM (the fixed array holds 131072 rows); nothing runs
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it; make that first call before any stream
 * capture begins.  A reset of the device's primary context (cudaDeviceReset)
 * invalidates the kept address: calling this entry point after such a reset
 * is not supported.  All calls on a device share the one array: two calls whose
 * work overlaps on the GPU (different streams, no ordering between them) race
 * on it and give wrong diagonals.  Order such calls on one stream or by events. */
hpmxp_status hpmxp_generate_noalloc(int64_t n, uint64_t seed, double margin, int diag_mode, double* A,
                                    int64_t lda, double* b, int64_t ldb, int64_t nrhs, void* stream);

/* ------------------------------------------------------------------------ */
/* Low-precision LU without pivoting (section "Algorithmic Framework", Fig. 1).
 *
 * Casts A (fp64) to the factor format (round to nearest even) and factors it
 * in place, right-looking, with Schur-update depth `nb` (128, 256 or 512):
 * the diagonal block is factored in fp32 arithmetic (recursively at depth 128),
 * the panels are formed by multiplying with fp32-inverted 128x128 diagonal
 * blocks, and the trailing update A22 <- A22 - L21 U12 is a tensor-core product
 * of low-precision operands accumulated in fp32 and rounded once into storage.
 *
 *   A        in, n x n fp64, lda >= n (not modified)
 *   prec     hpmxp_prec
 *   LU       out, n x n 16-bit (BF16 for HPMXP_BF16, HPMXP_FP8_E4M3 and
 *            HPMXP_BF16_TRAIL32, FP16 for HPMXP_FP16 and HPMXP_FP16_TRAIL32),
 *            column major; unit-lower L below the diagonal, U on and above it.
 *            ldlu >= n, ldlu % 8 == 0, LU 16-byte aligned.
 * The TRAIL32 formats take 4 n^2 bytes more workspace (the fp32 matrix) and
 * run without the look-ahead schedule.
 *   ws       scratch of hpmxp_factor_workspace(n, prec, nb) bytes
 * Returns HPMXP_EBREAKDOWN when a pivot is zero or not finite (the factors are
 * then unusable). */
size_t hpmxp_factor_workspace(int64_t n, int prec, int nb);
hpmxp_status hpmxp_factor(int64_t n, const double* A, int64_t lda, int prec, int nb, void* LU,
                          int64_t ldlu, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Balancing and scaling (section "Algorithmic Framework": implementations may
 * balance the input matrix with Theta(n^2) work, as the HPL harness does, and
 * scale it so that its values fit the low-precision format; both are part of
 * the timed solve and are undone at the end).
 *
 * hpmxp_balance computes power-of-two row and column scales of A:
 *   rs_i = 2^-floor(log2 max_j |a_ij|),  cs_j = 2^-floor(log2 max_i |rs_i a_ij|),
 * so that the largest magnitude of every row and column of diag(rs) A diag(cs)
 * lies in [1, 2); then rs is multiplied by the format's scale, 2^12 for FP16
 * (values up to 2^13 leave room below 65504 for the growth of the Schur
 * complements and keep the small entries out of FP16's subnormal range), 1 for
 * BF16 and FP8 (fp32's exponent range).  A zero or non-finite row or column
 * gets scale 1.  Two passes over A (16 n^2 bytes); the result does not depend
 * on the order of the reductions.
 *   A        in, n x n fp64, lda >= n
 *   prec     hpmxp_prec the factors will have
 *   rs, cs   out, n fp64 each (device, distinct, 8-byte aligned)
 *
 * hpmxp_factor_scaled factors diag(rs) A diag(cs) (hpmxp_factor with the
 * scales applied exactly, before the one rounding to the factor format);
 * hpmxp_solve_ir_scaled refines x for the ORIGINAL A and b with those factors,
 * using M^{-1} = diag(cs) U^{-1} L^{-1} diag(rs): the balancing is undone in
 * every preconditioner application, and x, the residuals and the scaled
 * residual are those of the input system.  rs and cs must both be given or
 * both be NULL (no balancing: the plain calls).  Because the scales are powers
 * of two, a BF16 factorization of a system whose values stay inside the
 * fp32 normal range gives factors that are exact rescalings of the unbalanced
 * ones, and the same x bit for bit. */
hpmxp_status hpmxp_balance(int64_t n, const double* A, int64_t lda, int prec, double* rs, double* cs,
                           void* stream);
hpmxp_status hpmxp_factor_scaled(int64_t n, const double* A, int64_t lda, int prec, int nb, const double* rs,
                                 const double* cs, void* LU, int64_t ldlu, void* ws, size_t ws_bytes,
                                 void* stream);

/* ------------------------------------------------------------------------ */
/* GMRES-based iterative refinement (section "Algorithmic Framework").
 *
 * x0 = U^{-1} L^{-1} b from the low-precision factors, then repeatedly
 * r = b - A x in fp64; stop when the HPL scaled residual
 * ||r||_inf / ((||A||_inf ||x||_inf + ||b||_inf) n 2^-53) < accept; otherwise run
 * restarted GMRES(restart) on M^{-1} A d = M^{-1} r with M = LU as a LEFT
 * preconditioner (modified Gram-Schmidt Arnoldi, Givens rotations, fp64) and
 * update x += d.  More than max_iters inner iterations in total is a failure
 * (the paper's 50-iteration rule).  An inner cycle stops once the
 * least-squares residual estimate |g_{j+1}| <= beta * max(inner_tol,
 * theta * accept / sr0), sr0 being the scaled residual when the cycle starts. */
typedef struct {
  int32_t restart;       /* GMRES restart length m, 1..64 (default 30) */
  int32_t max_iters;     /* cap on inner iterations summed over restarts (default 50) */
  double inner_tol;      /* relative floor of the inner stopping test (default 1e-12) */
  double theta;          /* adaptive inner-stopping factor, 0 disables (default 0.1) */
  double accept;         /* acceptance threshold of the scaled residual (default 16) */
  int32_t precond_fp32;  /* 1: the preconditioner M^{-1} = U^{-1} L^{-1} applied in fp32 arithmetic
                            (x0, each cycle's start and each Arnoldi step); 0: fp64 (default 0) */
  int32_t matvec_fp32;   /* 1: the Arnoldi product A v of the inner GMRES in fp32 (A truncated toward
                            zero, fp32 accumulation); 0: fp64 (default 0).  The outer residual
                            b - A x, the orthogonalization, rotations, update and the acceptance
                            check are fp64 whatever these two fields say */
} hpmxp_ir_params;

typedef struct {
  int32_t iters;         /* inner (Arnoldi) iterations, summed over restarts */
  int32_t outer;         /* restart cycles started */
  double scaled_resid;   /* scaled residual of the returned x */
  int32_t status;        /* hpmxp_status of this right-hand side */
  int32_t reserved;
} hpmxp_ir_info;

/* Fills *p with the defaults listed above. */
void hpmxp_ir_params_default(hpmxp_ir_params* p);

/*   A        in, n x n fp64, lda >= n
 *   LU       in, factors from hpmxp_factor with the same n and prec, ldlu as there
 *   b        in, n x nrhs fp64, ldb >= n
 *   x        out, n x nrhs fp64, ldx >= n; holds the last iterate even on failure
 *   nrhs     1..8 right-hand sides, refined together (one pass over A and LU per
 *            iteration serves all of them)
 *   prm      host, NULL for the defaults
 *   info     host, nrhs entries (may be NULL)
 *   ws       scratch of hpmxp_solve_workspace(n, nrhs, restart) bytes
 * Synchronizes `stream`.  Returns HPMXP_OK when every right-hand side met the
 * threshold, else the worst per-column status (ENOCONV, EBREAKDOWN). */
size_t hpmxp_solve_workspace(int64_t n, int64_t nrhs, int restart);

/* Optional room for an fp32 copy of A (truncated toward zero), used when
 * prm->matvec_fp32 = 1 and ws_bytes >= hpmxp_solve_workspace(n, nrhs,
 * restart) + hpmxp_solve_workspace_a32(n): the first residual of the solve
 * writes the copy as it reads A, and the inner GMRES operator's products read
 * it (4 bytes per entry instead of 8).  The products, and so every result, are
 * bit-for-bit those computed from A itself.  4 n^2 bytes, rounded up. */
size_t hpmxp_solve_workspace_a32(int64_t n);
hpmxp_status hpmxp_solve_ir(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu,
                            int prec, const double* b, int64_t ldb, double* x, int64_t ldx,
                            int64_t nrhs, const hpmxp_ir_params* prm, hpmxp_ir_info* info,
                            void* ws, size_t ws_bytes, void* stream);
/* hpmxp_solve_ir with the factors of diag(rs) A diag(cs) (see hpmxp_balance). */
hpmxp_status hpmxp_solve_ir_scaled(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu,
                                   int prec, const double* rs, const double* cs, const double* b, int64_t ldb,
                                   double* x, int64_t ldx, int64_t nrhs, const hpmxp_ir_params* prm,
                                   hpmxp_ir_info* info, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches of independent systems of different sizes (the same method per
 * system, section "Algorithmic Framework"; batching many small systems is this
 * library's serving use, the paper has one large system per run).
 *
 * Each hpmxp_problem names one system's caller-owned device buffers.  The
 * batched calls run all systems in lockstep with Schur-update depth 128: one
 * grouped launch per stage serves every system that is still active (one CTA
 * per system's diagonal block; one tensor-core launch walking all systems'
 * tiles for each of the row-panel, column-panel and Schur products), so a
 * batch of B systems of order up to N takes about 5 N / 128 launches instead
 * of 5 sum_b n_b / 128.  Each system's factors are bit-for-bit those of
 * hpmxp_factor(n_b, ..., nb = 128) of it alone (the same kernels compute every
 * tile).  Formats: HPMXP_BF16 and HPMXP_FP16. */
typedef struct {
  int64_t n;            /* order, 1..131072 */
  const double* A;      /* n x n fp64, column major, lda >= n */
  int64_t lda;
  void* LU;             /* factors, n x n 16-bit, ldlu >= n, ldlu % 8 == 0, 16-byte aligned */
  int64_t ldlu;
  const double* b;      /* right-hand sides, n x nrhs (the solve only) */
  int64_t ldb;
  double* x;            /* solutions, n x nrhs (the solve only) */
  int64_t ldx;
  int64_t nrhs;         /* 1..8 (the solve only) */
} hpmxp_problem;

/* probs: host array of `count` descriptors.  status: host, count entries (may
 * be NULL): each system's status (HPMXP_EBREAKDOWN for a zero or non-finite
 * pivot).  Returns HPMXP_OK when every system factored, else the first
 * failure.  Synchronizes `stream`. */
size_t hpmxp_factor_batched_workspace(const hpmxp_problem* probs, int count, int prec);
hpmxp_status hpmxp_factor_batched(const hpmxp_problem* probs, int count, int prec, hpmxp_status* status, void* ws,
                                  size_t ws_bytes, void* stream);

/* GMRES-IR of every system with its factors from hpmxp_factor_batched (or
 * hpmxp_factor), the parameters of hpmxp_solve_ir shared by all.  The systems
 * advance in lockstep: one host decision point per refinement phase for the
 * whole batch (each system's kernels on one of the library's streams, so small
 * systems run side by side), instead of one per system.  info: host, sum of
 * nrhs entries in problem order (may be NULL).  Returns HPMXP_OK when every
 * right-hand side of every system met the threshold, else the first failure.
 * Synchronizes `stream`. */
size_t hpmxp_solve_ir_batched_workspace(const hpmxp_problem* probs, int count, int restart);
hpmxp_status hpmxp_solve_ir_batched(const hpmxp_problem* probs, int count, int prec, const hpmxp_ir_params* prm,
                                    hpmxp_ir_info* info, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Backward-error check (section "Algorithmic Framework"): for every column c,
 * scaled_resid[c] = ||A x_c - b_c||_inf / ((||A||_inf ||x_c||_inf + ||b_c||_inf) n eps)
 * with eps = 2^-53, all in fp64.  The solution is valid when it is < 16.
 *   scaled_resid  host, nrhs entries
 *   ws            scratch of hpmxp_residual_workspace(n, nrhs) bytes
 * Synchronizes `stream`. */
size_t hpmxp_residual_workspace(int64_t n, int64_t nrhs);
hpmxp_status hpmxp_residual(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                            const double* b, int64_t ldb, int64_t nrhs, double* scaled_resid,
                            void* ws, size_t ws_bytes, void* stream);

/* r = b - A x for every column, fp64 (the refinement's residual kernels):
 *   r   out, n x nrhs fp64 (ldr >= n); the other arguments as hpmxp_residual. */
hpmxp_status hpmxp_residual_vector(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                                   const double* b, int64_t ldb, int64_t nrhs, double* r, int64_t ldr, void* ws,
                                   size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* FP64 LU without pivoting, for the study of section "Experimental Results"
 * (Figs. 2-4: the largest pivot and the residual norms of 64-bit LU with and
 * without partial pivoting on matrices with and without diagonal scaling).
 *
 * hpmxp_lu_f64 factors A in place, A = L U (unit-lower L below the diagonal,
 * U on and above), right-looking with block width 64, fp64 arithmetic in the
 * plain order: unblocked diagonal blocks (l = a / pivot, then one fused
 * multiply-add per update, pivots ascending), panels by substitution (terms
 * ascending, one division per L entry), trailing update one fp64 accumulation
 * over the 64 terms in ascending order per entry.  Returns HPMXP_EBREAKDOWN on
 * a zero or non-finite pivot (the factors then hold what was computed).
 *   A    in/out, n x n fp64, lda >= n
 *   ws   scratch of hpmxp_lu_f64_workspace(n) bytes (256-byte aligned)
 * Synchronizes `stream`.
 *
 * hpmxp_lu_solve_f64 overwrites B (n x nrhs, 1 <= nrhs <= 64) with
 * U^{-1} L^{-1} B for those factors (64-row blocks: substitution in the
 * diagonal block, a fp64 product into the rows after it). */
size_t hpmxp_lu_f64_workspace(int64_t n);
hpmxp_status hpmxp_lu_f64(int64_t n, double* A, int64_t lda, void* ws, size_t ws_bytes, void* stream);
hpmxp_status hpmxp_lu_solve_f64(int64_t n, const double* LU, int64_t ld, double* B, int64_t ldb, int64_t nrhs,
                                void* stream);

/* ------------------------------------------------------------------------ */
/* Schedule tuning of the factorization (this library's knobs; the paper has
 * no counterpart).  Process-wide, read by every factorization started
 * afterwards; a field of 0 keeps the built-in choice.  The autotuner
 * (autotune.py) searches them together with nb.
 *   gemm_tile     tile height of the 16-bit products with M, K >= 256: 128 or 256
 *                 (0: 256)
 *   reserve_sms   SMs kept free of the far Schur update for the next panel chain
 *                 in the look-ahead schedule (0: SMs / 16, at least 4)
 *   overlap_min   smallest far-update order run concurrently with the next panel
 *                 chain (0: 8192)
 *   sm_budget     most SMs that one call's persistent tensor-core GEMM grid and
 *                 cooperative preconditioner grid take (0: all).  For many
 *                 solves sharing the GPU: a smaller grid leaves SMs free for the
 *                 other solves' latency-bound kernels.  The request executor
 *                 sets its own value for its workers (hpmxp_serve.h).
 * Environment variables HPMXP_GEMM_TILE, HPMXP_RESERVE_SMS, HPMXP_OVERLAP_MIN
 * and HPMXP_SM_BUDGET, when set, take precedence (they fix a setting for
 * experiments).  Returns HPMXP_EINVAL for values out of range. */
typedef struct {
  int32_t gemm_tile;
  int32_t reserve_sms;
  int64_t overlap_min;
  int32_t sm_budget;
  int32_t reserved;   /* 0 */
} hpmxp_tuning;
hpmxp_status hpmxp_set_tuning(const hpmxp_tuning* t);
void hpmxp_get_tuning(hpmxp_tuning* t);

/* ------------------------------------------------------------------------ */
/* Measurement support (the paper has no counterpart; used by the benchmark).
 * hpmxp_launch_count: kernels this library has launched since it was loaded.
 * hpmxp_prof_enable(1) makes the library record a CUDA event pair around
 * every launch of the timed kinds, on the launching stream:
 *   kind 0  tensor-core GEMM, Schur update (C -= A B^T)   work = 2 M N K flops per launch
 *   kind 1  fp64 GEMV (residual)    work = 8 n^2 bytes of A per launch
 *   kind 2  preconditioner apply    work = 2 n^2 bytes of factors per launch
 *   kind 3  diagonal-block getrf    work = 2 b^3 flops per launch
 *   kind 4  fp32 GEMV (Arnoldi product with the fp32 operator)  work = 8 n^2 bytes of A
 *   kind 5  fp64 -> 16-bit cast     work = 10 n^2 bytes per launch
 *   kind 6  panel operand kernels (column-panel pack, substitution operands)
 *   kind 7  tensor-core GEMM, panel products (C = sign A B^T)  work = 2 M N K flops
 *   kind 8  balancing (hpmxp_balance)  work = 16 n^2 bytes of A per call
 * hpmxp_prof_read synchronizes the recorded events and returns the summed
 * event time, work and launch count of one kind since the last reset.
 * Returns HPMXP_EINVAL for a bad kind or NULL output.
 * hpmxp_prof_timeline writes up to max_spans recorded spans since the last
 * reset as triples (kind, start ms, end ms) on one clock (the first span's
 * start is 0) into out (3 * max_spans doubles, may be NULL) and returns how
 * many spans there are. */
unsigned long long hpmxp_launch_count(void);
void hpmxp_prof_enable(int on);
void hpmxp_prof_reset(void);
int hpmxp_prof_read(int kind, double* total_ms, double* total_work, long long* launches);
/* Algorithmic DRAM bytes recorded for a kind since the last reset (the GEMM
 * kinds 0 and 7: operands once, C read and / or written once; 0 for the
 * others), for comparison with the bytes a profiler measures. */
int hpmxp_prof_read_bytes(int kind, double* total_bytes);
/* Execution time the kernels of a kind measured themselves since the last
 * reset (the GEMM kinds 0 and 7: the global timer from the first CTA's start
 * after its stream dependency to the last CTA's end, summed over launches),
 * and how many launches recorded one.  Beside streams that run concurrently
 * this excludes the time a launch waits for SMs, which the event time of
 * hpmxp_prof_read includes.  Returns HPMXP_EINVAL for a bad kind. */
int hpmxp_prof_read_device(int kind, double* total_ms, long long* launches);
int hpmxp_prof_timeline(double* out, int max_spans);

#ifdef __cplusplus
}
#endif
#endif /* HPMXP_H_ */
