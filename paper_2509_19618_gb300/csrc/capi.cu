// C interface of libhpmxp.so (declared in include/hpmxp.h): argument
// validation, workspace sizing and status mapping around the kernels.
#include "internal.h"
#include "../../include/hpmxp_testing.h"

#include <atomic>

namespace hpmxp {

namespace {
std::atomic<long long> g_wait_polls{kSpinLimit};
std::atomic<unsigned long long> g_wait_ns{kWaitNs};
}  // namespace

WaitBudget wait_budget() { return WaitBudget{g_wait_polls.load(), g_wait_ns.load()}; }

hpmxp_status status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HPMXP_OK;
  if (e == cudaErrorInvalidValue) return HPMXP_EINVAL;
  return HPMXP_ECUDA;
}

hpmxp_status status_from_word(uint32_t w) {
  if (w & kErrTimeout) return HPMXP_ETIMEOUT;
  if (w & kErrBounds) return HPMXP_EINVAL;
  if (w & (kErrPivot | kErrNonFinite)) return HPMXP_EBREAKDOWN;
  return HPMXP_OK;
}

hpmxp_status solve_ir(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu, int prec,
                      const double* b, int64_t ldb, double* x, int64_t ldx, int64_t nrhs,
                      const hpmxp_ir_params& prm, hpmxp_ir_info* info, void* ws, size_t ws_bytes,
                      cudaStream_t st, const double* rs = nullptr, const double* cs = nullptr);
hpmxp_status residual_check(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                            const double* b, int64_t ldb, int64_t nrhs, double* out, void* ws, cudaStream_t st);
size_t solve_batched_ws_bytes(const hpmxp_problem* probs, int count, int restart);
hpmxp_status solve_ir_batched(const hpmxp_problem* probs, int count, int prec, const hpmxp_ir_params& prm,
                              hpmxp_ir_info* info, void* ws, cudaStream_t caller);
hpmxp_status residual_vector(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                             const double* b, int64_t ldb, int64_t nrhs, double* r, int64_t ldr, void* ws,
                             cudaStream_t st);

}  // namespace hpmxp

using namespace hpmxp;

namespace {
constexpr int64_t kMaxN = int64_t(1) << 17;
bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
bool prec_ok(int p) { return p >= HPMXP_BF16 && p <= HPMXP_FP16_TRAIL32; }
}  // namespace

extern "C" {

const char* hpmxp_status_string(hpmxp_status s) {
  switch (s) {
    case HPMXP_OK: return "ok";
    case HPMXP_EINVAL: return "invalid argument";
    case HPMXP_ENOMEM: return "workspace too small";
    case HPMXP_ECUDA: return "CUDA error";
    case HPMXP_ENOCONV: return "refinement did not converge within max_iters";
    case HPMXP_EBREAKDOWN: return "breakdown: zero or non-finite pivot or value";
    case HPMXP_ETIMEOUT: return "a bounded device wait ran out";
    case HPMXP_EINVALID: return "scaled residual above the acceptance threshold";
    default: return "unknown status";
  }
}

int hpmxp_version(void) { return 10000; }

size_t hpmxp_generate_workspace(int64_t n) { return n > 0 ? round_up<size_t>(16 * (size_t)n, 256) : 0; }

hpmxp_status hpmxp_generate(int64_t n, uint64_t seed, double margin, int diag_mode, double* A, int64_t lda,
                            double* b, int64_t ldb, int64_t nrhs, void* ws, size_t ws_bytes, void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || nrhs < 0 || (nrhs > 0 && (!b || ldb < n)) || !ws)
    return HPMXP_EINVAL;
  if (diag_mode < HPMXP_DIAG_DOMINANT || diag_mode > HPMXP_DIAG_DEPARTURE) return HPMXP_EINVAL;
  if (diag_mode == HPMXP_DIAG_DEPARTURE && !(margin > 0.0)) return HPMXP_EINVAL;
  if (!aligned(ws, 16)) return HPMXP_EINVAL;
  if (ws_bytes < hpmxp_generate_workspace(n)) return HPMXP_ENOMEM;
  cudaError_t e = launch_generate(n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, (unsigned long long*)ws,
                                  (cudaStream_t)stream);
  return status_from_cuda(e);
}

size_t hpmxp_factor_workspace(int64_t n, int prec, int nb) {
  if (n < 1 || !prec_ok(prec) || !(nb == 128 || nb == 256 || nb == 512)) return 0;
  return factor_ws_bytes(n, prec, nb);
}

hpmxp_status hpmxp_factor_scaled(int64_t n, const double* A, int64_t lda, int prec, int nb, const double* rs,
                                 const double* cs, void* LU, int64_t ldlu, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || !LU || ldlu < n || (ldlu % 8) != 0 || !aligned(LU, 16) || !ws ||
      !aligned(ws, 256) || !prec_ok(prec) || !(nb == 128 || nb == 256 || nb == 512) || (!rs != !cs))
    return HPMXP_EINVAL;
  if (ws_bytes < factor_ws_bytes(n, prec, nb)) return HPMXP_ENOMEM;
  return factor(n, A, lda, prec, nb, LU, ldlu, ws, ws_bytes, (cudaStream_t)stream, rs, cs);
}

hpmxp_status hpmxp_factor(int64_t n, const double* A, int64_t lda, int prec, int nb, void* LU, int64_t ldlu,
                          void* ws, size_t ws_bytes, void* stream) {
  return hpmxp_factor_scaled(n, A, lda, prec, nb, nullptr, nullptr, LU, ldlu, ws, ws_bytes, stream);
}

namespace {
bool batch_problem_ok(const hpmxp_problem& q, bool solve) {
  if (q.n < 1 || q.n > kMaxN || !q.A || q.lda < q.n || !q.LU || q.ldlu < q.n || (q.ldlu % 8) || !aligned(q.LU, 16))
    return false;
  if (solve && (!q.b || q.ldb < q.n || !q.x || q.ldx < q.n || q.nrhs < 1 || q.nrhs > 8)) return false;
  return true;
}
}  // namespace

size_t hpmxp_factor_batched_workspace(const hpmxp_problem* probs, int count, int prec) {
  if (!probs || count < 1 || !(prec == HPMXP_BF16 || prec == HPMXP_FP16)) return 0;
  for (int q = 0; q < count; ++q)
    if (probs[q].n < 1 || probs[q].n > kMaxN) return 0;
  return factor_batched_ws_bytes(probs, count);
}

hpmxp_status hpmxp_factor_batched(const hpmxp_problem* probs, int count, int prec, hpmxp_status* status, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!probs || count < 1 || !(prec == HPMXP_BF16 || prec == HPMXP_FP16) || !ws || !aligned(ws, 256))
    return HPMXP_EINVAL;
  for (int q = 0; q < count; ++q)
    if (!batch_problem_ok(probs[q], false)) return HPMXP_EINVAL;
  if (ws_bytes < factor_batched_ws_bytes(probs, count)) return HPMXP_ENOMEM;
  return factor_batched(probs, count, prec, status, ws, ws_bytes, (cudaStream_t)stream);
}

size_t hpmxp_solve_ir_batched_workspace(const hpmxp_problem* probs, int count, int restart) {
  if (!probs || count < 1 || restart < 1 || restart > 64) return 0;
  for (int q = 0; q < count; ++q)
    if (probs[q].n < 1 || probs[q].n > kMaxN || probs[q].nrhs < 1 || probs[q].nrhs > 8) return 0;
  return solve_batched_ws_bytes(probs, count, restart);
}

hpmxp_status hpmxp_solve_ir_batched(const hpmxp_problem* probs, int count, int prec, const hpmxp_ir_params* prm,
                                    hpmxp_ir_info* info, void* ws, size_t ws_bytes, void* stream) {
  hpmxp_ir_params p;
  hpmxp_ir_params_default(&p);
  if (prm) p = *prm;
  if (!probs || count < 1 || !prec_ok(prec) || !ws || !aligned(ws, 256) || p.restart < 1 || p.restart > 64 ||
      p.max_iters < 0 || !(p.accept > 0.0) || p.inner_tol < 0.0 || p.theta < 0.0 ||
      (p.precond_fp32 != 0 && p.precond_fp32 != 1) || (p.matvec_fp32 != 0 && p.matvec_fp32 != 1))
    return HPMXP_EINVAL;
  for (int q = 0; q < count; ++q)
    if (!batch_problem_ok(probs[q], true)) return HPMXP_EINVAL;
  if (ws_bytes < solve_batched_ws_bytes(probs, count, p.restart)) return HPMXP_ENOMEM;
  return solve_ir_batched(probs, count, prec, p, info, ws, (cudaStream_t)stream);
}

hpmxp_status hpmxp_balance(int64_t n, const double* A, int64_t lda, int prec, double* rs, double* cs,
                           void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || !rs || !cs || rs == cs || !aligned(rs, 8) || !aligned(cs, 8) ||
      !prec_ok(prec))
    return HPMXP_EINVAL;
  return status_from_cuda(launch_balance(n, A, lda, prec, rs, cs, (cudaStream_t)stream));
}

void hpmxp_ir_params_default(hpmxp_ir_params* p) {
  if (!p) return;
  p->restart = 30;
  p->max_iters = 50;
  p->inner_tol = 1e-12;
  p->theta = 0.1;
  p->accept = 16.0;
  p->precond_fp32 = 0;
  p->matvec_fp32 = 0;
}

size_t hpmxp_solve_workspace(int64_t n, int64_t nrhs, int restart) {
  if (n < 1 || nrhs < 1 || nrhs > 8 || restart < 1 || restart > 64) return 0;
  return solve_ws_bytes(n, nrhs, restart);
}

size_t hpmxp_solve_workspace_a32(int64_t n) { return n < 1 ? 0 : solve_a32_bytes(n); }

hpmxp_status hpmxp_solve_ir(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu, int prec,
                            const double* b, int64_t ldb, double* x, int64_t ldx, int64_t nrhs,
                            const hpmxp_ir_params* prm, hpmxp_ir_info* info, void* ws, size_t ws_bytes,
                            void* stream) {
  return hpmxp_solve_ir_scaled(n, A, lda, LU, ldlu, prec, nullptr, nullptr, b, ldb, x, ldx, nrhs, prm, info, ws,
                               ws_bytes, stream);
}

hpmxp_status hpmxp_solve_ir_scaled(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu,
                                   int prec, const double* rs, const double* cs, const double* b, int64_t ldb,
                                   double* x, int64_t ldx, int64_t nrhs, const hpmxp_ir_params* prm,
                                   hpmxp_ir_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (!rs != !cs) return HPMXP_EINVAL;
  hpmxp_ir_params p;
  hpmxp_ir_params_default(&p);
  if (prm) p = *prm;
  if (n < 1 || n > kMaxN || !A || lda < n || !LU || ldlu < n || !b || ldb < n || !x || ldx < n || nrhs < 1 ||
      nrhs > 8 || !ws || !aligned(ws, 256) || !prec_ok(prec) || p.restart < 1 || p.restart > 64 ||
      p.max_iters < 0 || !(p.accept > 0.0) || p.inner_tol < 0.0 || p.theta < 0.0 ||
      (p.precond_fp32 != 0 && p.precond_fp32 != 1) || (p.matvec_fp32 != 0 && p.matvec_fp32 != 1))
    return HPMXP_EINVAL;
  if (ws_bytes < solve_ws_bytes(n, nrhs, p.restart)) return HPMXP_ENOMEM;
  return solve_ir(n, A, lda, LU, ldlu, prec, b, ldb, x, ldx, nrhs, p, info, ws, ws_bytes, (cudaStream_t)stream, rs,
                  cs);
}

size_t hpmxp_residual_workspace(int64_t n, int64_t nrhs) {
  if (n < 1 || nrhs < 1 || nrhs > 8) return 0;
  return residual_ws_bytes(n, nrhs);
}

hpmxp_status hpmxp_residual(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                            const double* b, int64_t ldb, int64_t nrhs, double* scaled_resid, void* ws,
                            size_t ws_bytes, void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || !x || ldx < n || !b || ldb < n || nrhs < 1 || nrhs > 8 ||
      !scaled_resid || !ws || !aligned(ws, 256))
    return HPMXP_EINVAL;
  if (ws_bytes < residual_ws_bytes(n, nrhs)) return HPMXP_ENOMEM;
  return residual_check(n, A, lda, x, ldx, b, ldb, nrhs, scaled_resid, ws, (cudaStream_t)stream);
}

hpmxp_status hpmxp_residual_vector(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                                   const double* b, int64_t ldb, int64_t nrhs, double* r, int64_t ldr, void* ws,
                                   size_t ws_bytes, void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || !x || ldx < n || !b || ldb < n || !r || ldr < n || nrhs < 1 ||
      nrhs > 8 || !ws || !aligned(ws, 256))
    return HPMXP_EINVAL;
  if (ws_bytes < residual_ws_bytes(n, nrhs)) return HPMXP_ENOMEM;
  return residual_vector(n, A, lda, x, ldx, b, ldb, nrhs, r, ldr, ws, (cudaStream_t)stream);
}

size_t hpmxp_lu_f64_workspace(int64_t n) { return n < 1 ? 0 : 256; }

hpmxp_status hpmxp_lu_f64(int64_t n, double* A, int64_t lda, void* ws, size_t ws_bytes, void* stream) {
  if (n < 1 || n > kMaxN || !A || lda < n || !ws || !aligned(ws, 256)) return HPMXP_EINVAL;
  if (ws_bytes < hpmxp_lu_f64_workspace(n)) return HPMXP_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* status = (uint32_t*)ws;
  cudaError_t e = cudaMemsetAsync(status, 0, 4, st);
  if (e == cudaSuccess) e = lu_f64(n, A, lda, status, st);
  uint32_t word = 0;
  if (e == cudaSuccess) e = read_to_host(&word, status, 4, st);
  if (e != cudaSuccess) return status_from_cuda(e);
  return status_from_word(word);
}

hpmxp_status hpmxp_lu_solve_f64(int64_t n, const double* LU, int64_t ld, double* B, int64_t ldb, int64_t nrhs,
                                void* stream) {
  if (n < 1 || n > kMaxN || !LU || ld < n || !B || ldb < n || nrhs < 1 || nrhs > 64) return HPMXP_EINVAL;
  return status_from_cuda(lu_solve_f64(n, LU, ld, B, ldb, nrhs, (cudaStream_t)stream));
}

// ---------------------------------------------------------------------------
// Test hooks (include/hpmxp_testing.h)
// ---------------------------------------------------------------------------
hpmxp_status hpmxp_test_gemm(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb,
                             void* C, int64_t ldc, void* R, int64_t ldr, int mode, float sign, int fmt,
                             int fp8, const float* sA, int sa_ld, const float* sB, int sb_ld, int engine,
                             uint32_t* status, void* stream) {
  const int c32 = mode == 2;   // fp32 C, subtract mode
  if (c32) mode = kEpiSub;
  if (M < 0 || N < 0 || K <= 0 || (K % 128) || !A || !B || !status || (mode == kEpiSub && !C) ||
      (mode != kEpiSub && mode != kEpiStore) || (fmt != kBF16 && fmt != kFP16) ||
      (fp8 && (!sA || !sB || K > 512)) || (!C && !R) || (c32 && (R || fp8)))
    return HPMXP_EINVAL;
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.R = R; g.ldr = ldr; g.mode = mode; g.sign = sign; g.fmt = fmt; g.fp8 = fp8; g.c32 = c32;
  g.sA = sA; g.sa_ld = sa_ld; g.sB = sB; g.sb_ld = sb_ld; g.status = status;
  cudaError_t e = engine == 1 ? gemm_simt(g, (cudaStream_t)stream) : gemm_tc(g, (cudaStream_t)stream);
  return status_from_cuda(e);
}

hpmxp_status hpmxp_test_cast(int64_t n, const double* A, int64_t lda, int prec, void* out, int64_t ldo,
                             void* stream) {
  if (n < 1 || !A || lda < n || !out || ldo < n || (ldo % 8) || !aligned(out, 16) || !prec_ok(prec))
    return HPMXP_EINVAL;
  return status_from_cuda(launch_cast(n, A, lda, out, ldo, fmt_of(prec),
                                      (cudaStream_t)stream));
}

hpmxp_status hpmxp_test_precond(int64_t n, const void* LU, int64_t ldlu, int prec, const double* v,
                                int64_t ldv, double* z, int64_t ldz, int64_t nrhs, int fp32, void* ws,
                                size_t ws_bytes, void* stream) {
  if (n < 1 || n > kMaxN || !LU || ldlu < n || !v || ldv < n || !z || ldz < n || nrhs < 1 || nrhs > 8 ||
      !ws || !aligned(ws, 256) || !prec_ok(prec))
    return HPMXP_EINVAL;
  if (ws_bytes < solve_ws_bytes(n, nrhs, 1)) return HPMXP_ENOMEM;
  return precond_apply(n, LU, ldlu, fmt_of(prec), v, ldv, z, ldz, nrhs, fp32, ws,
                       (cudaStream_t)stream);
}

hpmxp_status hpmxp_test_set_wait_budget(long long polls, unsigned long long ns) {
  if (polls == 0 && ns == 0) {
    g_wait_polls.store(kSpinLimit);
    g_wait_ns.store(kWaitNs);
    return HPMXP_OK;
  }
  if (polls < 1 || polls > kSpinLimit || ns > kWaitNs) return HPMXP_EINVAL;
  g_wait_polls.store(polls);
  g_wait_ns.store(ns);
  return HPMXP_OK;
}

hpmxp_status hpmxp_test_fill_smem(uint32_t pattern, void* stream) {
  return status_from_cuda(fill_smem(pattern, (cudaStream_t)stream));
}

hpmxp_status hpmxp_test_decode16(const uint16_t* codes, double* out, int64_t count, int fmt, void* stream) {
  if (count < 0 || (count > 0 && (!codes || !out)) || (fmt != HPMXP_BF16 && fmt != HPMXP_FP16)) return HPMXP_EINVAL;
  return status_from_cuda(decode16(codes, out, count, fmt, (cudaStream_t)stream));
}

}  // extern "C"
