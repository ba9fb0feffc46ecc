// Internal declarations shared by the translation units of libhpmxp.so.
// Not part of the public interface (include/hpmxp.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/hpmxp.h"

namespace hpmxp {

// ---------------------------------------------------------------------------
// Device status word.  Kernels never trap: a failed check or a bounded wait
// that runs out ORs a bit into a status word in the caller's workspace, and
// the host maps it to an hpmxp_status after synchronizing.
// ---------------------------------------------------------------------------
enum : uint32_t {
  kErrTimeout = 1u,     // a bounded device wait ran out
  kErrPivot = 2u,       // zero or non-finite pivot in a diagonal block
  kErrNonFinite = 4u,   // non-finite value in the refinement
  kErrBounds = 8u,      // a device-side bounds/shape check failed
};

// Bounds of every device-side wait: at most kSpinLimit polls and at most
// kWaitNs nanoseconds of the global timer (checked every 64 or 256 polls).  A
// legitimate wait here lasts microseconds to milliseconds.
constexpr long long kSpinLimit = 1ll << 28;
constexpr unsigned long long kWaitNs = 2000000000ull;

// The bound of the waits whose running out is an error (a peer CTA that never
// publishes, a pipeline stage that never fills) is passed to the kernels as
// an argument: the defaults above, unless the test hook
// hpmxp_test_set_wait_budget lowered it.  The waits with which a CTA drains
// its own copies and tensor-core work before it exits always keep the
// defaults, so a short budget cannot make a CTA leave work in flight.
struct WaitBudget {
  long long polls;
  unsigned long long ns;
};
WaitBudget wait_budget();

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Round up / ceil division helpers.
template <class T>
__host__ __device__ inline T cdiv(T a, T b) { return (a + b - 1) / b; }
template <class T>
__host__ __device__ inline T round_up(T a, T b) { return cdiv(a, b) * b; }

// 16-bit storage formats of the factors.
enum Fmt16 { kBF16 = 0, kFP16 = 1 };
// Storage format of the factors of a precision (hpmxp_prec).
inline int fmt_of(int prec) { return (prec == HPMXP_FP16 || prec == HPMXP_FP16_TRAIL32) ? kFP16 : kBF16; }
inline bool trail32_of(int prec) { return prec == HPMXP_BF16_TRAIL32 || prec == HPMXP_FP16_TRAIL32; }

__device__ inline float ld16(const uint16_t* p, int fmt) {
  const uint16_t h = *p;
  if (fmt == kBF16) return __uint_as_float((uint32_t)h << 16);
  return __half2float(__ushort_as_half(h));
}
__device__ inline float u16_to_f32(uint16_t h, int fmt) {
  if (fmt == kBF16) return __uint_as_float((uint32_t)h << 16);
  return __half2float(__ushort_as_half(h));
}
// The same value as an fp64, its bit pattern assembled with integer
// operations from the IEEE 754 fields (sign; exponent rebased from bias 127
// (BF16) or 15 (FP16) to 1023; fraction moved to the top of the 52-bit
// field; subnormals normalised by their leading one; Inf / NaN kept).  The
// conversion is exact, so the result equals (double)u16_to_f32(h, fmt); it
// keeps the conversion off GB300's narrow fp64 unit, which then does the
// FMAs only.
__device__ inline double u16_to_f64(uint16_t h, int fmt) {
  const uint32_t sgn = (uint32_t)(h & 0x8000u) << 16;
  const int fbits = fmt == kBF16 ? 7 : 10;                 // fraction bits
  const uint32_t emax = fmt == kBF16 ? 0xffu : 0x1fu;     // exponent field all ones
  const uint32_t bias_shift = fmt == kBF16 ? 896u : 1008u; // 1023 - 127, 1023 - 15
  const uint32_t e = ((uint32_t)h >> fbits) & emax, m = (uint32_t)h & ((1u << fbits) - 1u);
  uint32_t hi;
  if (e == emax) {
    hi = sgn | 0x7ff00000u | (m << (20 - fbits));
  } else if (e != 0) {
    hi = sgn | ((e + bias_shift) << 20) | (m << (20 - fbits));
  } else if (m == 0) {
    hi = sgn;
  } else {
    // subnormal m 2^(1 - bias - fbits) = 2^(p + 1 - bias - fbits) (1 + f), p = the leading one's bit
    const int p = 31 - __clz(m);
    const uint32_t f = (m << (fbits - p)) & ((1u << fbits) - 1u);
    hi = sgn | (((uint32_t)(p + 1 - fbits) + bias_shift) << 20) | (f << (20 - fbits));
  }
  return __hiloint2double((int)hi, 0);
}
__device__ inline uint16_t f32_to_u16(float v, int fmt) {
  if (fmt == kBF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  return __half_as_ushort(__float2half_rn(v));
}

// ---------------------------------------------------------------------------
// Launch helpers implemented in the .cu files.
// ---------------------------------------------------------------------------

// gen.cu
cudaError_t launch_generate(int64_t n, uint64_t seed, double margin, int mode, double* A,
                            int64_t lda, double* b, int64_t ldb, int64_t nrhs,
                            unsigned long long* sums, cudaStream_t st);

// GEMM engines (gemm_tc.cu: tcgen05 tensor cores; lu.cu: a SIMT validation
// engine that accumulates with one fp32 FMA per term in ascending k).
//
// D(i, j) for i < M, j < N is acc(i, j) = sum_{k < K} A(i, k) B(j, k), both
// operands K-major 16-bit (A(i,k) at A[i*lda + k], B(j,k) at B[j*ldb + k]),
// K a multiple of 128 (128-deep fp8 slices for the E4M3 kind).
// Epilogue (`mode`):
//   kEpiSub    C(i,j) = st(C(i,j) - acc)    C column major 16-bit, in place
//              (fp32 C with c32: C(i,j) = fl32(C(i,j) - acc), the fp32-stored trailing matrix)
//   kEpiStore  C(i,j) = st(sign * acc)      C column major (C may be NULL)
//              and, if R != NULL, R(i,j) = same value, R row major (R[i*ldr + j])
enum EpiMode { kEpiSub = 0, kEpiStore = 1 };
struct GemmArgs {
  int M, N, K;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  void* C; int64_t ldc;
  void* R; int64_t ldr;
  int mode;
  float sign;
  int fmt;              // kBF16 / kFP16 operands and outputs
  // E4M3 variant (operands are 8-bit, K-major, lda/ldb in elements=bytes):
  // scales sA[(i/128) * sa_ld + kb], sB[(j/128) * sb_ld + kb] per 128-deep slice kb.
  int fp8;
  const float* sA; int sa_ld;
  const float* sB; int sb_ld;
  uint32_t* status;
  int max_ctas;         // 0: one CTA per SM; else at most this many (leaves SMs for concurrent work)
  int c32;              // 1: C is fp32 column major (ldc in elements), mode kEpiSub: C = fl32(C - acc)
};
cudaError_t gemm_tc(const GemmArgs& g, cudaStream_t st);
cudaError_t gemm_simt(const GemmArgs& g, cudaStream_t st);

// Grouped launches of the tensor-core engine: several independent products of
// the same kind (same mode, sign, format and K, 16-bit operands, K < 256 so
// all take 128-row tiles, R given for all or none) in ONE launch, the
// persistent CTAs walking the concatenated tile lists.  One item per product,
// in device memory (its tensor maps are read from there by the TMA unit).
struct alignas(128) GemmGroupItem {
  unsigned char maps[3][128];   // CUtensorMap of A, B and C
  int M, N, tiles_i, tile_begin;
  void* R;
  int64_t ldr;
};
// Encodes the items of `count` products into `items` (host memory); returns
// false if they cannot share a launch.  *total_tiles receives the tile count.
bool gemm_group_encode(const GemmArgs* gs, int count, GemmGroupItem* items, int* total_tiles);
// Launches the grouped product: proto carries the shared fields (mode, sign,
// fmt, K, status, max_ctas), dev_items the encoded items copied to the device;
// flops and bytes (the items' total) only feed the optional event timing.
cudaError_t gemm_tc_grouped(const GemmArgs& proto, const GemmGroupItem* dev_items, int nitems, int total_tiles,
                            cudaStream_t st, double flops = 0.0, double bytes = 0.0);
// Returns the engine selected for the factorization (0 = tcgen05, 1 = SIMT
// validation engine, chosen by HPMXP_GEMM_ENGINE=simt for parity tests).
int gemm_engine();

// lu.cu
// rs / cs (optional, NULL = 1): the cast converts diag(rs) A diag(cs)
cudaError_t launch_cast(int64_t n, const double* A, int64_t lda, void* out, int64_t ldo, int fmt, cudaStream_t st,
                        const double* rs = nullptr, const double* cs = nullptr);
// power-of-two row / column equilibration and the format's scale into rs, cs (n each)
cudaError_t launch_balance(int64_t n, const double* A, int64_t lda, int prec, double* rs, double* cs,
                           cudaStream_t st);
size_t factor_ws_bytes(int64_t n, int prec, int nb);
size_t factor_batched_ws_bytes(const hpmxp_problem* probs, int count);
hpmxp_status factor_batched(const hpmxp_problem* probs, int count, int prec, hpmxp_status* status, void* ws,
                            size_t ws_bytes, cudaStream_t st);
hpmxp_status factor(int64_t n, const double* A, int64_t lda, int prec, int nb, void* LU,
                    int64_t ldlu, void* ws, size_t ws_bytes, cudaStream_t st, const double* rs = nullptr,
                    const double* cs = nullptr);

// study.cu: fp64 LU without pivoting (block 64, in place) and its solves
cudaError_t lu_f64(int64_t n, double* A, int64_t ld, uint32_t* status, cudaStream_t st);
cudaError_t lu_solve_f64(int64_t n, const double* LU, int64_t ld, double* X, int64_t ldx, int64_t nrhs,
                         cudaStream_t st);

// ir.cu
size_t solve_batched_ws_bytes(const hpmxp_problem* probs, int count, int restart);
size_t solve_ws_bytes(int64_t n, int64_t nrhs, int restart);
size_t solve_a32_bytes(int64_t n);   // optional fp32 copy of A after the solve workspace
cudaError_t fill_smem(uint32_t pattern, cudaStream_t st);   // test support
cudaError_t decode16(const uint16_t* codes, double* out, int64_t count, int fmt, cudaStream_t st);   // test support
size_t residual_ws_bytes(int64_t n, int64_t nrhs);
hpmxp_status precond_apply(int64_t n, const void* LU, int64_t ldlu, int fmt, const double* v, int64_t ldv,
                           double* z, int64_t ldz, int64_t nrhs, int fp32, void* ws, cudaStream_t st,
                           const double* rs = nullptr, const double* cs = nullptr);

// prof.cu: launch counting and optional event timing (kinds below).
enum ProfKind { kProfGemm = 0, kProfGemv = 1, kProfPrecond = 2, kProfGetrf = 3, kProfGemv32 = 4, kProfCast = 5,
                kProfPanel = 6, kProfGemmStore = 7, kProfBalance = 8, kProfKinds = 9 };
void count_launches(int k);
bool prof_on();
// Programmatic dependent launch.  A kernel launched by launch_pdl may start
// while the previous kernel of its stream is still running: it must call
// pdl_wait() before its first access to global memory (the wait returns once
// that kernel has completed and its writes are visible; it is a no-op for a
// normal launch).  pdl_trigger() lets the next such kernel start early.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif
bool pdl_enabled();   // HPMXP_PDL=0 turns it off (every launch_pdl becomes a plain launch)
// Schedule tuning (hpmxp_set_tuning, environment overrides applied): the
// effective values, 0 = built-in choice.
hpmxp_tuning tuning();
// SMs one call's persistent / cooperative grids may take, 0 = all: the calling
// thread's own value (SmBudgetScope) if set, else the process-wide tuning.
int sm_budget();
struct SmBudgetScope {
  explicit SmBudgetScope(int sms);
  ~SmBudgetScope();
  int prev;
};
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

void* prof_begin(cudaStream_t st);
// work: the kind's unit (flops or bytes, see hpmxp.h); bytes: algorithmic DRAM
// bytes of the launch where the kind records them (the GEMM kinds)
void prof_end(void* token, int kind, double work, cudaStream_t st, double bytes = 0.0);
// device execution span slot for the launch between prof_begin(token) and
// prof_end (kernels that record their own span); NULL when not measuring
unsigned long long* prof_device_span(void* token);

cudaError_t host_wait(cudaStream_t st);   // waits for `st` (spinning unless HPMXP_BLOCKING_WAIT=1)
cudaError_t read_to_host(void* dst, const void* src, size_t bytes, cudaStream_t st);   // + host_wait
hpmxp_status status_from_cuda(cudaError_t e);
hpmxp_status status_from_word(uint32_t w);

}  // namespace hpmxp
