// fp64 GMRES-based iterative refinement (section "Algorithmic Framework":
// x0 from the low-precision factors, then GMRES with the factors as a left
// preconditioner, fp64 working precision, at most 50 iterations, HPL
// backward-error criterion below 16).
//
// Kernels:
//   gemv_partial / gemv_finish  r = b - A x for up to 8 columns; A (fp64,
//       column major) is read once for all columns, coalesced 16-byte loads,
//       split over column chunks with a deterministic second pass.  The
//       first pass can also accumulate |A| row sums (||A||_inf).
//   precond_kernel<T>  z = U^{-1} L^{-1} v with the 16-bit factors, in T =
//       float or double arithmetic, both sweeps in one cooperative launch:
//       block rows of 128 are owned round-robin by the CTAs; the owner of a
//       block solves it (a product with the inverted diagonal block) as soon
//       as every earlier block has been applied, and publishes it as tagged
//       64-bit words that the other CTAs poll (bounded).
//   mgs_step / vec_norm / givens / cycle_start / cycle_finish / update:
//       modified Gram-Schmidt Arnoldi, Givens least squares, x += V y.
// All control decisions are taken on the device; the host reads a few
// words per Arnoldi step to decide whether to launch the next one.
#include "internal.h"

#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

namespace hpmxp {
namespace {

constexpr int kMaxM = 64;     // largest restart length
constexpr int kMaxK = 8;      // right-hand sides refined together
constexpr int kRedBlocks = 304;

__device__ inline unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ inline double bits_d(unsigned long long b) { return __longlong_as_double((long long)b); }

// |a| as an fp32 lower bound from the top word of the fp64 pattern (exponent
// rebias, 20 mantissa bits, tiny values flushed to 0): integer ops only, so
// the ||A||_inf estimate of the stopping test costs no fp64 instructions.
__device__ inline float abs_f32_est(double a) {
  const int hi = __double2hiint(a) & 0x7fffffff;
  const int t = hi - (896 << 20);
  return t > 0 ? __int_as_float(min(t, 0x7f7fffff >> 3) << 3) : 0.0f;
}

// fp64 -> fp32 truncated toward zero, integer operations only (exponent
// rebias and the top 23 mantissa bits; values below the fp32 normal range
// flush to zero, which the generated systems never produce).
__device__ inline float trunc_f32(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const int e = (int)((hi >> 20) & 0x7ff) - 896;          // fp32 biased exponent
  const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t sign = hi & 0x80000000u;
  return e > 0 ? __uint_as_float(sign | ((uint32_t)min(e, 255) << 23) | mant) : __uint_as_float(sign);
}

// ---------------------------------------------------------------------------
// Per right-hand-side state of the refinement (device memory).
// ---------------------------------------------------------------------------
struct RhsState {
  double H[(kMaxM + 1) * kMaxM];   // Hessenberg, column major (m+1) x m
  double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
  double beta, tol, sr, hn;
  double anorm, bnorm;
  unsigned long long rn_bits, xn_bits, bn_bits, an_bits;   // max-reductions (non-negative doubles)
  int outer_active;   // refinement still running
  int cycle_active;   // inside a GMRES cycle, Arnoldi steps still wanted
  int k;              // Arnoldi steps done in the current cycle
  int iters, outer, status;
};

struct Brief {          // copied to the host after each control kernel
  int outer_active, cycle_active, iters, outer, status;
  int pad;
  double sr;
};

struct SolveParams {
  int n_rhs, m, max_iters;
  double inner_tol, theta, accept;
  int64_t n;
};

// ---------------------------------------------------------------------------
// GEMV: P[c][i + r*n] = sum_{j in chunk c} A(i, j) X(j, r); optional |A| row
// sums (fp32 estimate or exact fp64) into RS[c][i].
// 256 threads x 2 rows = 512 rows per CTA; the chunk's X is staged in shared
// memory once; each thread keeps 8 independent 16-byte column loads in
// flight (HBM bytes in flight per SM is what bounds this kernel).
// ---------------------------------------------------------------------------
constexpr int kGemvRows = 512;
constexpr int kGemvThreads = 256;
constexpr int kGemvChunkElems = 4096;   // columns x right-hand sides staged per CTA

template <int K, int kAbs, bool kF32 = false>   // kAbs: 0 none, 1 fp32 estimate, 2 fp64 exact
__global__ void __launch_bounds__(kGemvThreads) gemv_partial_kernel(int64_t n, const double* __restrict__ A,
                                                                    int64_t lda, const double* __restrict__ X,
                                                                    int64_t ldx, int64_t chunk,
                                                                    float* __restrict__ A32, int64_t ld32,
                                                                    double* __restrict__ P, void* __restrict__ RS) {
  __shared__ double xs[kGemvChunkElems];   // xs[r * chunk + jj]
  const int64_t i = (int64_t)blockIdx.x * kGemvRows + 2 * threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(j0 + chunk, n);
  const int cnt = (int)(j1 - j0);
  for (int t = threadIdx.x; t < cnt * K; t += kGemvThreads) {
    const int jj = t % cnt, r = t / cnt;
    xs[r * chunk + jj] = X[j0 + jj + r * ldx];
  }
  __syncthreads();
  if (i >= n) return;
  double acc0[K], acc1[K];
  float facc0[K], facc1[K];
#pragma unroll
  for (int r = 0; r < K; ++r) { acc0[r] = 0.0; acc1[r] = 0.0; facc0[r] = 0.0f; facc1[r] = 0.0f; }
  float s0 = 0.0f, s1 = 0.0f;
  double d0 = 0.0, d1 = 0.0;
  const bool two = i + 1 < n;
  const bool vec = two && ((((uintptr_t)(A + i)) & 15) == 0) && ((lda & 1) == 0);
  const double* col = A + i + j0 * lda;
  // optional copy of the visited entries, truncated to fp32, for the fp32 operator's later products
  float* col32 = A32 ? A32 + i + j0 * ld32 : nullptr;
  auto body = [&](double a0, double a1, int jj) {
    if (kF32) {
      // fp32 operator: A truncated to fp32, products accumulated in fp32
      const float f0 = trunc_f32(a0), f1 = trunc_f32(a1);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const float xv = (float)xs[r * chunk + jj];
        facc0[r] = __fmaf_rn(f0, xv, facc0[r]);
        facc1[r] = __fmaf_rn(f1, xv, facc1[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const double xv = xs[r * chunk + jj];
        acc0[r] = __fma_rn(a0, xv, acc0[r]);
        acc1[r] = __fma_rn(a1, xv, acc1[r]);
      }
    }
    if (kAbs == 1) { s0 += abs_f32_est(a0); s1 += abs_f32_est(a1); }
    if (kAbs == 2) { d0 += fabs(a0); d1 += fabs(a1); }
  };
  int jj = 0;
  if (vec) {
    for (; jj + 8 <= cnt; jj += 8) {
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcs(reinterpret_cast<const double2*>(col + (int64_t)u * lda));
      col += 8 * lda;
      if (col32) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          *reinterpret_cast<float2*>(col32 + (int64_t)u * ld32) = make_float2(trunc_f32(v[u].x), trunc_f32(v[u].y));
        col32 += 8 * ld32;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) body(v[u].x, v[u].y, jj + u);
    }
  }
  for (; jj < cnt; ++jj) {
    const double a0 = col[0], a1 = two ? col[1] : 0.0;
    col += lda;
    if (col32) {
      col32[0] = trunc_f32(a0);
      if (two) col32[1] = trunc_f32(a1);
      col32 += ld32;
    }
    body(a0, a1, jj);
  }
  double* Pc = P + (int64_t)blockIdx.y * n * K;
#pragma unroll
  for (int r = 0; r < K; ++r) {
    Pc[i + r * n] = kF32 ? (double)facc0[r] : acc0[r];
    if (two) Pc[i + 1 + r * n] = kF32 ? (double)facc1[r] : acc1[r];
  }
  if (kAbs == 1) {
    float* R = (float*)RS + (int64_t)blockIdx.y * n;
    R[i] = s0;
    if (two) R[i + 1] = s1;
  } else if (kAbs == 2) {
    double* R = (double*)RS + (int64_t)blockIdx.y * n;
    R[i] = d0;
    if (two) R[i + 1] = d1;
  }
}

// The fp32 operator's product from the fp32 copy of A: the same chunks, the
// same fp32 accumulation over each chunk's columns in order as the fp64-read
// variant (so the same partial sums), 4 rows per thread, 16-byte loads.
constexpr int kGemv32Rows = 4 * kGemvThreads;
template <int K>
__global__ void __launch_bounds__(kGemvThreads) gemv32_partial_kernel(int64_t n, const float* __restrict__ A32,
                                                                      int64_t ld32, const double* __restrict__ X,
                                                                      int64_t ldx, int64_t chunk,
                                                                      double* __restrict__ P) {
  __shared__ double xs[kGemvChunkElems];
  const int64_t i = (int64_t)blockIdx.x * kGemv32Rows + 4 * threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(j0 + chunk, n);
  const int cnt = (int)(j1 - j0);
  for (int t = threadIdx.x; t < cnt * K; t += kGemvThreads) {
    const int jj = t % cnt, r = t / cnt;
    xs[r * chunk + jj] = X[j0 + jj + r * ldx];
  }
  __syncthreads();
  if (i >= n) return;
  const int rows = (int)min((int64_t)4, n - i);
  float acc[4][K];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < K; ++r) acc[q][r] = 0.0f;
  const float* col = A32 + i + j0 * ld32;
  int jj = 0;
  if (rows == 4) {
    for (; jj + 8 <= cnt; jj += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcs(reinterpret_cast<const float4*>(col + (int64_t)u * ld32));
      col += 8 * ld32;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float a[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const float xv = (float)xs[r * chunk + jj + u];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q][r] = __fmaf_rn(a[q], xv, acc[q][r]);
        }
      }
    }
  }
  for (; jj < cnt; ++jj) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const float xv = (float)xs[r * chunk + jj];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < rows) acc[q][r] = __fmaf_rn(col[q], xv, acc[q][r]);
    }
    col += ld32;
  }
  double* Pc = P + (int64_t)blockIdx.y * n * K;
#pragma unroll
  for (int r = 0; r < K; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < rows) Pc[i + q + r * n] = (double)acc[q][r];
}

// out(i, r) = B(i, r) - sum_c P[c](i, r), or + sum_c P[c](i, r) when B is NULL
// (chunks in order); max-reduces
// |out|, |X| (when xn) and the row sums (when abs_mode) into the states.
__global__ void gemv_finish_kernel(int64_t n, int K, int nchunk, const double* __restrict__ P,
                                   const double* __restrict__ B, int64_t ldb, double* __restrict__ out,
                                   int64_t ldo, const double* __restrict__ X, int64_t ldx, int abs_mode,
                                   const void* __restrict__ RS, RhsState* st, int track_norms) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ unsigned long long smax[3 * kMaxK + 1];
  if (threadIdx.x < 3 * kMaxK + 1) smax[threadIdx.x] = 0;
  __syncthreads();
  if (i < n) {
    for (int r = 0; r < K; ++r) {
      double s = 0.0;
      for (int c = 0; c < nchunk; ++c) s += P[(int64_t)c * n * K + i + r * n];
      const double v = B ? B[i + r * ldb] - s : s;
      out[i + r * ldo] = v;
      if (track_norms) {
        atomicMax(&smax[r], dbits(fabs(v)));
        atomicMax(&smax[kMaxK + r], dbits(fabs(X[i + r * ldx])));
        if (B) atomicMax(&smax[2 * kMaxK + r], dbits(fabs(B[i + r * ldb])));
      }
    }
    if (abs_mode == 1) {
      float s = 0.0f;
      for (int c = 0; c < nchunk; ++c) s += ((const float*)RS)[(int64_t)c * n + i];
      atomicMax(&smax[3 * kMaxK], dbits((double)s));
    } else if (abs_mode == 2) {
      double s = 0.0;
      for (int c = 0; c < nchunk; ++c) s += ((const double*)RS)[(int64_t)c * n + i];
      atomicMax(&smax[3 * kMaxK], dbits(s));
    }
  }
  __syncthreads();
  if (threadIdx.x < K && track_norms) {
    const int r = threadIdx.x;
    atomicMax(&st[r].rn_bits, smax[r]);
    atomicMax(&st[r].xn_bits, smax[kMaxK + r]);
    if (B) atomicMax(&st[r].bn_bits, smax[2 * kMaxK + r]);
    if (abs_mode) atomicMax(&st[r].an_bits, smax[3 * kMaxK]);
  }
}

// ---------------------------------------------------------------------------
// Preconditioner: 128-row blocks, the diagonal blocks of L and U inverted once
// per solve (setup kernel below, in the arithmetic type T), so the diagonal
// solve is a parallel 128 x 128 product.  Each published block is a run of
// 64-bit words that carry their epoch: (fp32 value | epoch << 32) for T =
// float, two words (high half | epoch << 32), (low half | epoch << 32) per
// value for T = double; a reader's poll of the words delivers the data itself,
// with no separate flag.  Before it waits for z_c, every CTA issues the copies
// of what it will multiply z_c with: the owner of block c+1 its off-diagonal
// tile (and, for float, the inverted diagonal block; the fp64 inverse, 128 KB,
// is read from L2), and each CTA the tiles of its first two blocks that z_c
// updates.
// ---------------------------------------------------------------------------
constexpr int kTB32 = 128;

template <class T> __device__ inline T fma_t(T a, T b, T c);
template <> __device__ inline float fma_t<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ inline double fma_t<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
// a 16-bit factor entry as T (exact either way; the fp64 one built with integer operations)
template <class T> __device__ inline T u16_to(uint16_t h, int fmt);
template <> __device__ inline float u16_to<float>(uint16_t h, int fmt) { return u16_to_f32(h, fmt); }
template <> __device__ inline double u16_to<double>(uint16_t h, int fmt) { return u16_to_f64(h, fmt); }

// Inverse of diagonal block c (c < nb) of the unit-lower L (which == 0) or of
// U (which == 1) in T arithmetic, from the 16-bit factors: one thread per
// column, column-oriented substitution.  Output inv[(which * nb + c) * 128 *
// 128 + j * 128 + i] = inverse(i, j).
template <class T>
__global__ void __launch_bounds__(128) diag_inv_kernel(int64_t n, const uint16_t* __restrict__ LU, int64_t ld,
                                                       int fmt, T* __restrict__ inv) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  float* t = reinterpret_cast<float*>(dsm_raw);                         // t[j * 129 + i] = block(i, j)
  T* x = reinterpret_cast<T*>(dsm_raw + sizeof(float) * kTB32 * 130);   // x[j * 129 + i] = inverse(i, j)
  const int nb = (int)cdiv<int64_t>(n, kTB32);
  const int c = blockIdx.x, which = blockIdx.y, tid = threadIdx.x;
  const int64_t base = (int64_t)c * kTB32;
  for (int idx = tid; idx < kTB32 * kTB32; idx += 128) {
    const int i = idx % kTB32, j = idx / kTB32;
    const bool in = base + i < n && base + j < n;
    t[j * 129 + i] = in ? u16_to_f32(LU[base + i + (base + j) * ld], fmt) : (i == j ? 1.0f : 0.0f);
  }
  __syncthreads();
  const int j = tid;   // column of the inverse
  if (which == 0) {    // L X = I, unit lower: X(i, j) = -sum_{k=j}^{i-1} L(i, k) X(k, j)
    for (int i = 0; i < kTB32; ++i) x[j * 129 + i] = i == j ? (T)1 : (T)0;
    for (int i = j + 1; i < kTB32; ++i) {
      T s = (T)0;
      for (int k = j; k < i; ++k) s = fma_t<T>((T)t[k * 129 + i], x[j * 129 + k], s);
      x[j * 129 + i] = -s;
    }
  } else {             // U Y = I: Y(i, j) = (delta - sum_{k=i+1}^{j} U(i, k) Y(k, j)) / U(i, i)
    for (int i = 0; i < kTB32; ++i) x[j * 129 + i] = (T)0;
    x[j * 129 + j] = (T)1 / (T)t[j * 129 + j];
    for (int i = j - 1; i >= 0; --i) {
      T s = (T)0;
      for (int k = i + 1; k <= j; ++k) s = fma_t<T>((T)t[k * 129 + i], x[j * 129 + k], s);
      x[j * 129 + i] = -s / (T)t[i * 129 + i];
    }
  }
  __syncthreads();
  T* out = inv + ((int64_t)which * nb + c) * kTB32 * kTB32;
  for (int idx = tid; idx < kTB32 * kTB32; idx += 128) out[idx] = x[(idx / kTB32) * 129 + idx % kTB32];
}

template <class T>
size_t diag_inv_smem() { return sizeof(float) * kTB32 * 130 + sizeof(T) * kTB32 * 129; }

// Chain blocks of the fp64 preconditioner, once per solve: forward
// P_c = Linv_c L(c, c-1) (c >= 1), backward Q_c = Uinv_c U(c, c+1) (c <= nb-2),
// fp64 products of the fp64 inverses and the 16-bit factor tiles (terms t
// ascending).  out[((which * nb + c) * 128 + j) * 128 + i] = P(i, j).  With
// them the wavefront's dependent step is one product: z_{c+1} = y_{c+1} -
// P_{c+1} z_c, y_{c+1} = Linv_{c+1} (v_{c+1} - sum_{k<c} L(c+1,k) z_k) being
// known before z_c is.
__global__ void __launch_bounds__(256) chain_blocks_kernel(int64_t n, const uint16_t* __restrict__ LU, int64_t ld,
                                                           int fmt, const double* __restrict__ dinv,
                                                           double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char cb_raw[];
  float* tile = reinterpret_cast<float*>(cb_raw);   // tile[t * 128 + j] = T(t, j)
  const int nb = (int)cdiv<int64_t>(n, kTB32);
  const int c = blockIdx.x, which = blockIdx.y, tid = threadIdx.x;
  const int nbr = which == 0 ? c - 1 : c + 1;   // block column of the neighbour tile
  if (nbr < 0 || nbr >= nb) return;
  const int64_t r0 = (int64_t)c * kTB32, c0 = (int64_t)nbr * kTB32;
  for (int idx = tid; idx < kTB32 * kTB32; idx += 256) {
    const int t = idx % kTB32, j = idx / kTB32;   // coalesced over t (column major source)
    const bool in = r0 + t < n && c0 + j < n;
    tile[t * kTB32 + j] = in ? u16_to_f32(LU[r0 + t + (c0 + j) * ld], fmt) : 0.0f;
  }
  __syncthreads();
  const double* inv = dinv + ((int64_t)which * nb + c) * kTB32 * kTB32;
  const int i = tid % kTB32, jh = (tid / kTB32) * 64;
  double acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = 0.0;
  for (int t = 0; t < kTB32; ++t) {
    const double a = inv[(int64_t)t * kTB32 + i];
#pragma unroll
    for (int q = 0; q < 64; ++q) acc[q] = __fma_rn(a, (double)tile[t * kTB32 + jh + q], acc[q]);
  }
  double* o = out + ((int64_t)which * nb + c) * kTB32 * kTB32;
#pragma unroll
  for (int q = 0; q < 64; ++q) o[(int64_t)(jh + q) * kTB32 + i] = acc[q];
}

// words of one published value
template <class T> constexpr int kWords = sizeof(T) / 4;
// threads of the preconditioner's CTAs: each 128 x 128 product is split over
// kPrecondThreads / 128 column groups (512 threads for fp32 measured no faster
// than 256: the step is bound by the hand-off, not the products)
template <class T> constexpr int kPrecondThreads = 256;

__device__ inline unsigned long long tag_word(uint32_t bits, int epoch) {
  return (unsigned long long)bits | ((unsigned long long)(unsigned)epoch << 32);
}

__device__ inline void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class T, int K>
__global__ void __launch_bounds__(kPrecondThreads<T>) precond_kernel(int64_t n, const uint16_t* __restrict__ LU, int64_t ld,
                                                      int fmt, const T* __restrict__ dinv,
                                                      const double* __restrict__ pch,
                                                      const double* __restrict__ v, int64_t ldv,
                                                      double* __restrict__ z, int64_t ldz,
                                                      unsigned long long* __restrict__ pub, int epoch,
                                                      uint32_t* status, long long wait_polls,
                                                      unsigned long long wait_ns, const double* __restrict__ rs,
                                                      const double* __restrict__ cs) {
  constexpr bool kInvInSmem = sizeof(T) == 4;   // the fp32 inverse (64 KB) is staged; the fp64 one stays in L2
  constexpr int W = kWords<T>;
  constexpr int NT = kPrecondThreads<T>;   // threads: NT / 128 groups of 128 rows ...
  constexpr int HG = NT / kTB32;
  constexpr int HC = kTB32 / HG;           // ... each multiplying HC of a tile's columns
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nb = (int)cdiv<int64_t>(n, kTB32);
  const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x;
  const int nown = (nb - me + G - 1) / G;
  uint16_t* tl = reinterpret_cast<uint16_t*>(sm_raw);             // 3 x [128][128] 16-bit tiles, tl[j*128+i]
  float* ti = reinterpret_cast<float*>(tl + 3 * kTB32 * kTB32);   // [128][128] fp32 inverse (float only)
  T* acc = reinterpret_cast<T*>(kInvInSmem ? (unsigned char*)(ti + kTB32 * kTB32) : (unsigned char*)ti);
  T* zc = acc + (size_t)nown * kTB32 * K;                         // [128][K] block c
  T* zs = zc + kTB32 * K;                                         // [128][K] block being solved
  T* part = zs + kTB32 * K;                                       // [HG][128][K]
  T* ys = part + HG * kTB32 * K;                                  // [128][K] y of the next block (fp64)
  __shared__ int abort_flag;
  if (tid == 0) abort_flag = 0;
  unsigned long long* fpub = pub;
  unsigned long long* bpub = pub + (size_t)nb * kTB32 * K * W;
  for (int o = 0; o < nown; ++o)
    for (int t = tid; t < kTB32 * K; t += NT) {
      const int ii = t % kTB32, r = t / kTB32;
      const int64_t i = (int64_t)(me + o * G) * kTB32 + ii;
      // balanced factors (LU of diag(rs) A diag(cs)): M^{-1} v = diag(cs) U^{-1} L^{-1} diag(rs) v;
      // rs and cs are powers of two, so the scalings are exact
      acc[((size_t)o * kTB32 + ii) * K + r] = i < n ? (T)(rs ? v[i + r * ldv] * rs[i] : v[i + r * ldv]) : (T)0;
    }
  // abort_flag (and acc) must be written before any thread reads them: shared
  // memory starts with whatever the SM's previous block left there
  __syncthreads();

  // asynchronous copies: 16-bit tile (rb, cb) of LU into buffer slot, zero outside the matrix
  auto fetch_tile = [&](int slot, int rb, int cb) {
    uint16_t* dst = tl + (size_t)slot * kTB32 * kTB32;
    const int64_t i0 = (int64_t)rb * kTB32, j0 = (int64_t)cb * kTB32;
#pragma unroll
    for (int q = 0; q < 2048 / NT; ++q) {
      const int chunk = tid + q * NT;             // 2048 chunks of 8 rows
      const int jj = chunk >> 4, ii = (chunk & 15) * 8;
      const int64_t i = i0 + ii, j = j0 + jj;
      int bytes = 0;
      if (j < n && i < n) bytes = (int)min((int64_t)16, (n - i) * 2);
      const uint16_t* src = bytes ? LU + i + j * ld : LU;
      cp_async16((uint32_t)__cvta_generic_to_shared(dst + jj * kTB32 + ii), src, bytes);
    }
  };
  auto inv_block = [&](int which, int cb) { return dinv + ((int64_t)which * nb + cb) * kTB32 * kTB32; };
  // fp64: the HC inverse entries a thread multiplies, M(ii, h*HC .. h*HC+HC-1),
  // loaded into registers when the block becomes next; used by its solve
  T invr[kInvInSmem ? 1 : HC];
  auto fetch_inv = [&](int which, int cb) {
    const T* src = inv_block(which, cb);
    if constexpr (kInvInSmem) {
#pragma unroll
      for (int q = 0; q < 4096 / NT; ++q) {
        const int chunk = tid + q * NT;           // 4096 chunks of 4 floats
        cp_async16((uint32_t)__cvta_generic_to_shared(ti + chunk * 4), src + chunk * 4, 16);
      }
    } else {
      const int ii = tid % kTB32, h = tid / kTB32;
#pragma unroll
      for (int q = 0; q < HC; ++q) invr[q] = __ldcg(src + (h * HC + q) * kTB32 + ii);
    }
  };
  // fp64: the chain block P (which 0) / Q (which 1) of block cb into the same registers
  auto fetch_chain = [&](int which, int cb) {
    if constexpr (!kInvInSmem) {
      const double* src = pch + ((int64_t)which * nb + cb) * kTB32 * kTB32;
      const int ii = tid % kTB32, h = tid / kTB32;
#pragma unroll
      for (int q = 0; q < HC; ++q) invr[q] = __ldcg(src + (h * HC + q) * kTB32 + ii);
    }
  };
  // out[i][r] (-)= sum_j M(i, j) w[j][r]; M a 16-bit tile (T16) or the inverse (Tinv, fp32 in
  // shared memory or T in global memory)
  auto product = [&](const uint16_t* T16, const T* Tinv, const T* w, T* out, bool subtract) {
    const int ii = tid % kTB32, h = tid / kTB32;
    T s[K];
#pragma unroll
    for (int r = 0; r < K; ++r) s[r] = (T)0;
    if (T16) {
#pragma unroll 8
      for (int jj = h * HC; jj < h * HC + HC; ++jj) {
        const T tv = u16_to<T>(T16[jj * kTB32 + ii], fmt);
#pragma unroll
        for (int r = 0; r < K; ++r) s[r] = fma_t<T>(tv, w[jj * K + r], s[r]);
      }
    } else {
#pragma unroll 16
      for (int jj = h * HC; jj < h * HC + HC; ++jj) {
        const T tv = Tinv[jj * kTB32 + ii];
#pragma unroll
        for (int r = 0; r < K; ++r) s[r] = fma_t<T>(tv, w[jj * K + r], s[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) part[(h * kTB32 + ii) * K + r] = s[r];
    __syncthreads();
    for (int t = tid; t < kTB32 * K; t += NT) {
      T tot = part[t];
#pragma unroll
      for (int g = 1; g < HG; ++g) tot += part[g * kTB32 * K + t];
      out[t] = subtract ? out[t] - tot : tot;
    }
    __syncthreads();
  };
  // all copies issued by this CTA have landed (ready) / all but the latest group (ready_prev)
  auto ready = [&]() { cp_async_wait<0>(); __syncthreads(); };
  auto ready_prev = [&]() { cp_async_wait<1>(); __syncthreads(); };
  // wait for the tagged words of block c and unpack them into dst; a wait
  // that runs out (at most wait_polls polls and wait_ns of the global timer)
  // sets the timeout bit and the CTA's abort flag, and the other threads of
  // the CTA stop polling once they see the flag
  volatile int* abort_v = &abort_flag;
  auto receive = [&](const unsigned long long* src, int c, T* dst) {
    const unsigned long long* w = src + (size_t)c * kTB32 * K * W;
    const unsigned long long t0 = global_ns();
    for (int t = tid; t < kTB32 * K; t += NT) {
      uint32_t bits[W];
#pragma unroll
      for (int h = 0; h < W; ++h) {
        unsigned long long word = 0;
        for (long long it = 0;; ++it) {
          asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(word) : "l"(w + (size_t)t * W + h) : "memory");
          if ((int)(word >> 32) == epoch) break;
          if (it >= wait_polls || ((it & 63) == 63 && (global_ns() - t0 > wait_ns || *abort_v))) {
            atomicOr(status, kErrTimeout);
            *abort_v = 1;
            break;
          }
        }
        bits[h] = (uint32_t)(word & 0xffffffffu);
      }
      if constexpr (W == 1) dst[t] = __uint_as_float(bits[0]);
      else dst[t] = __hiloint2double((int)bits[0], (int)bits[1]);
    }
    __syncthreads();
  };
  // fp64: out = M w (or from - M w) with M in the invr registers (thread: row ii,
  // columns h*HC .. h*HC+HC-1), the column groups summed in order through `part`
  auto reg_product = [&](const T* w, T* out, const T* from) {
    const int ii = tid % kTB32, h = tid / kTB32;
    T sr[K];
#pragma unroll
    for (int r = 0; r < K; ++r) sr[r] = (T)0;
#pragma unroll
    for (int q = 0; q < HC; ++q)
#pragma unroll
      for (int r = 0; r < K; ++r) sr[r] = fma_t<T>(invr[kInvInSmem ? 0 : q], w[(h * HC + q) * K + r], sr[r]);
#pragma unroll
    for (int r = 0; r < K; ++r) part[(h * kTB32 + ii) * K + r] = sr[r];
    __syncthreads();
    for (int t = tid; t < kTB32 * K; t += NT) {
      T tot = part[t];
#pragma unroll
      for (int g = 1; g < HG; ++g) tot += part[g * kTB32 * K + t];
      out[t] = from ? from[t] - tot : tot;
    }
    __syncthreads();
  };
  // zs = Tinv acc_o (or, with chain, zs as computed by the caller), stored back
  // into acc_o and published (backward: also into z)
  auto solve = [&](int o, int c, bool backward, unsigned long long* dst, bool chained = false) {
    T* a = acc + (size_t)o * kTB32 * K;
    if (!chained) {
      if constexpr (kInvInSmem) product(nullptr, reinterpret_cast<const T*>(ti), a, zs, false);
      else reg_product(a, zs, nullptr);
    }
    unsigned long long* wd = dst + (size_t)c * kTB32 * K * W;
    for (int t = tid; t < kTB32 * K; t += NT) {
      a[t] = zs[t];
      if constexpr (W == 1) {
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(wd + t), "l"(tag_word(__float_as_uint(zs[t]), epoch))
                     : "memory");
      } else {
        const double d = zs[t];
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(wd + 2 * t),
                     "l"(tag_word((uint32_t)__double2hiint(d), epoch)) : "memory");
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(wd + 2 * t + 1),
                     "l"(tag_word((uint32_t)__double2loint(d), epoch)) : "memory");
      }
      if (backward) {
        const int ii = t / K, r = t % K;
        const int64_t i = (int64_t)c * kTB32 + ii;
        if (i < n) z[i + r * ldz] = cs ? (double)zs[t] * cs[i] : (double)zs[t];
      }
    }
    __syncthreads();
  };
  // The first two owned blocks that block c updates (past c in the sweep's
  // direction, other than `skip`): their tiles go to slots 1 and 2 before z_c
  // is awaited, since the tiles do not depend on it.  Returns how many.
  int pre_o[2];
  auto prefetch_updates = [&](int c, bool forward, int skip) {
    int k = 0;
    for (int o = 0; o < nown && k < 2; ++o) {
      const int rb = me + o * G;
      if (o == skip || (forward ? rb <= c : rb >= c)) continue;
      fetch_tile(1 + k, rb, c);
      pre_o[k++] = o;
    }
    return k;
  };
  // updates of the owned blocks by z_c: the `npre` prefetched ones from slots 1, 2, then
  // the rest with tiles double buffered in slots 1, 2
  auto stream_updates = [&](int c, bool forward, int skip, int npre) {
    for (int k = 0; k < npre; ++k)
      product(tl + (size_t)(1 + k) * kTB32 * kTB32, nullptr, zc, acc + (size_t)pre_o[k] * kTB32 * K, true);
    int pending = -1, slot = 1;
    for (int o = 0; o < nown; ++o) {
      const int rb = me + o * G;
      if (o == skip || (forward ? rb <= c : rb >= c)) continue;
      bool done = false;
      for (int k = 0; k < npre; ++k) done = done || pre_o[k] == o;
      if (done) continue;
      if (pending < 0) { fetch_tile(slot, rb, c); cp_async_commit(); pending = o; continue; }
      // compute the pending one while the next streams in
      fetch_tile(3 - slot, rb, c);
      cp_async_commit();
      ready_prev();
      product(tl + (size_t)slot * kTB32 * kTB32, nullptr, zc, acc + (size_t)pending * kTB32 * K, true);
      pending = o;
      slot = 3 - slot;
    }
    if (pending >= 0) {
      ready();
      product(tl + (size_t)slot * kTB32 * kTB32, nullptr, zc, acc + (size_t)pending * kTB32 * K, true);
    }
  };

  // fp32: once a CTA has solved block b, the tile and inverse that its next
  // block b' = b +- G will take on the chain are fetched at the end of that
  // iteration (into slot 0 and the inverse buffer, unused until then), so they
  // have landed when z_{b'-+1} arrives; `early` names b'
  int early = -1;
  auto fetch_early = [&](int nx, int which, bool forward) {
    if constexpr (kInvInSmem) {
      if (nx >= 0 && nx < nb) {
        fetch_tile(0, nx, forward ? nx - 1 : nx + 1);
        fetch_inv(which, nx);
        cp_async_commit();
        early = nx;
      }
    }
  };

  // ---------------- forward: L y = v ----------------
  if (me == 0) { fetch_inv(0, 0); cp_async_commit(); ready(); solve(0, 0, false, fpub); }
  for (int c = 0; c < nb && !abort_flag; ++c) {
    const bool next_mine = c + 1 < nb && (c + 1) % G == me;
    if (c % G != me) {
      const int last = me + (nown - 1) * G;
      if (nown == 0 || last <= c) continue;
    }
    const int skip = next_mine ? (c + 1) / G : -1;
    if (next_mine) {
      if constexpr (kInvInSmem) {
        if (early != c + 1) {
          fetch_tile(0, c + 1, c);
          fetch_inv(0, c + 1);
        }
      } else {
        // fp64: y = Linv_{c+1} acc_{c+1} before z_c is awaited (acc_{c+1} has every
        // term but z_c's), then the chain block P_{c+1} into the registers
        fetch_inv(0, c + 1);
        reg_product(acc + (size_t)skip * kTB32 * K, ys, nullptr);
        fetch_chain(0, c + 1);
      }
    }
    const int npre = prefetch_updates(c, true, skip);
    cp_async_commit();
    if (c % G == me) {
      for (int t = tid; t < kTB32 * K; t += NT) zc[t] = acc[(size_t)(c / G) * kTB32 * K + t];
    } else {
      receive(fpub, c, zc);
      if (abort_flag) break;
    }
    ready();
    if (next_mine) {
      if constexpr (kInvInSmem) {
        product(tl, nullptr, zc, acc + (size_t)skip * kTB32 * K, true);
        solve(skip, c + 1, false, fpub);
      } else {
        reg_product(zc, zs, ys);   // z_{c+1} = y_{c+1} - P_{c+1} z_c
        solve(skip, c + 1, false, fpub, true);
      }
    }
    stream_updates(c, true, skip, npre);
    if (next_mine) fetch_early(c + 1 + G, 0, true);
  }
  ready();
  early = -1;

  // ---------------- backward: U z = y ----------------
  if ((nb - 1) % G == me && !abort_flag) {
    fetch_inv(1, nb - 1);
    cp_async_commit();
    ready();
    solve((nb - 1) / G, nb - 1, true, bpub);
  }
  for (int c = nb - 1; c >= 0 && !abort_flag; --c) {
    const bool next_mine = c - 1 >= 0 && (c - 1) % G == me;
    if (c % G != me && (nown == 0 || me >= c)) continue;
    const int skip = next_mine ? (c - 1) / G : -1;
    if (next_mine) {
      if constexpr (kInvInSmem) {
        if (early != c - 1) {
          fetch_tile(0, c - 1, c);
          fetch_inv(1, c - 1);
        }
      } else {
        fetch_inv(1, c - 1);
        reg_product(acc + (size_t)skip * kTB32 * K, ys, nullptr);
        fetch_chain(1, c - 1);
      }
    }
    const int npre = prefetch_updates(c, false, skip);
    cp_async_commit();
    if (c % G == me) {
      for (int t = tid; t < kTB32 * K; t += NT) zc[t] = acc[(size_t)(c / G) * kTB32 * K + t];
    } else {
      receive(bpub, c, zc);
      if (abort_flag) break;
    }
    ready();
    if (next_mine) {
      if constexpr (kInvInSmem) {
        product(tl, nullptr, zc, acc + (size_t)skip * kTB32 * K, true);
        solve(skip, c - 1, true, bpub);
      } else {
        reg_product(zc, zs, ys);   // z_{c-1} = y_{c-1} - Q_{c-1} z_c
        solve(skip, c - 1, true, bpub, true);
      }
    }
    stream_updates(c, false, skip, npre);
    if (next_mine) fetch_early(c - 1 - G, 1, false);
  }
  ready();
}

// ---------------------------------------------------------------------------
// Vector kernels.  Deterministic reductions: per-thread strided partials,
// fixed-shape block tree, per-block partials summed in order by the last CTA.
// ---------------------------------------------------------------------------
__device__ inline double block_sum(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// For every rhs r that is in an active cycle: optionally w -= h_prev v_prev
// (h_prev = H(i-1, j)), then reduce either <w, v_i> (into H(i, j)) or <w, w>
// (into hn, as a square root) when i == j + 1.
__global__ void __launch_bounds__(256) mgs_kernel(int64_t n, int K, int m, int j, int i, double* W, int64_t ldw,
                                                  const double* V, int64_t ldv_col, int64_t ldv_rhs,
                                                  RhsState* st, double* partials, unsigned int* counter) {
  __shared__ double sh[256];
  __shared__ bool last;
  for (int r = 0; r < K; ++r) {
    const bool act = st[r].cycle_active != 0;
    double part = 0.0;
    if (act) {
      double* w = W + r * ldw;
      const double* vprev = i > 0 ? V + r * ldv_rhs + (int64_t)(i - 1) * ldv_col : nullptr;
      const double hprev = i > 0 ? st[r].H[(i - 1) + j * (m + 1)] : 0.0;
      const double* vi = i <= j ? V + r * ldv_rhs + (int64_t)i * ldv_col : nullptr;
      for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double wt = w[t];
        if (vprev) { wt = __fma_rn(-hprev, vprev[t], wt); w[t] = wt; }
        part = vi ? __fma_rn(wt, vi[t], part) : __fma_rn(wt, wt, part);
      }
    }
    const double bs = block_sum(part, sh);
    if (threadIdx.x == 0) partials[(int64_t)r * kRedBlocks + blockIdx.x] = bs;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < K) {
    const int r = threadIdx.x;
    if (st[r].cycle_active) {
      double s = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) s += partials[(int64_t)r * kRedBlocks + b];
      if (i <= j) st[r].H[i + j * (m + 1)] = s;
      else st[r].hn = sqrt(s);
    }
  }
  if (threadIdx.x == 0) *counter = 0;
}

// The tail of Arnoldi step j in one CTA, for systems small enough that one SM
// streams w and the basis faster than j + 4 launches would start: modified
// Gram-Schmidt (for i = 0 .. j, H(i, j) = <w, v_i> then w -= H(i, j) v_i, and
// hn = ||w||), the Givens update, and v_{j+1} = w / hn.  Every entry of w sees
// the same operations as in mgs_kernel; the dot products are summed by this
// CTA's fixed tree instead of across CTAs.
__device__ void givens_rhs(const SolveParams& sp, int j, RhsState* st, Brief* brief, int r);
constexpr int kFusedMgsThreads = 1024;
constexpr int64_t kFusedMgsMaxElems = 16384;   // n * K at most
__global__ void __launch_bounds__(kFusedMgsThreads) arnoldi_tail_kernel(SolveParams sp, int64_t n, int K, int m,
                                                                        int j, double* W, int64_t ldw, double* V,
                                                                        int64_t ldv_col, int64_t ldv_rhs,
                                                                        RhsState* st, Brief* brief) {
  __shared__ double sh[kFusedMgsThreads];
  for (int r = 0; r < K; ++r) {
    if (!st[r].cycle_active) continue;   // the same value for every thread
    double* w = W + r * ldw;
    double hprev = 0.0;
    for (int i = 0; i <= j + 1; ++i) {
      const double* vprev = i > 0 ? V + r * ldv_rhs + (int64_t)(i - 1) * ldv_col : nullptr;
      const double* vi = i <= j ? V + r * ldv_rhs + (int64_t)i * ldv_col : nullptr;
      double part = 0.0;
      for (int64_t t = threadIdx.x; t < n; t += kFusedMgsThreads) {
        double wt = w[t];
        if (vprev) { wt = __fma_rn(-hprev, vprev[t], wt); w[t] = wt; }
        part = vi ? __fma_rn(wt, vi[t], part) : __fma_rn(wt, wt, part);
      }
      const double s = block_sum(part, sh);   // ends with a barrier: w's updates are visible
      if (threadIdx.x == 0) {
        if (i <= j) st[r].H[i + j * (m + 1)] = s;
        else st[r].hn = sqrt(s);
      }
      hprev = s;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < K) givens_rhs(sp, j, st, brief, threadIdx.x);
  __syncthreads();
  for (int r = 0; r < K; ++r) {
    if (!st[r].cycle_active) continue;
    const double hn = st[r].hn;
    const double* w = W + r * ldw;
    double* v = V + r * ldv_rhs + (int64_t)(j + 1) * ldv_col;
    for (int64_t t = threadIdx.x; t < n; t += kFusedMgsThreads) v[t] = w[t] / hn;
  }
}

// ||z||_2 for cycle start (beta), into st[r].beta, for rhs with outer_active.
__global__ void __launch_bounds__(256) norm2_kernel(int64_t n, int K, const double* Z, int64_t ldz, RhsState* st,
                                                    double* partials, unsigned int* counter) {
  __shared__ double sh[256];
  __shared__ bool last;
  for (int r = 0; r < K; ++r) {
    double part = 0.0;
    if (st[r].outer_active) {
      const double* z = Z + r * ldz;
      for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        part = __fma_rn(z[t], z[t], part);
    }
    const double bs = block_sum(part, sh);
    if (threadIdx.x == 0) partials[(int64_t)r * kRedBlocks + blockIdx.x] = bs;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < K) {
    const int r = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += partials[(int64_t)r * kRedBlocks + b];
    st[r].beta = sqrt(s);
  }
  if (threadIdx.x == 0) *counter = 0;
}

// dst(:, r) = src(:, r) / d_r with d_r = st[r].beta (which == 0) or st[r].hn (which == 1),
// for rhs whose flag (cycle_active or outer_active) is set.
__global__ void scale_kernel(int64_t n, int K, const double* src, int64_t lds, double* dst, int64_t ldd,
                             const RhsState* st, int which) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  for (int r = 0; r < K; ++r) {
    const bool act = which == 0 ? st[r].outer_active != 0 : st[r].cycle_active != 0;
    if (!act) continue;
    const double d = which == 0 ? st[r].beta : st[r].hn;
    dst[t + r * ldd] = src[t + r * lds] / d;
  }
}

__global__ void init_kernel(int K, RhsState* st) {
  if ((int)threadIdx.x < K) st[threadIdx.x].outer_active = 1;
}

// Outer check: scaled residual from the max-reductions; decide per rhs.
__global__ void check_kernel(SolveParams sp, RhsState* st, Brief* brief, int first) {
  const int r = threadIdx.x;
  if (r >= sp.n_rhs) return;
  RhsState& s = st[r];
  if (first) {
    s.anorm = bits_d(s.an_bits);
    s.bnorm = bits_d(s.bn_bits);
  }
  if (s.outer_active) {
    const double rn = bits_d(s.rn_bits), xn = bits_d(s.xn_bits);
    const double sr = rn / ((s.anorm * xn + s.bnorm) * ((double)sp.n * 0x1p-53));
    s.sr = sr;
    if (!isfinite(sr)) { s.status = HPMXP_EBREAKDOWN; s.outer_active = 0; }
    else if (sr < sp.accept) { s.status = HPMXP_OK; s.outer_active = 0; }
    else if (s.iters >= sp.max_iters) { s.status = HPMXP_ENOCONV; s.outer_active = 0; }
  }
  s.rn_bits = 0; s.xn_bits = 0;
  s.cycle_active = 0;
  brief[r].outer_active = s.outer_active; brief[r].cycle_active = 0;
  brief[r].iters = s.iters; brief[r].outer = s.outer; brief[r].status = s.status; brief[r].sr = s.sr;
}

// Cycle start (after beta = ||M^{-1} r||): g = beta e1, tolerance.
__global__ void cycle_start_kernel(SolveParams sp, RhsState* st, Brief* brief) {
  const int r = threadIdx.x;
  if (r >= sp.n_rhs) return;
  RhsState& s = st[r];
  s.cycle_active = 0;
  if (s.outer_active) {
    if (!(isfinite(s.beta) && s.beta > 0.0)) {
      s.status = HPMXP_EBREAKDOWN; s.outer_active = 0;
    } else {
      s.outer += 1;
      s.k = 0;
      for (int t = 0; t <= sp.m; ++t) s.g[t] = 0.0;
      s.g[0] = s.beta;
      const double adapt = sp.theta > 0.0 ? sp.theta * sp.accept / s.sr : 0.0;
      s.tol = s.beta * fmax(sp.inner_tol, adapt);
      s.cycle_active = s.iters < sp.max_iters ? 1 : 0;
    }
  }
  brief[r].outer_active = s.outer_active; brief[r].cycle_active = s.cycle_active;
  brief[r].status = s.status; brief[r].iters = s.iters; brief[r].outer = s.outer; brief[r].sr = s.sr;
}

// Givens update of column j (after MGS filled H(0..j, j) and hn).
// Givens update of right-hand side r after Arnoldi step j (thread r)
__device__ void givens_rhs(const SolveParams& sp, int j, RhsState* st, Brief* brief, int r) {
  RhsState& s = st[r];
  if (s.cycle_active) {
    const int ld = sp.m + 1;
    double* h = s.H + j * ld;
    const double hn = s.hn;
    h[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a0 = h[i], a1 = h[i + 1];
      h[i] = s.cs[i] * a0 + s.sn[i] * a1;
      h[i + 1] = -s.sn[i] * a0 + s.cs[i] * a1;
    }
    const double hj = h[j];
    const double den = hypot(hj, hn);
    if (!(isfinite(den) && den != 0.0)) {
      s.status = HPMXP_EBREAKDOWN; s.outer_active = 0; s.cycle_active = 0;
    } else {
      s.cs[j] = hj / den;
      s.sn[j] = hn / den;
      h[j] = den;
      h[j + 1] = 0.0;
      s.g[j + 1] = -s.sn[j] * s.g[j];
      s.g[j] = s.cs[j] * s.g[j];
      s.iters += 1;
      s.k = j + 1;
      if (hn == 0.0 || fabs(s.g[j + 1]) <= s.tol || s.k >= sp.m || s.iters >= sp.max_iters) s.cycle_active = 0;
      if (!isfinite(s.g[j + 1])) { s.status = HPMXP_EBREAKDOWN; s.outer_active = 0; s.cycle_active = 0; }
    }
  }
  brief[r].cycle_active = s.cycle_active; brief[r].outer_active = s.outer_active;
  brief[r].iters = s.iters; brief[r].status = s.status;
}
__global__ void givens_kernel(SolveParams sp, int j, RhsState* st, Brief* brief) {
  if ((int)threadIdx.x < sp.n_rhs) givens_rhs(sp, j, st, brief, threadIdx.x);
}

// y = H(0:k, 0:k)^{-1} g(0:k) by back substitution.
__global__ void cycle_finish_kernel(SolveParams sp, RhsState* st) {
  const int r = threadIdx.x;
  if (r >= sp.n_rhs) return;
  RhsState& s = st[r];
  if (!s.outer_active) { s.k = 0; return; }
  const int ld = sp.m + 1;
  for (int i = s.k - 1; i >= 0; --i) {
    double acc = s.g[i];
    for (int t = i + 1; t < s.k; ++t) acc = __fma_rn(-s.H[i + t * ld], s.y[t], acc);
    s.y[i] = acc / s.H[i + i * ld];
  }
}

// x(:, r) += V_r(:, 0:k) y_r
__global__ void update_kernel(int64_t n, int K, double* X, int64_t ldx, const double* V, int64_t ldv_col,
                              int64_t ldv_rhs, const RhsState* st) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  for (int r = 0; r < K; ++r) {
    const int k = st[r].outer_active ? st[r].k : 0;
    double xv = X[t + r * ldx];
    for (int i = 0; i < k; ++i) xv = __fma_rn(V[r * ldv_rhs + (int64_t)i * ldv_col + t], st[r].y[i], xv);
    X[t + r * ldx] = xv;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct SolveWs {
  uint32_t* status;
  RhsState* st;
  Brief* brief;
  unsigned int* counter;
  double* partials;  // kMaxK * kRedBlocks
  double* r;         // n x K
  double* w;         // n x K
  double* tmp;       // n x K
  double* V;         // K x (m+1) x n
  double* P;         // nchunk x n x K
  void* RS;          // nchunk x n (fp64 size)
  void* pub;         // 2 sweeps x round_up(n, 128) x K values x (1 or 2) 8-byte tagged words
  void* dinv;        // 2 x nb128 x 128 x 128 inverted diagonal blocks (float or double)
  double* pch;       // 2 x nb128 x 128 x 128 chain blocks of the fp64 preconditioner
  float* a32;        // optional fp32 copy of A (ld32), written by the first residual, NULL if none
  int64_t ld32;
  size_t bytes;
};

// Column chunks of the GEMV: each chunk's X (chunk x K doubles) fits the
// CTA's staging buffer; there are enough CTAs to keep every SM loaded (about
// 8 per SM), but no CTA reads fewer than 32 columns (128 KB of A), so a small
// system does not spread a short product over every SM.
int gemv_chunks(int64_t n, int K = kMaxK) {
  const int64_t rb = cdiv<int64_t>(n, kGemvRows);
  const int64_t spread = std::min<int64_t>(cdiv<int64_t>(8 * 152, rb), cdiv<int64_t>(n, 32));
  int64_t c = std::max<int64_t>(cdiv<int64_t>(n * K, kGemvChunkElems), spread);
  c = std::max<int64_t>(1, std::min<int64_t>(c, cdiv<int64_t>(n, 8)));
  return (int)c;
}

// tagged words of both sweeps, sized for fp64 values (two words each)
size_t pub_bytes(int64_t n, int64_t K) { return sizeof(unsigned long long) * 2 * 2 * round_up<int64_t>(n, kTB32) * K; }

SolveWs carve_solve(void* base, int64_t n, int64_t K, int m) {
  SolveWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? (char*)base + off : nullptr;
    off += round_up<size_t>(bytes, 256);
    return p;
  };
  const int nchunk = gemv_chunks(n);
  w.status = (uint32_t*)take(256);
  w.st = (RhsState*)take(sizeof(RhsState) * kMaxK);
  w.brief = (Brief*)take(sizeof(Brief) * kMaxK);
  w.counter = (unsigned int*)take(256);
  w.partials = (double*)take(sizeof(double) * kMaxK * kRedBlocks);
  w.r = (double*)take(sizeof(double) * n * K);
  w.w = (double*)take(sizeof(double) * n * K);
  w.tmp = (double*)take(sizeof(double) * n * K);
  w.V = (double*)take(sizeof(double) * n * (m + 1) * K);
  w.P = (double*)take(sizeof(double) * nchunk * n * K);
  w.RS = take(sizeof(double) * nchunk * n);
  w.pub = take(pub_bytes(n, K));
  w.dinv = take(sizeof(double) * 2 * round_up<int64_t>(n, kTB32) * kTB32);
  w.pch = (double*)take(sizeof(double) * 2 * round_up<int64_t>(n, kTB32) * kTB32);
  w.bytes = off;
  return w;
}

// abs_mode: 0 plain, 1 with the fp32 |A| estimate (the first residual; also
// fills w.a32 when there is one), 2 exact |A| row sums, 3 the fp32 operator's
// product (from w.a32 when there is one)
template <int K>
cudaError_t gemv_k(int64_t n, const double* A, int64_t lda, const double* X, int64_t ldx, int abs_mode,
                   const SolveWs& w, int nchunk, cudaStream_t st) {
  const int64_t chunk = cdiv<int64_t>(n, nchunk);
  if (chunk * K > kGemvChunkElems) return cudaErrorInvalidValue;
  dim3 grid((unsigned)cdiv<int64_t>(n, kGemvRows), (unsigned)nchunk);
  const int T = kGemvThreads;
  double* P = w.P;
  void* RS = w.RS;
  if (abs_mode == 3 && w.a32) {
    dim3 g32((unsigned)cdiv<int64_t>(n, kGemv32Rows), (unsigned)nchunk);
    gemv32_partial_kernel<K><<<g32, T, 0, st>>>(n, w.a32, w.ld32, X, ldx, chunk, P);
  } else if (abs_mode == 3) {
    gemv_partial_kernel<K, 0, true><<<grid, T, 0, st>>>(n, A, lda, X, ldx, chunk, nullptr, 0, P, RS);
  } else if (abs_mode == 0) {
    gemv_partial_kernel<K, 0><<<grid, T, 0, st>>>(n, A, lda, X, ldx, chunk, nullptr, 0, P, RS);
  } else if (abs_mode == 1) {
    gemv_partial_kernel<K, 1><<<grid, T, 0, st>>>(n, A, lda, X, ldx, chunk, w.a32, w.ld32, P, RS);
  } else {
    gemv_partial_kernel<K, 2><<<grid, T, 0, st>>>(n, A, lda, X, ldx, chunk, nullptr, 0, P, RS);
  }
  return cudaGetLastError();
}

// out = b - A X (b may be NULL: out = -A X), with optional norm tracking.
cudaError_t residual(int64_t n, int K, const double* A, int64_t lda, const double* X, int64_t ldx,
                     const double* B, int64_t ldb, double* out, int64_t ldo, int abs_mode, int track,
                     const SolveWs& w, cudaStream_t st) {
  const int nchunk = gemv_chunks(n, K);
  cudaError_t e;
  void* tok = prof_begin(st);
  switch (K) {
    case 1: e = gemv_k<1>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 2: e = gemv_k<2>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 3: e = gemv_k<3>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 4: e = gemv_k<4>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 5: e = gemv_k<5>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 6: e = gemv_k<6>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    case 7: e = gemv_k<7>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
    default: e = gemv_k<8>(n, A, lda, X, ldx, abs_mode, w, nchunk, st); break;
  }
  if (e != cudaSuccess) return e;
  gemv_finish_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, K, nchunk, w.P, B, ldb, out, ldo, X, ldx,
                                                                      abs_mode == 3 ? 0 : abs_mode, w.RS, w.st,
                                                                      track);
  prof_end(tok, abs_mode == 3 ? kProfGemv32 : kProfGemv, 8.0 * (double)n * (double)n, st);
  count_launches(2);
  return cudaGetLastError();
}

// Dynamic shared memory cap of the preconditioner kernels (the attribute is
// set to this one value, never to a per-call size).
constexpr size_t kMaxPrecondSmem = 200 * 1024;

template <class T>
size_t precond_smem(int64_t n, int K, int G) {
  const int nb = (int)cdiv<int64_t>(n, kTB32);
  const int nown = cdiv(nb, G);
  const size_t inv = sizeof(T) == 4 ? sizeof(float) * kTB32 * kTB32 : 0;
  const size_t groups = kPrecondThreads<T> / kTB32;
  return sizeof(uint16_t) * 3 * kTB32 * kTB32 + inv +
         sizeof(T) * ((size_t)nown * kTB32 * K + 2 * kTB32 * K + groups * kTB32 * K + kTB32 * K) + 64;
}

template <class T, int K>
cudaError_t precond_launch_k(int64_t n, const uint16_t* LU, int64_t ld, int fmt, const T* dinv, const double* pch,
                             const double* v,
                             int64_t ldv, double* z, int64_t ldz, unsigned long long* pub, int epoch,
                             uint32_t* status, int G, size_t smem, cudaStream_t st, const double* rs,
                             const double* cs) {
  auto kern = precond_kernel<T, K>;
  // one value for every call: concurrent solves on other threads set the same cap
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxPrecondSmem);
  if (e != cudaSuccess) return e;
  const WaitBudget wb = wait_budget();
  long long polls = wb.polls;
  unsigned long long ns = wb.ns;
  void* args[] = {&n,  (void*)&LU, &ld,     &fmt,   (void*)&dinv, (void*)&pch, (void*)&v,  &ldv, &z,
                  &ldz, &pub,      &epoch, &status, &polls,      &ns,         (void*)&rs, (void*)&cs};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(kPrecondThreads<T>), args, smem, st);
}

template <class T>
cudaError_t precond_launch(int K, int64_t n, const uint16_t* LU, int64_t ld, int fmt, const T* dinv,
                           const double* pch, const double* v, int64_t ldv, double* z, int64_t ldz, unsigned long long* pub,
                           int epoch, uint32_t* status, int G, size_t smem, cudaStream_t st, const double* rs,
                           const double* cs) {
#define HPMXP_PRECOND_K(KK) \
  precond_launch_k<T, KK>(n, LU, ld, fmt, dinv, pch, v, ldv, z, ldz, pub, epoch, status, G, smem, st, rs, cs)
  switch (K) {
    case 1: return HPMXP_PRECOND_K(1);
    case 2: return HPMXP_PRECOND_K(2);
    case 3: return HPMXP_PRECOND_K(3);
    case 4: return HPMXP_PRECOND_K(4);
    case 5: return HPMXP_PRECOND_K(5);
    case 6: return HPMXP_PRECOND_K(6);
    case 7: return HPMXP_PRECOND_K(7);
    default: return HPMXP_PRECOND_K(8);
  }
#undef HPMXP_PRECOND_K
}

template <class T>
cudaError_t diag_inv_launch(int64_t n, const uint16_t* LU, int64_t ld, int fmt, void* dinv, cudaStream_t st) {
  const size_t ism = diag_inv_smem<T>();
  cudaError_t e = cudaFuncSetAttribute(diag_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
  if (e != cudaSuccess) return e;
  diag_inv_kernel<T><<<dim3((unsigned)cdiv<int64_t>(n, kTB32), 2), 128, ism, st>>>(n, LU, ld, fmt, (T*)dinv);
  count_launches(1);
  return cudaGetLastError();
}

struct Solver {
  int64_t n;
  int K, m;
  const double* A; int64_t lda;
  const uint16_t* LU; int64_t ldlu; int fmt;
  const double* rs = nullptr;   // balancing of the factors (NULL: none)
  const double* cs = nullptr;
  const double* B; int64_t ldb;
  double* X; int64_t ldx;
  hpmxp_ir_params prm;
  SolveWs w;
  cudaStream_t st;
  int epoch = 0;
  int G = 0;
  size_t psmem = 0;
  Brief brief[kMaxK];

  int64_t ldv_rhs() const { return n * (m + 1); }

  cudaError_t precond(const double* v, int64_t ldv, double* z, int64_t ldz) {
    ++epoch;
    void* tok = prof_begin(st);
    unsigned long long* pub = (unsigned long long*)w.pub;
    cudaError_t e = prm.precond_fp32
                        ? precond_launch<float>(K, n, LU, ldlu, fmt, (const float*)w.dinv, nullptr, v, ldv, z, ldz,
                                                pub, epoch, w.status, G, psmem, st, rs, cs)
                        : precond_launch<double>(K, n, LU, ldlu, fmt, (const double*)w.dinv, w.pch, v, ldv, z, ldz,
                                                 pub, epoch, w.status, G, psmem, st, rs, cs);
    prof_end(tok, kProfPrecond, 2.0 * (double)n * (double)n, st);
    count_launches(1);
    return e;
  }

  cudaError_t read_brief() {
    return read_to_host(brief, w.brief, sizeof(Brief) * K, st);
  }
  // Arnoldi step j after w = M^{-1} A v_j: modified Gram-Schmidt, the Givens
  // update (into the brief) and v_{j+1}; one CTA for small systems, else one
  // launch per projection, then the rotation and the scaling
  void arnoldi_tail(int j) {
    const SolveParams sp{K, m, prm.max_iters, prm.inner_tol, prm.theta, prm.accept, n};
    if (n * K <= kFusedMgsMaxElems) {
      arnoldi_tail_kernel<<<1, kFusedMgsThreads, 0, st>>>(sp, n, K, m, j, w.w, n, w.V, n, ldv_rhs(), w.st, w.brief);
      count_launches(1);
      return;
    }
    for (int i = 0; i <= j + 1; ++i)
      mgs_kernel<<<kRedBlocks, 256, 0, st>>>(n, K, m, j, i, w.w, n, w.V, n, ldv_rhs(), w.st, w.partials, w.counter);
    givens_kernel<<<1, 32, 0, st>>>(sp, j, w.st, w.brief);
    scale_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, K, w.w, n, w.V + (int64_t)(j + 1) * n, ldv_rhs(),
                                                                   w.st, 1);
    count_launches(j + 4);
  }
  bool any(int Brief::*f) const {
    for (int r = 0; r < K; ++r)
      if (brief[r].*f) return true;
    return false;
  }

  cudaError_t setup() {
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // one CTA per SM at most: a cooperative launch keeps all of them resident
    const int nb = (int)cdiv<int64_t>(n, kTB32);
    // one CTA per owned share of block rows; an SM budget takes fewer CTAs as
    // long as their shares still fit in shared memory
    const int budget = sm_budget();
    const int gmax = std::max(1, std::min(nb, sms));
    G = std::max(1, std::min(gmax, budget > 0 ? budget : gmax));
    auto smem_for = [&](int g) {
      return prm.precond_fp32 ? precond_smem<float>(n, K, g) : precond_smem<double>(n, K, g);
    };
    while (G < gmax && smem_for(G) > kMaxPrecondSmem) ++G;
    psmem = smem_for(G);
    if (psmem > kMaxPrecondSmem) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(w.pub, 0, pub_bytes(n, K), st)) != cudaSuccess) return e;
    e = prm.precond_fp32 ? diag_inv_launch<float>(n, LU, ldlu, fmt, w.dinv, st)
                         : diag_inv_launch<double>(n, LU, ldlu, fmt, w.dinv, st);
    if (e != cudaSuccess) return e;
    if (!prm.precond_fp32) {
      constexpr size_t kChainSmem = sizeof(float) * kTB32 * kTB32;
      e = cudaFuncSetAttribute(chain_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmem);
      if (e != cudaSuccess) return e;
      chain_blocks_kernel<<<dim3((unsigned)cdiv<int64_t>(n, kTB32), 2), 256, kChainSmem, st>>>(
          n, LU, ldlu, fmt, (const double*)w.dinv, w.pch);
      count_launches(1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(w.st, 0, sizeof(RhsState) * kMaxK, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.counter, 0, 256, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.status, 0, 4, st)) != cudaSuccess) return e;
    init_kernel<<<1, 32, 0, st>>>(K, w.st);
    count_launches(1);
    return cudaGetLastError();
  }

  cudaError_t run() {
    cudaError_t e = setup();
    if (e != cudaSuccess) return e;
    SolveParams sp{K, m, prm.max_iters, prm.inner_tol, prm.theta, prm.accept, n};

    // x0 = U^{-1} L^{-1} b
    if ((e = precond(B, ldb, X, ldx)) != cudaSuccess) return e;
    bool first = true;
    for (;;) {
      // r = b - A x, norms; decide
      if ((e = residual(n, K, A, lda, X, ldx, B, ldb, w.r, n, first ? 1 : 0, 1, w, st)) != cudaSuccess) return e;
      check_kernel<<<1, 32, 0, st>>>(sp, w.st, w.brief, first ? 1 : 0);
      count_launches(1);
      first = false;
      if ((e = read_brief()) != cudaSuccess) return e;
      if (!any(&Brief::outer_active)) break;
      // cycle start: z = M^{-1} r, beta, v0 = z / beta
      if ((e = precond(w.r, n, w.tmp, n)) != cudaSuccess) return e;
      norm2_kernel<<<kRedBlocks, 256, 0, st>>>(n, K, w.tmp, n, w.st, w.partials, w.counter);
      cycle_start_kernel<<<1, 32, 0, st>>>(sp, w.st, w.brief);
      scale_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, K, w.tmp, n, w.V, ldv_rhs(), w.st, 0);
      count_launches(3);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = read_brief()) != cudaSuccess) return e;
      if (!any(&Brief::outer_active)) break;
      for (int j = 0; j < m && any(&Brief::cycle_active); ++j) {
        // w = M^{-1} (A v_j); the product in fp32 or fp64 as matvec_fp32 says
        if ((e = residual(n, K, A, lda, w.V + (int64_t)j * n, ldv_rhs(), nullptr, 0, w.tmp, n,
                          prm.matvec_fp32 ? 3 : 0, 0, w, st)) != cudaSuccess)
          return e;
        if ((e = precond(w.tmp, n, w.w, n)) != cudaSuccess) return e;
        arnoldi_tail(j);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = read_brief()) != cudaSuccess) return e;
      }
      cycle_finish_kernel<<<1, 32, 0, st>>>(sp, w.st);
      update_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, K, X, ldx, w.V, n, ldv_rhs(), w.st);
      count_launches(2);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

}  // namespace

// Test support: every SM's shared memory filled with `pattern`, so that a
// kernel launched next finds nonzero leftovers there instead of the zeros a
// quiet GPU tends to leave.
__global__ void fill_smem_kernel(uint32_t pattern, uint32_t words) {
  extern __shared__ uint32_t sw[];
  for (uint32_t t = threadIdx.x; t < words; t += blockDim.x) sw[t] = pattern;
  __syncthreads();
  if (sw[(threadIdx.x * 7u) % words] != pattern) asm volatile("" ::: "memory");
}

// Test support: the fp64 decoding of 16-bit factor entries, one per thread.
__global__ void decode16_kernel(const uint16_t* __restrict__ codes, double* __restrict__ out, int64_t count,
                                int fmt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = u16_to_f64(codes[i], fmt);
}

cudaError_t decode16(const uint16_t* codes, double* out, int64_t count, int fmt, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  decode16_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(codes, out, count, fmt);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t fill_smem(uint32_t pattern, cudaStream_t st) {
  int dev = 0, sms = 0, maxb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxb, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fill_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
  if (e != cudaSuccess) return e;
  fill_smem_kernel<<<2 * sms, 1024, (size_t)maxb, st>>>(pattern, (uint32_t)maxb / 4);
  count_launches(1);
  return cudaGetLastError();
}

size_t solve_ws_bytes(int64_t n, int64_t nrhs, int restart) { return carve_solve(nullptr, n, nrhs, restart).bytes; }
int64_t a32_ld(int64_t n) { return round_up<int64_t>(n, 4); }
size_t solve_a32_bytes(int64_t n) { return round_up<size_t>(sizeof(float) * (size_t)a32_ld(n) * (size_t)n, 256); }
size_t residual_ws_bytes(int64_t n, int64_t nrhs) { return carve_solve(nullptr, n, nrhs, 1).bytes; }

hpmxp_status solve_ir(int64_t n, const double* A, int64_t lda, const void* LU, int64_t ldlu, int prec,
                      const double* b, int64_t ldb, double* x, int64_t ldx, int64_t nrhs,
                      const hpmxp_ir_params& prm, hpmxp_ir_info* info, void* ws, size_t ws_bytes,
                      cudaStream_t st, const double* rs, const double* cs) {
  Solver s;
  s.n = n; s.K = (int)nrhs; s.m = prm.restart;
  s.A = A; s.lda = lda;
  s.LU = (const uint16_t*)LU; s.ldlu = ldlu; s.fmt = fmt_of(prec);
  s.rs = rs; s.cs = cs;
  s.B = b; s.ldb = ldb; s.X = x; s.ldx = ldx;
  s.prm = prm;
  s.w = carve_solve(ws, n, nrhs, prm.restart);
  // room for the fp32 copy of A after the workspace proper: the fp32 Arnoldi
  // products then read 4 instead of 8 bytes per entry
  if (prm.matvec_fp32 && ws_bytes >= s.w.bytes + solve_a32_bytes(n)) {
    s.w.a32 = (float*)((char*)ws + s.w.bytes);
    s.w.ld32 = a32_ld(n);
  }
  s.st = st;
  cudaError_t e = s.run();
  if (e != cudaSuccess) return status_from_cuda(e);
  uint32_t word = 0;
  e = read_to_host(&word, s.w.status, 4, st);
  if (e == cudaSuccess) e = s.read_brief();
  if (e != cudaSuccess) return status_from_cuda(e);
  if (word) return status_from_word(word);
  int worst = HPMXP_OK;
  for (int r = 0; r < s.K; ++r) {
    if (info) {
      info[r].iters = s.brief[r].iters;
      info[r].outer = s.brief[r].outer;
      info[r].scaled_resid = s.brief[r].sr;
      info[r].status = s.brief[r].status;
      info[r].reserved = 0;
    }
    if (s.brief[r].status != HPMXP_OK && worst == HPMXP_OK) worst = s.brief[r].status;
  }
  return (hpmxp_status)worst;
}

// ---------------------------------------------------------------------------
// Batched GMRES-IR: every system's refinement as a state machine (the phases
// of Solver::run), advanced in lockstep.  Each round issues every active
// system's next phase on its stream (systems spread over a pool of streams,
// so small systems' kernels run side by side) with an asynchronous copy of its
// brief, then waits once per system and decides every next phase on the host:
// one host decision point per phase for the whole batch.
// ---------------------------------------------------------------------------
namespace {
constexpr int kPoolStreams = 8;

struct StreamPool {
  std::mutex mu;
  bool ok = false;
  cudaStream_t st[kPoolStreams] = {};
  cudaEvent_t ev[kPoolStreams] = {};
};

StreamPool& stream_pool(int dev) {
  static StreamPool tab[64];
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  StreamPool& p = tab[dev & 63];
  if (!p.ok) {
    bool good = true;
    for (int i = 0; i < kPoolStreams && good; ++i)
      good = cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.ev[i], cudaEventDisableTiming) == cudaSuccess;
    p.ok = good;
  }
  return p;
}

enum Phase { kResid, kCycle, kArnoldi, kDone };

struct BatchItem {
  Solver s;
  Phase ph = kResid;
  int j = 0;            // next Arnoldi step
  bool first = true;    // the first residual also takes ||A||
  bool finish = false;  // cycle_finish + update to issue before the next residual
  cudaEvent_t ev = nullptr;
  Brief* host = nullptr;   // pinned copy of the brief
};

size_t batch_solve_bytes(const hpmxp_problem* probs, int count, int restart) {
  size_t b = 0;
  for (int q = 0; q < count; ++q) b += round_up<size_t>(solve_ws_bytes(probs[q].n, probs[q].nrhs, restart), 256);
  return b;
}
}  // namespace

size_t solve_batched_ws_bytes(const hpmxp_problem* probs, int count, int restart) {
  return batch_solve_bytes(probs, count, restart);
}

hpmxp_status solve_ir_batched(const hpmxp_problem* probs, int count, int prec, const hpmxp_ir_params& prm,
                              hpmxp_ir_info* info, void* ws, cudaStream_t caller) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_from_cuda(e);
  StreamPool& pool = stream_pool(dev);
  if (!pool.ok) return HPMXP_ECUDA;
  std::lock_guard<std::mutex> lk(pool.mu);   // one batched solve drives a device's pool at a time
  // pinned briefs and per-system events, kept by the calling thread
  struct HostSide {
    Brief* pinned = nullptr;
    size_t cap = 0;
    std::vector<cudaEvent_t> ev;
    ~HostSide() {
      if (pinned) cudaFreeHost(pinned);
      for (cudaEvent_t x : ev) cudaEventDestroy(x);
    }
  };
  thread_local HostSide hs;
  const size_t need = (size_t)count * kMaxK;
  if (hs.cap < need) {
    if (hs.pinned) cudaFreeHost(hs.pinned);
    hs.pinned = nullptr;
    hs.cap = 0;
    if ((e = cudaMallocHost(&hs.pinned, sizeof(Brief) * need)) != cudaSuccess) return status_from_cuda(e);
    hs.cap = need;
  }
  while ((int)hs.ev.size() < count) {
    cudaEvent_t x;
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) return status_from_cuda(e);
    hs.ev.push_back(x);
  }
  std::vector<BatchItem> it((size_t)count);
  char* base = (char*)ws;
  for (int q = 0; q < count; ++q) {
    Solver& s = it[q].s;
    s.n = probs[q].n; s.K = (int)probs[q].nrhs; s.m = prm.restart;
    s.A = probs[q].A; s.lda = probs[q].lda;
    s.LU = (const uint16_t*)probs[q].LU; s.ldlu = probs[q].ldlu; s.fmt = fmt_of(prec);
    s.B = probs[q].b; s.ldb = probs[q].ldb; s.X = probs[q].x; s.ldx = probs[q].ldx;
    s.prm = prm;
    s.w = carve_solve(base, s.n, s.K, prm.restart);
    base += round_up<size_t>(s.w.bytes, 256);
    s.st = pool.st[q % kPoolStreams];
    it[q].ev = hs.ev[q];
    it[q].host = hs.pinned + (size_t)q * kMaxK;
  }
  // fork from the caller's stream
  cudaEvent_t fork_ev = pool.ev[0];
  if ((e = cudaEventRecord(fork_ev, caller)) != cudaSuccess) return status_from_cuda(e);
  for (int i = 0; i < kPoolStreams && i < count; ++i)
    if ((e = cudaStreamWaitEvent(pool.st[i], fork_ev, 0)) != cudaSuccess) return status_from_cuda(e);
  for (int q = 0; q < count && e == cudaSuccess; ++q) {
    Solver& s = it[q].s;
    if ((e = s.setup()) == cudaSuccess) e = s.precond(s.B, s.ldb, s.X, s.ldx);   // x0 = U^{-1} L^{-1} b
  }
  auto any = [](const BatchItem& b, int Brief::*f) {
    for (int r = 0; r < b.s.K; ++r)
      if (b.host[r].*f) return true;
    return false;
  };
  int active = count;
  while (active > 0 && e == cudaSuccess) {
    // issue every active system's next phase
    for (int q = 0; q < count && e == cudaSuccess; ++q) {
      BatchItem& b = it[q];
      if (b.ph == kDone) continue;
      Solver& s = b.s;
      const SolveParams sp{s.K, s.m, s.prm.max_iters, s.prm.inner_tol, s.prm.theta, s.prm.accept, s.n};
      const cudaStream_t st = s.st;
      if (b.finish) {
        cycle_finish_kernel<<<1, 32, 0, st>>>(sp, s.w.st);
        update_kernel<<<(unsigned)cdiv<int64_t>(s.n, 256), 256, 0, st>>>(s.n, s.K, s.X, s.ldx, s.w.V, s.n,
                                                                         s.ldv_rhs(), s.w.st);
        count_launches(2);
        b.finish = false;
      }
      if (b.ph == kResid) {
        e = residual(s.n, s.K, s.A, s.lda, s.X, s.ldx, s.B, s.ldb, s.w.r, s.n, b.first ? 1 : 0, 1, s.w, st);
        check_kernel<<<1, 32, 0, st>>>(sp, s.w.st, s.w.brief, b.first ? 1 : 0);
        count_launches(1);
        b.first = false;
      } else if (b.ph == kCycle) {
        e = s.precond(s.w.r, s.n, s.w.tmp, s.n);
        norm2_kernel<<<kRedBlocks, 256, 0, st>>>(s.n, s.K, s.w.tmp, s.n, s.w.st, s.w.partials, s.w.counter);
        cycle_start_kernel<<<1, 32, 0, st>>>(sp, s.w.st, s.w.brief);
        scale_kernel<<<(unsigned)cdiv<int64_t>(s.n, 256), 256, 0, st>>>(s.n, s.K, s.w.tmp, s.n, s.w.V, s.ldv_rhs(),
                                                                         s.w.st, 0);
        count_launches(3);
      } else {   // Arnoldi step j
        const int j = b.j;
        e = residual(s.n, s.K, s.A, s.lda, s.w.V + (int64_t)j * s.n, s.ldv_rhs(), nullptr, 0, s.w.tmp, s.n,
                     s.prm.matvec_fp32 ? 3 : 0, 0, s.w, st);
        if (e == cudaSuccess) e = s.precond(s.w.tmp, s.n, s.w.w, s.n);
        s.arnoldi_tail(j);
      }
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.host, s.w.brief, sizeof(Brief) * s.K, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(b.ev, st);
    }
    if (e != cudaSuccess) break;
    // one decision point for the batch
    for (int q = 0; q < count && e == cudaSuccess; ++q) {
      BatchItem& b = it[q];
      if (b.ph == kDone) continue;
      if ((e = cudaEventSynchronize(b.ev)) != cudaSuccess) break;
      if (b.ph == kResid) {
        b.ph = any(b, &Brief::outer_active) ? kCycle : kDone;
      } else if (b.ph == kCycle) {
        if (!any(b, &Brief::outer_active)) {
          b.ph = kDone;
        } else if (any(b, &Brief::cycle_active) && b.s.m > 0) {
          b.ph = kArnoldi;
          b.j = 0;
        } else {
          b.finish = true;
          b.ph = kResid;
        }
      } else {
        b.j += 1;
        if (!(b.j < b.s.m && any(b, &Brief::cycle_active))) {
          b.finish = true;
          b.ph = kResid;
        }
      }
      if (b.ph == kDone) --active;
    }
  }
  // join back to the caller's stream
  for (int i = 0; i < kPoolStreams && i < count; ++i) {
    cudaEventRecord(pool.ev[i], pool.st[i]);
    cudaStreamWaitEvent(caller, pool.ev[i], 0);
  }
  if (e != cudaSuccess) return status_from_cuda(e);
  int worst = HPMXP_OK;
  int64_t off = 0;
  for (int q = 0; q < count; ++q) {
    BatchItem& b = it[q];
    uint32_t word = 0;
    if ((e = read_to_host(&word, b.s.w.status, 4, caller)) != cudaSuccess) return status_from_cuda(e);
    if (word && worst == HPMXP_OK) worst = status_from_word(word);
    for (int r = 0; r < b.s.K; ++r) {
      if (info) {
        info[off + r].iters = b.host[r].iters;
        info[off + r].outer = b.host[r].outer;
        info[off + r].scaled_resid = b.host[r].sr;
        info[off + r].status = b.host[r].status;
        info[off + r].reserved = 0;
      }
      if (b.host[r].status != HPMXP_OK && worst == HPMXP_OK) worst = b.host[r].status;
    }
    off += b.s.K;
  }
  return (hpmxp_status)worst;
}

hpmxp_status precond_apply(int64_t n, const void* LU, int64_t ldlu, int fmt, const double* v, int64_t ldv,
                           double* z, int64_t ldz, int64_t nrhs, int fp32, void* ws, cudaStream_t st,
                           const double* rs, const double* cs) {
  Solver s;
  s.n = n; s.K = (int)nrhs; s.m = 1;
  s.LU = (const uint16_t*)LU; s.ldlu = ldlu; s.fmt = fmt;
  s.rs = rs; s.cs = cs;
  hpmxp_ir_params_default(&s.prm);
  s.prm.precond_fp32 = fp32;
  s.w = carve_solve(ws, n, nrhs, 1);
  s.st = st;
  cudaError_t e = s.setup();
  if (e == cudaSuccess) e = s.precond(v, ldv, z, ldz);
  uint32_t word = 0;
  if (e == cudaSuccess) e = read_to_host(&word, s.w.status, 4, st);
  if (e != cudaSuccess) return status_from_cuda(e);
  return status_from_word(word);
}

// r = b - A x (fp64, the refinement's residual kernels), every column.
hpmxp_status residual_vector(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                             const double* b, int64_t ldb, int64_t nrhs, double* r, int64_t ldr, void* ws,
                             cudaStream_t st) {
  SolveWs w = carve_solve(ws, n, nrhs, 1);
  cudaError_t e = cudaMemsetAsync(w.st, 0, sizeof(RhsState) * kMaxK, st);
  if (e == cudaSuccess) e = residual(n, (int)nrhs, A, lda, x, ldx, b, ldb, r, ldr, 0, 0, w, st);
  return status_from_cuda(e);
}

hpmxp_status residual_check(int64_t n, const double* A, int64_t lda, const double* x, int64_t ldx,
                            const double* b, int64_t ldb, int64_t nrhs, double* out, void* ws, cudaStream_t st) {
  SolveWs w = carve_solve(ws, n, nrhs, 1);
  cudaError_t e = cudaMemsetAsync(w.st, 0, sizeof(RhsState) * kMaxK, st);
  if (e != cudaSuccess) return status_from_cuda(e);
  e = residual(n, (int)nrhs, A, lda, x, ldx, b, ldb, w.r, n, 2, 1, w, st);
  if (e != cudaSuccess) return status_from_cuda(e);
  std::vector<RhsState> hs(nrhs);
  e = read_to_host(hs.data(), w.st, sizeof(RhsState) * (size_t)nrhs, st);
  if (e != cudaSuccess) return status_from_cuda(e);
  for (int64_t r = 0; r < nrhs; ++r) {
    double rn, xn, bn, an;
    memcpy(&rn, &hs[r].rn_bits, 8); memcpy(&xn, &hs[r].xn_bits, 8);
    memcpy(&bn, &hs[r].bn_bits, 8); memcpy(&an, &hs[r].an_bits, 8);
    out[r] = rn / ((an * xn + bn) * ((double)n * 0x1p-53));
  }
  return HPMXP_OK;
}

}  // namespace hpmxp
