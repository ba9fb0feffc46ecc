// Low-precision blocked right-looking LU without pivoting (section
// "Algorithmic Framework", Fig. 1 and the paragraph after it).
//
// Schedule for update depth NB (128, 256 or 512), at every diagonal block
// D = [k, k+b):
//   (i)   factor D in fp32 arithmetic: a single-CTA shared-memory kernel for
//         128-wide sub-blocks (getrf + fp32 inverses of its L and U factors),
//         sub-blocks of a wider D chained by 128-deep panel/Schur products;
//   (ii)  U12 = L_D^{-1} A12 and L21 = A21 U_D^{-1} by block substitution over
//         the 128-wide sub-blocks s, each step ONE product with fp32
//         accumulation against a concatenated operand [W_s | Linv_ss] or
//         [Z_s ; Uinv_ss] (W_s = -Linv_ss L_{s,0:s}, Z_s = -U_{0:s,s} Uinv_ss);
//   (iii) A22 <- st(A22 - L21 U12), one tensor-core product of depth b.
// Every product runs on the GEMM engine (tcgen05 by default).  Operands are
// kept K-major: U12 is K-major in the column-major factor array already, and
// the column panel is packed row-major once per step.
//
// Streams (Factorizer::run): the caller's stream carries the diagonal block
// and the U12 chain; a third stream the L21 chain; a lowest-priority fourth
// W_s / Z_s (they depend only on the diagonal block, so they are made while it
// is still being factored); with look-ahead a second stream takes the far part
// of each Schur update.  The chain's kernels are launched as programmatic
// dependents (launch_pdl) and wait for their predecessor before touching
// global memory.
#include "internal.h"

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

namespace hpmxp {
namespace {

constexpr int kB = 128;         // base (sub-)block width

// ---------------------------------------------------------------------------
// fp64 -> 16-bit float, round to nearest even, written from the IEEE 754
// definition on the bit pattern (exponent rebias, 45- or 42-bit round-off with
// ties to even, subnormal quantum for tiny values, overflow to infinity).
// ---------------------------------------------------------------------------
// With k != 0 the value converted is x * 2^k (a power-of-two balancing
// scale): the scaling only moves the exponent, so it is one integer add here;
// an fp64-subnormal x (far below every 16-bit format) is scaled by an fp64
// multiply first.
template <int kMant, int kBias>
__device__ inline uint16_t f64_to_f16bits(double x, int k = 0) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  int e = (int)((u >> 52) & 0x7ff);
  if (e == 0 && k != 0 && (u << 1) != 0) {
    u = (unsigned long long)__double_as_longlong(x * ldexp(1.0, k));
    e = (int)((u >> 52) & 0x7ff);
    k = 0;
  }
  const uint32_t sign = (uint32_t)(u >> 63) << 15;
  const unsigned long long m = u & ((1ull << 52) - 1);
  constexpr int kExpBits = 15 - kMant;
  constexpr uint32_t kInf = ((1u << kExpBits) - 1) << kMant;
  if (e == 0x7ff) return (uint16_t)(sign | kInf | (m ? (1u << (kMant - 1)) : 0u));
  if (e == 0) return (uint16_t)sign;            // zero; fp64 subnormals are far below the 16-bit ones
  e += k;                                       // exponent of x * 2^k (may leave fp64's range: handled below)
  const int E = e - 1023 + kBias;             // biased target exponent
  if (E >= (1 << kExpBits) - 1) return (uint16_t)(sign | kInf);
  if (E >= 1) {
    constexpr int kDrop = 52 - kMant;
    const unsigned long long keep = m >> kDrop, rem = m & ((1ull << kDrop) - 1);
    const unsigned long long half = 1ull << (kDrop - 1);
    uint32_t r = ((uint32_t)E << kMant) | (uint32_t)keep;
    if (rem > half || (rem == half && (keep & 1))) r += 1;   // may carry into the exponent / infinity
    return (uint16_t)(sign | r);
  }
  // target subnormal: value = mf 2^(e-1075) = q * 2^(1 - kBias - kMant)
  const unsigned long long mf = m | (1ull << 52);
  const int s = 1075 - e - (kBias - 1 + kMant);  // right shift taking mf to units of the quantum
  if (s > 63) return (uint16_t)sign;
  const unsigned long long q = mf >> s, rem = mf & ((1ull << s) - 1), half = 1ull << (s - 1);
  uint32_t r = (uint32_t)q;
  if (rem > half || (rem == half && (q & 1))) r += 1;
  return (uint16_t)(sign | r);
}

__device__ inline uint16_t f64_to_u16(double x, int fmt) {
  return fmt == kBF16 ? f64_to_f16bits<7, 127>(x) : f64_to_f16bits<10, 15>(x);
}

// Exponent k of a power of two 2^k (a normal fp64 value).
__device__ inline int pow2_exponent(double s) {
  return (int)(((unsigned long long)__double_as_longlong(s) >> 52) & 0x7ff) - 1023;
}

// f64_to_u16(x * 2^k): the power-of-two scale is an exponent add inside the
// conversion (GB300's fp64 rate is low enough that one fp64 multiply per
// entry would cost as much as reading the matrix).
__device__ inline uint16_t f64_to_u16_pow2(double x, int k, int fmt) {
  return fmt == kBF16 ? f64_to_f16bits<7, 127>(x, k) : f64_to_f16bits<10, 15>(x, k);
}

// A (fp64, column major) -> LU (16-bit, column major), optionally of the
// balanced matrix diag(rs) A diag(cs) (rs, cs powers of two, so the fp64
// products are exact and the one rounding is the cast's).  CTA (x, y)
// converts rows 2048 y .. +2047 of columns kCastCols x .. +kCastCols-1; each
// thread 8 consecutive rows (their scale exponents read once for all the
// columns) with four 16-byte loads and one 16-byte store per column when
// aligned (LU is 16-byte aligned with ldlu % 8 == 0), entry by entry otherwise.
constexpr int kCastRows = 256 * 8;
constexpr int kCastCols = 4;
__global__ void __launch_bounds__(256) cast_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                                   uint16_t* __restrict__ LU, int64_t ldlu, int fmt,
                                                   const double* __restrict__ rs, const double* __restrict__ cs) {
  const int64_t i = (int64_t)blockIdx.y * kCastRows + 8 * (int64_t)threadIdx.x;
  if (i >= n) return;
  int er[8];   // exponents of the power-of-two row scales of the thread's rows
#pragma unroll
  for (int k = 0; k < 8; ++k) er[k] = (rs && i + k < n) ? pow2_exponent(rs[i + k]) : 0;
  const int64_t jend = min((int64_t)(blockIdx.x + 1) * kCastCols, n);
  for (int64_t j = (int64_t)blockIdx.x * kCastCols; j < jend; ++j) {
    const double* src = A + i + j * lda;
    uint16_t* dst = LU + i + j * ldlu;
    const int kc = cs ? pow2_exponent(cs[j]) : 0;
    if (i + 8 <= n && (((uintptr_t)src) & 15) == 0) {
      double2 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldcs(reinterpret_cast<const double2*>(src) + k);
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        w[k] = (uint32_t)f64_to_u16_pow2(v[k].x, kc + er[2 * k], fmt) |
               ((uint32_t)f64_to_u16_pow2(v[k].y, kc + er[2 * k + 1], fmt) << 16);
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      for (int k = 0; k < 8 && i + k < n; ++k) dst[k] = f64_to_u16_pow2(src[k], kc + er[k], fmt);
    }
  }
}

// ---------------------------------------------------------------------------
// 32-bit trailing matrix (Fig. 1 with 32-bit storage of the matrix being
// updated): A (fp64, optionally balanced by powers of two) -> W (fp32, round
// to nearest even), and a region of W -> the 16-bit factor array when it
// becomes a panel (one rounding, nearest even).
// ---------------------------------------------------------------------------
__device__ inline double times_pow2(double x, int k) {   // x * 2^k, an exponent add for normal x
  if (k == 0) return x;
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff || e + k <= 0 || e + k >= 0x7ff) return x * ldexp(1.0, k);
  return __longlong_as_double((long long)(u + ((unsigned long long)(int64_t)k << 52)));
}

__global__ void __launch_bounds__(256) cast32_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                                     float* __restrict__ W, int64_t ldw,
                                                     const double* __restrict__ rs, const double* __restrict__ cs) {
  const int64_t j = blockIdx.x;   // column (grid x holds up to 2^31 - 1)
  const int64_t i = (int64_t)blockIdx.y * 256 + threadIdx.x;
  if (i >= n) return;
  const int k = (rs ? pow2_exponent(rs[i]) : 0) + (cs ? pow2_exponent(cs[j]) : 0);
  W[i + j * ldw] = __double2float_rn(times_pow2(__ldcs(A + i + j * lda), k));
}

__global__ void __launch_bounds__(256) round32_kernel(int64_t rows, int64_t cols, const float* __restrict__ W,
                                                      int64_t ldw, uint16_t* __restrict__ LU, int64_t ld, int fmt) {
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= rows) return;
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y) LU[i + j * ld] = f32_to_u16(W[i + j * ldw], fmt);
}

// ---------------------------------------------------------------------------
// Balancing and scaling (section "Algorithmic Framework": a Theta(n^2)
// balancing of the input borrowed from the HPL harness, and a scaling that
// makes the values fit the low-precision format, both timed and undone).
// Power-of-two row then column equilibration: rs_i = 2^-floor(log2 max_j
// |a_ij|), cs_j = 2^-floor(log2 max_i |rs_i a_ij|), so every row and column of
// diag(rs) A diag(cs) has its largest magnitude in [1, 2); a row or column
// with a non-finite entry, or only zeros, gets scale 1; then rs *= 2^k, the
// format's scale (k = 12 for FP16, whose range ends at 65504 and whose normal
// range at 2^-14; 0 for BF16, which has fp32's range).  Row maxima are taken
// on the bit patterns of non-negative doubles (ordered like the values, NaN
// and infinity above every finite value); the column pass needs only
// floor(log2 |rs_i a_ij|) = floor(log2 |a_ij|) + log2 rs_i, an integer max:
// no fp64 arithmetic per entry, and any reduction order gives the same bits.
// ---------------------------------------------------------------------------
constexpr int kBalRows = 512;        // rows per CTA of the row pass (256 threads x 2)
constexpr int kBalChunk = 1024;      // columns per CTA of the row pass

__device__ inline unsigned long long abs_bits(double a) {
  return (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
}

// pass 1: rmax[i] = max_j |a_ij| as a bit pattern (rmax zeroed first)
__global__ void __launch_bounds__(256) row_absmax_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                                         unsigned long long* __restrict__ rmax) {
  const int64_t i = (int64_t)blockIdx.x * kBalRows + 2 * threadIdx.x;
  if (i >= n) return;
  const int64_t j0 = (int64_t)blockIdx.y * kBalChunk, j1 = min(j0 + (int64_t)kBalChunk, n);
  const bool two = i + 1 < n;
  const bool vec = two && ((((uintptr_t)(A + i)) & 15) == 0) && ((lda & 1) == 0);
  unsigned long long m0 = 0, m1 = 0;
  const double* col = A + i + j0 * lda;
  int64_t j = j0;
  if (vec) {
    for (; j + 8 <= j1; j += 8) {   // eight 16-byte loads in flight per thread
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcs(reinterpret_cast<const double2*>(col + (int64_t)u * lda));
      col += 8 * lda;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        m0 = max(m0, abs_bits(v[u].x));
        m1 = max(m1, abs_bits(v[u].y));
      }
    }
  }
  for (; j < j1; ++j, col += lda) {
    m0 = max(m0, abs_bits(col[0]));
    if (two) m1 = max(m1, abs_bits(col[1]));
  }
  atomicMax(rmax + i, m0);
  if (two) atomicMax(rmax + i + 1, m1);
}

// 2^-floor(log2 m) for a finite m > 0, else 1 (a zero or non-finite row or
// column is left unscaled)
__device__ inline double pow2_inverse(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 1.0;
  int e;
  frexp(m, &e);                       // m = f 2^e, f in [0.5, 1): floor(log2 m) = e - 1
  return ldexp(1.0, 1 - e);
}

// floor(log2 |a|) for a finite nonzero a; kZeroLog for 0, kBadLog for inf / NaN
constexpr int kZeroLog = -100000, kBadLog = 100000;
__device__ inline int floor_log2_abs(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0x7ff) return kBadLog;
  if (e != 0) return e - 1023;
  if ((u & 0x000fffffffffffffull) == 0) return kZeroLog;
  int f;
  frexp(a, &f);                      // fp64 subnormal
  return f - 1;
}

// rmax bits -> rs_i (in place); the format scale is applied after the column pass
__global__ void row_scale_kernel(int64_t n, double* rs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rs[i] = pow2_inverse(rs[i]);
}

// pass 2: kBalCols columns per CTA (each row's rs read once for all of
// them): cs_j = 2^-floor(log2 max_i |rs_i a_ij|)
constexpr int kBalCols = 8;
__global__ void __launch_bounds__(256) col_scale_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ rs, double* __restrict__ cs) {
  __shared__ int wmax[8][kBalCols];
  const int64_t j0 = (int64_t)blockIdx.x * kBalCols;
  const int nc = (int)min((int64_t)kBalCols, n - j0);
  int m[kBalCols];
#pragma unroll
  for (int c = 0; c < kBalCols; ++c) m[c] = kZeroLog;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    const int er = pow2_exponent(rs[i]);
    double a[kBalCols];
#pragma unroll
    for (int c = 0; c < kBalCols; ++c) a[c] = c < nc ? __ldcs(A + i + (j0 + c) * lda) : 0.0;
#pragma unroll
    for (int c = 0; c < kBalCols; ++c) {
      const int l = floor_log2_abs(a[c]);
      m[c] = max(m[c], l >= kBadLog ? kBadLog : (l <= kZeroLog ? kZeroLog : l + er));
    }
  }
#pragma unroll
  for (int c = 0; c < kBalCols; ++c) {
    for (int o = 16; o > 0; o >>= 1) m[c] = max(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5][c] = m[c];
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    int mm = wmax[0][c];
    for (int w = 1; w < 8; ++w) mm = max(mm, wmax[w][c]);
    cs[j0 + c] = (mm == kZeroLog || mm == kBadLog) ? 1.0 : ldexp(1.0, -mm);
  }
}

__global__ void format_scale_kernel(int64_t n, double* rs, double s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rs[i] *= s;
}

// ---------------------------------------------------------------------------
// (i) Diagonal block of width b <= 128, one CTA of 16 warps, entirely in
// shared memory (fp32).  Factorization: right-looking unblocked elimination
// (l = a / pivot, then a -= l u by fused multiply-add, pivots ascending),
// organised in 16-column panels: warps 0-3 eliminate the panel (one row per
// lane, pivot row through shared memory, one named barrier per pivot), all
// warps then solve the panel's row strip and apply the rank-16 update.  Every
// entry still receives its updates one FMA at a time in ascending pivot
// order, so the result is identical to the unblocked loop.
// Inverses of the stored unit-lower L and upper U, each by 16-row blocks in
// the same per-entry operation order as the plain recurrences
//   X = L^{-1}: X[r][c] = -sum_{t=c}^{r-1} L[r][t] X[t][c]   (t ascending)
//   Y = U^{-1}: Y[c][c] = 1 / U[c][c];
//               Y[r][c] = (-sum_{t=c}^{r+1} U[r][t] Y[t][c]) / U[r][r] (t descending)
// computed concurrently by warps 0-7 (X) and 8-15 (Y), rounded to storage
// and written as the K-major GEMM operands Linv (Linv[p*ldl + t]) and Uinv^T
// (UinvT[p*ldu + t] = Uinv[t][p]).  128 x 128 zero-padded.
// ---------------------------------------------------------------------------
constexpr int kGetrfThreads = 512;
constexpr int kP = 132;    // shared pitch (floats): 16-byte aligned columns
constexpr int kPW = 16;    // panel width
constexpr size_t kGetrfSmem = sizeof(float) * (3 * kB * kP + 2 * kPW + 8);
static_assert(kGetrfSmem <= 232448, "getrf's shared memory fits one CTA");

__device__ inline void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// rank-kPW update of the block rows [i0, i1) x cols [j0, j1) of M (pitch kP):
// M(i, j) += sgn * sum_{t in order} L(i, t) * R(t, j) with L(i,t) = Lm[t*kP + i],
// R(t, j) = Rm[j*kP + t]; kDesc walks t from t1-1 down to t0, else up.  4x4
// register micro-tiles dealt out one per thread of the group (tile rows
// fastest), so a narrow block keeps every lane busy.  A full 16-deep slice
// (t0 a multiple of 16) reads R four pivots at a time; the terms of every
// entry still come one FMA at a time in the same order.
template <bool kDesc>
__device__ inline void rank_update(float* M, const float* Lm, const float* Rm, int i0, int i1, int j0, int j1,
                                   int t0, int t1, float sgn, int wid, int nwarps, int lane) {
  const int ni = (i1 - i0 + 3) / 4, nj = (j1 - j0 + 3) / 4;
  const bool full = t1 - t0 == kPW && (t0 & 3) == 0;
  for (int k = 32 * wid + lane; k < ni * nj; k += 32 * nwarps) {
    {
      const int ti = k % ni, tj = k / ni;
      const int i = i0 + 4 * ti, j = j0 + 4 * tj;
      float acc[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][c] = M[(j + c) * kP + i + r];
      if (full) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int tg = t0 + 4 * (kDesc ? 3 - g : g);
          float rv[4][4];   // rv[c][u] = R(tg + u, j + c)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 r4 = *reinterpret_cast<const float4*>(&Rm[(j + c) * kP + tg]);
            rv[c][0] = r4.x; rv[c][1] = r4.y; rv[c][2] = r4.z; rv[c][3] = r4.w;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int uu = kDesc ? 3 - u : u;
            const float4 l4 = *reinterpret_cast<const float4*>(&Lm[(tg + uu) * kP + i]);
            const float l[4] = {sgn * l4.x, sgn * l4.y, sgn * l4.z, sgn * l4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int r = 0; r < 4; ++r) acc[r][c] = __fmaf_rn(l[r], rv[c][uu], acc[r][c]);
          }
        }
      } else {
        for (int k = 0; k < t1 - t0; ++k) {
          const int t = kDesc ? t1 - 1 - k : t0 + k;
          const float4 l4 = *reinterpret_cast<const float4*>(&Lm[t * kP + i]);
          const float l[4] = {sgn * l4.x, sgn * l4.y, sgn * l4.z, sgn * l4.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float u = Rm[(j + c) * kP + t];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][c] = __fmaf_rn(l[r], u, acc[r][c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (i + r < i1 && j + c < j1) M[(j + c) * kP + i + r] = acc[r][c];
    }
  }
}

// The 16 floats v[0..15] = p[0..15] (p 16-byte aligned).
__device__ inline void load16(float (&v)[kPW], const float* p) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float4 q = *reinterpret_cast<const float4*>(p + 4 * m);
    v[4 * m] = q.x; v[4 * m + 1] = q.y; v[4 * m + 2] = q.z; v[4 * m + 3] = q.w;
  }
}
__device__ inline void store16(float* p, const float (&v)[kPW]) {
#pragma unroll
  for (int m = 0; m < 4; ++m)
    *reinterpret_cast<float4*>(p + 4 * m) = make_float4(v[4 * m], v[4 * m + 1], v[4 * m + 2], v[4 * m + 3]);
}

// The pieces of the diagonal-block kernels.  `a` holds the block in fp32
// (pitch kP, zero outside b x b); x = L^{-1}, y = U^{-1} (x[c * kP + r] = X(r, c)).

// a <- D (16-bit, column major), zero outside b x b; threads tid .. of nt
__device__ __forceinline__ void load_block(float* a, const uint16_t* __restrict__ D, int64_t ldd, int b, int fmt,
                                           bool vec, int tid, int nt) {
  if (vec) {
    for (int v = tid; v < kB * kB / 8; v += nt) {
      const int i = 8 * (v % (kB / 8)), j = v / (kB / 8);
      const uint4 w = *reinterpret_cast<const uint4*>(D + i + (int64_t)j * ldd);
      const uint32_t h[4] = {w.x, w.y, w.z, w.w};
      float f[8];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        f[2 * m] = u16_to_f32((uint16_t)(h[m] & 0xFFFFu), fmt);
        f[2 * m + 1] = u16_to_f32((uint16_t)(h[m] >> 16), fmt);
      }
      *reinterpret_cast<float4*>(&a[j * kP + i]) = make_float4(f[0], f[1], f[2], f[3]);
      *reinterpret_cast<float4*>(&a[j * kP + i + 4]) = make_float4(f[4], f[5], f[6], f[7]);
    }
  } else {
    for (int idx = tid; idx < kB * kB; idx += nt) {
      const int i = idx % kB, j = idx / kB;
      a[j * kP + i] = (i < b && j < b) ? u16_to_f32(D[i + (int64_t)j * ldd], fmt) : 0.0f;
    }
  }
}

// LU without pivoting of a (b x b) in fp32, in place; kGetrfThreads threads.
// A zero or non-finite pivot sets kErrPivot.
__device__ __forceinline__ void lu_block(float* a, float* urow, int b, uint32_t* status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool bad = false;
  // (a) panel: rows p0..b-1 (one per lane of warps 0-3), columns p0..p0+pw-1
  auto eliminate = [&](int p0, int pw) {
    const int i = p0 + 32 * warp + lane;
    const bool has = i < b;
    float pr[kPW];
#pragma unroll
    for (int c = 0; c < kPW; ++c) pr[c] = (has && c < pw) ? a[(p0 + c) * kP + i] : 0.0f;
#pragma unroll
    for (int cp = 0; cp < kPW; ++cp) {
      if (cp >= pw) break;
      const int p = p0 + cp;
      float* ur = urow + (cp & 1) * kPW;
      if (warp == 0 && lane == cp) store16(ur, pr);   // row p is lane cp of warp 0
      named_sync(1, 128);
      float u[kPW];
      load16(u, ur);
      const float piv = u[cp];
      if (!(isfinite(piv) && piv != 0.0f)) bad = true;
      if (has && i > p) {
        const float l = __fdiv_rn(pr[cp], piv);
        pr[cp] = l;
#pragma unroll
        for (int c = cp + 1; c < kPW; ++c)
          if (c < pw) pr[c] = __fmaf_rn(-l, u[c], pr[c]);
      }
    }
    if (has) {
#pragma unroll
      for (int c = 0; c < kPW; ++c)
        if (c < pw) a[(p0 + c) * kP + i] = pr[c];
    }
  };
  if (warp < 4) eliminate(0, min(kPW, b));
  __syncthreads();
  for (int p0 = 0; p0 < b; p0 += kPW) {
    const int e = p0 + kPW;   // a ragged panel is the last one: nothing follows it
    if (e >= b) break;
    // (b) row strip: rows p0..e-1, columns e..b-1, unit-lower solve with the
    // panel, right-looking (pivot q ascending, so each entry's terms keep
    // their order and the loads of step q+1 overlap step q)
    for (int j = e + tid; j < b; j += kGetrfThreads) {
      float col[kPW];
      load16(col, &a[j * kP + p0]);
#pragma unroll
      for (int q = 0; q < kPW - 1; ++q) {
        float lq[kPW];   // column p0 + q of the panel, rows p0 .. p0 + 15
        load16(lq, &a[(p0 + q) * kP + p0]);
#pragma unroll
        for (int r = q + 1; r < kPW; ++r) col[r] = __fmaf_rn(-lq[r], col[q], col[r]);
      }
      store16(&a[j * kP + p0], col);
    }
    __syncthreads();
    // (c) trailing update rows/cols e..b-1, pivots p0..e-1 ascending, with
    // look-ahead: warps 0-3 update the next panel's columns [e, e2) and go on
    // to eliminate it while warps 4-15 update the columns after it
    const int e2 = min(e + kPW, b);
    if (warp < 4) {
      rank_update<false>(a, a, a, e, b, e, e2, p0, e, -1.0f, warp, 4, lane);
      named_sync(1, 128);
      eliminate(e, e2 - e);
    } else if (e2 < b) {
      rank_update<false>(a, a, a, e, b, e2, b, p0, e, -1.0f, warp - 4, kGetrfThreads / 32 - 4, lane);
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicOr(status, kErrPivot);

}

// D <- round(a); a <- the stored values (the factors' exact fp32 values);
// with x / y given also X = I and Y = diag(1 / stored U)
__device__ __forceinline__ void round_block(float* a, uint16_t* __restrict__ D, int64_t ldd, int b, int fmt,
                                            bool vec, float* x, float* y, int tid, int nt) {
  if (vec) {
    for (int v = tid; v < kB * kB / 8; v += nt) {
      const int i = 8 * (v % (kB / 8)), j = v / (kB / 8);
      float f[8];
      const float4 f0 = *reinterpret_cast<const float4*>(&a[j * kP + i]);
      const float4 f1 = *reinterpret_cast<const float4*>(&a[j * kP + i + 4]);
      f[0] = f0.x; f[1] = f0.y; f[2] = f0.z; f[3] = f0.w; f[4] = f1.x; f[5] = f1.y; f[6] = f1.z; f[7] = f1.w;
      uint32_t h[4];
      float xs[8], ys[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const uint16_t hm = f32_to_u16(f[m], fmt);
        if (m & 1) h[m >> 1] |= (uint32_t)hm << 16; else h[m >> 1] = hm;
        f[m] = u16_to_f32(hm, fmt);
        xs[m] = i + m == j ? 1.0f : 0.0f;
        ys[m] = i + m == j ? __fdiv_rn(1.0f, f[m]) : 0.0f;
      }
      *reinterpret_cast<uint4*>(D + i + (int64_t)j * ldd) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(&a[j * kP + i]) = make_float4(f[0], f[1], f[2], f[3]);
      *reinterpret_cast<float4*>(&a[j * kP + i + 4]) = make_float4(f[4], f[5], f[6], f[7]);
      if (x) {
        *reinterpret_cast<float4*>(&x[j * kP + i]) = make_float4(xs[0], xs[1], xs[2], xs[3]);
        *reinterpret_cast<float4*>(&x[j * kP + i + 4]) = make_float4(xs[4], xs[5], xs[6], xs[7]);
      }
      if (y) {
        *reinterpret_cast<float4*>(&y[j * kP + i]) = make_float4(ys[0], ys[1], ys[2], ys[3]);
        *reinterpret_cast<float4*>(&y[j * kP + i + 4]) = make_float4(ys[4], ys[5], ys[6], ys[7]);
      }
    }
  } else {
    for (int idx = tid; idx < kB * kB; idx += nt) {
      const int i = idx % kB, j = idx / kB;
      float v = 0.0f;
      if (i < b && j < b) {
        const uint16_t h = f32_to_u16(a[j * kP + i], fmt);
        D[i + (int64_t)j * ldd] = h;
        v = u16_to_f32(h, fmt);
      }
      a[j * kP + i] = v;
      if (x) x[j * kP + i] = (i == j && i < b) ? 1.0f : 0.0f;
      if (y) y[j * kP + i] = (i == j && i < b) ? __fdiv_rn(1.0f, v) : 0.0f;
    }
  }
}

// X = I and Y = diag(1 / a_ii) for a block whose a already holds stored values
__device__ __forceinline__ void init_inverse(float* m, const float* a, int b, bool upper, int tid, int nt) {
  for (int idx = tid; idx < kB * kB; idx += nt) {
    const int i = idx % kB, j = idx / kB;
    m[j * kP + i] = (i == j && i < b) ? (upper ? __fdiv_rn(1.0f, a[j * kP + i]) : 1.0f) : 0.0f;
  }
}

// X = L^{-1} (unit lower part of a), 16-row blocks top-down, by the NT
// threads gt = 0 .. NT-1 (warps gw) of one group with barrier BAR.  The
// result does not depend on NT: every entry takes its terms in one order.
template <int NT, int BAR>
__device__ __forceinline__ void inv_lower(float* x, const float* a, int b, int gt, int gw, int lane) {
  for (int t0 = 0; t0 < b; t0 += kPW) {
    const int t1 = min(t0 + kPW, b);
    // rows t0..t1-1, every column c < t1: within-block terms t = t0 .. r-1 in
    // ascending order; X(t, c) = 0 for t < c, so those terms are exact no-ops
    // and each entry sees the same operations as the plain recurrence
    for (int c = gt; c < t1; c += NT) {
      float col[kPW];
      if (t1 - t0 == kPW) {
        load16(col, &x[c * kP + t0]);
#pragma unroll
        for (int q = 0; q < kPW - 1; ++q) {
          float lq[kPW];   // column t0 + q of L, rows t0 .. t0 + 15
          load16(lq, &a[(t0 + q) * kP + t0]);
#pragma unroll
          for (int r = q + 1; r < kPW; ++r) col[r] = __fmaf_rn(-lq[r], col[q], col[r]);
        }
        store16(&x[c * kP + t0], col);
      } else {
#pragma unroll
        for (int r = 0; r < kPW; ++r) col[r] = (t0 + r < t1) ? x[c * kP + t0 + r] : 0.0f;
#pragma unroll
        for (int q = 0; q < kPW - 1; ++q) {
#pragma unroll
          for (int r = q + 1; r < kPW; ++r)
            if (t0 + r < t1) col[r] = __fmaf_rn(-a[(t0 + q) * kP + t0 + r], col[q], col[r]);
        }
#pragma unroll
        for (int r = 0; r < kPW; ++r)
          if (t0 + r < t1) x[c * kP + t0 + r] = col[r];
      }
    }
    named_sync(BAR, NT);
    // rows t1..b-1, columns 0..t1-1: add -L(r, t) X(t, c) for t = t0..t1-1 ascending
    if (t1 < b) rank_update<false>(x, a, x, t1, b, 0, t1, t0, t1, -1.0f, gw, NT / 32, lane);
    named_sync(BAR, NT);
  }
}

// Y = U^{-1} (upper part of a, Y's diagonal preset to 1 / U(r, r)), 16-row
// blocks bottom-up, by the NT threads of one group with barrier BAR
template <int NT, int BAR>
__device__ __forceinline__ void inv_upper(float* y, const float* a, int b, int gt, int gw, int lane) {
  const int nblk = (b + kPW - 1) / kPW;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int t0 = bi * kPW, t1 = min(t0 + kPW, b);
    // rows t1-1 down to t0, every column c >= t0, right-looking: finalize row
    // t0+q (divide, unless it is the diagonal or below it), then add its term
    // to the rows above it; terms come in descending t, rows t > c carry 0
    for (int c = t0 + gt; c < b; c += NT) {
      float col[kPW];
      if (t1 - t0 == kPW) {
        load16(col, &y[c * kP + t0]);
        // uq = column rq of U, rows t0 .. t0 + 15 (uq[q] = U(rq, rq)); the
        // next column is fetched while this one is applied
        float uq[kPW], un[kPW];
        load16(uq, &a[(t0 + kPW - 1) * kP + t0]);
#pragma unroll
        for (int q = kPW - 1; q >= 0; --q) {
          const int rq = t0 + q;
          if (q > 0) load16(un, &a[(rq - 1) * kP + t0]);
          if (rq < c) col[q] = __fdiv_rn(-col[q], uq[q]);
#pragma unroll
          for (int r = 0; r < q; ++r) col[r] = __fmaf_rn(uq[r], col[q], col[r]);
          if (q > 0) {
#pragma unroll
            for (int r = 0; r < kPW; ++r) uq[r] = un[r];
          }
        }
        store16(&y[c * kP + t0], col);
      } else {
#pragma unroll
        for (int r = 0; r < kPW; ++r) col[r] = (t0 + r < t1) ? y[c * kP + t0 + r] : 0.0f;
#pragma unroll
        for (int q = kPW - 1; q >= 0; --q) {
          const int rq = t0 + q;
          if (rq < t1 && rq < c) col[q] = __fdiv_rn(-col[q], a[rq * kP + rq]);
#pragma unroll
          for (int r = 0; r < q; ++r)
            if (rq < t1) col[r] = __fmaf_rn(a[rq * kP + t0 + r], col[q], col[r]);
        }
#pragma unroll
        for (int r = 0; r < kPW; ++r)
          if (t0 + r < t1) y[c * kP + t0 + r] = col[r];
      }
    }
    named_sync(BAR, NT);
    // rows 0..t0-1, columns t0..b-1: add U(r, t) Y(t, c) for t = t1-1 down to t0
    if (t0 > 0) rank_update<true>(y, a, y, 0, t0, t0, b, t0, t1, 1.0f, gw, NT / 32, lane);
    named_sync(BAR, NT);
  }
}

// Linv[p][t] = X(p, t) and UinvT[p][t] = Y(t, p), rounded; zero outside b x b
__device__ __forceinline__ void store_inverse(const float* m, bool upper, int b, int fmt, uint16_t* __restrict__ out,
                                              int64_t ldo, int tid, int nt) {
  if ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && (ldo & 7) == 0) {
    for (int v = tid; v < kB * kB / 8; v += nt) {
      const int t0 = 8 * (v % (kB / 8)), pp = v / (kB / 8);
      uint32_t h[4];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool in = pp < b && t0 + q < b;
        const uint16_t e = in ? f32_to_u16(upper ? m[pp * kP + t0 + q] : m[(t0 + q) * kP + pp], fmt) : (uint16_t)0;
        if (q & 1) h[q >> 1] |= (uint32_t)e << 16; else h[q >> 1] = e;
      }
      *reinterpret_cast<uint4*>(out + (int64_t)pp * ldo + t0) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  } else {
    for (int idx = tid; idx < kB * kB; idx += nt) {
      const int t = idx % kB, pp = idx / kB;
      const bool in = pp < b && t < b;
      out[(int64_t)pp * ldo + t] = in ? f32_to_u16(upper ? m[pp * kP + t] : m[t * kP + pp], fmt) : (uint16_t)0;
    }
  }
}

__device__ __forceinline__ bool block_vec(int b, const uint16_t* D, int64_t ldd) {
  return b == kB && (reinterpret_cast<uintptr_t>(D) & 15) == 0 && (ldd & 7) == 0;
}

// The whole diagonal block in one CTA: LU, then L^{-1} (warps 0-7) beside
// U^{-1} (warps 8-15), then both inverses stored (the batched factorization's
// grouped kernel)
__device__ __forceinline__ void getrf_block(int b, uint16_t* __restrict__ D, int64_t ldd, int fmt,
                                            uint16_t* __restrict__ linv, int64_t ldl, uint16_t* __restrict__ uinvT,
                                            int64_t ldu, uint32_t* status) {
  extern __shared__ float sm[];
  float* a = sm;
  float* x = sm + kB * kP;
  float* y = sm + 2 * kB * kP;
  float* urow = sm + 3 * kB * kP; // [2][kPW] pivot row of the current panel step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool vec = block_vec(b, D, ldd);
  load_block(a, D, ldd, b, fmt, vec, tid, kGetrfThreads);
  __syncthreads();
  lu_block(a, urow, b, status);
  round_block(a, D, ldd, b, fmt, vec, x, y, tid, kGetrfThreads);
  __syncthreads();
  if (warp < 8) inv_lower<256, 2>(x, a, b, tid, warp, lane);
  else inv_upper<256, 3>(y, a, b, tid - 256, warp - 8, lane);
  __syncthreads();
  store_inverse(x, false, b, fmt, linv, ldl, tid, kGetrfThreads);
  store_inverse(y, true, b, fmt, uinvT, ldu, tid, kGetrfThreads);
}

// The single-system factorization splits the block's work over two kernels:
// the LU (one CTA), then its two inverses side by side (CTA 0: L^{-1}, CTA 1:
// U^{-1}, all kGetrfThreads threads each), from the stored factors.  The
// same operations per entry as getrf_block, so the same bits.
constexpr size_t kLuSmem = sizeof(float) * (kB * kP + 2 * kPW + 8);
constexpr size_t kInvSmem = sizeof(float) * 2 * kB * kP;

__global__ void __launch_bounds__(kGetrfThreads)
getrf_lu_kernel(int b, uint16_t* __restrict__ D, int64_t ldd, int fmt, uint32_t* status) {
  extern __shared__ float sm[];
  float* a = sm;
  float* urow = sm + kB * kP;
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x;
  const bool vec = block_vec(b, D, ldd);
  load_block(a, D, ldd, b, fmt, vec, tid, kGetrfThreads);
  __syncthreads();
  lu_block(a, urow, b, status);
  round_block(a, D, ldd, b, fmt, vec, nullptr, nullptr, tid, kGetrfThreads);
}

__global__ void __launch_bounds__(kGetrfThreads)
getrf_inv_kernel(int b, const uint16_t* __restrict__ D, int64_t ldd, int fmt, uint16_t* __restrict__ linv,
                 int64_t ldl, uint16_t* __restrict__ uinvT, int64_t ldu) {
  extern __shared__ float sm[];
  float* a = sm;
  float* m = sm + kB * kP;
  pdl_wait();      // the LU kernel has stored the factors
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool upper = blockIdx.x == 1;
  load_block(a, D, ldd, b, fmt, block_vec(b, D, ldd), tid, kGetrfThreads);
  __syncthreads();
  init_inverse(m, a, b, upper, tid, kGetrfThreads);
  __syncthreads();
  if (upper) inv_upper<kGetrfThreads, 1>(m, a, b, tid, warp, lane);
  else inv_lower<kGetrfThreads, 1>(m, a, b, tid, warp, lane);
  __syncthreads();
  if (upper) store_inverse(m, true, b, fmt, uinvT, ldu, tid, kGetrfThreads);
  else store_inverse(m, false, b, fmt, linv, ldl, tid, kGetrfThreads);
}

// Grouped diagonal blocks: CTA t factors task t's block (batched
// factorization: one launch for the current block of every problem).
struct GetrfTask {
  uint16_t* D;
  int64_t ldd;
  uint16_t* linv;
  int64_t ldl;
  uint16_t* uinvT;
  int64_t ldu;
  uint32_t* status;
  int b;
};
__global__ void __launch_bounds__(kGetrfThreads) getrf_grouped_kernel(const GetrfTask* __restrict__ tasks, int fmt) {
  pdl_wait();
  pdl_trigger();
  const GetrfTask t = tasks[blockIdx.x];
  getrf_block(t.b, t.D, t.ldd, fmt, t.linv, t.ldl, t.uinvT, t.ldu, t.status);
}

// Column-major block (rows x cols at src, lds) -> row-major (dst[i*ldd + j]),
// through 64 x 64 tiles in shared memory (t[j][i], rows padded to 144 bytes).
// A whole tile with 16-byte aligned columns and rows moves by 16-byte loads
// (8 rows of one column) and 16-byte stores (8 columns of one row); the
// gathers in between read 32 consecutive rows per warp (no bank conflicts).
constexpr int kPackT = 64, kPackPad = 72;
__device__ __forceinline__ void pack_tile(int64_t rows, int cols, const uint16_t* __restrict__ src, int64_t lds,
                                          uint16_t* __restrict__ dst, int64_t ldd, int64_t bx, int by) {
  __shared__ __align__(16) uint16_t t[kPackT][kPackPad];
  const int64_t i0 = bx * kPackT;
  const int j0 = by * kPackT;
  const bool whole = i0 + kPackT <= rows && j0 + kPackT <= cols && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                     (lds & 7) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (ldd & 7) == 0;
  if (whole) {
    for (int v = threadIdx.x; v < kPackT * kPackT / 8; v += blockDim.x) {
      const int j = v >> 3, ic = (v & 7) * 8;
      *reinterpret_cast<uint4*>(&t[j][ic]) =
          *reinterpret_cast<const uint4*>(src + (i0 + ic) + (int64_t)(j0 + j) * lds);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < kPackT * kPackT / 8; v += blockDim.x) {
      const int i = v & (kPackT - 1), jc = (v >> 6) * 8;
      uint32_t h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) h[e] = (uint32_t)t[jc + 2 * e][i] | ((uint32_t)t[jc + 2 * e + 1][i] << 16);
      *reinterpret_cast<uint4*>(dst + (i0 + i) * ldd + j0 + jc) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  } else {
    for (int v = threadIdx.x; v < kPackT * kPackT; v += blockDim.x) {
      const int j = v >> 6, i = v & (kPackT - 1);
      t[j][i] = (i0 + i < rows && j0 + j < cols) ? src[(i0 + i) + (int64_t)(j0 + j) * lds] : (uint16_t)0;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < kPackT * kPackT; v += blockDim.x) {
      const int i = v >> 6, j = v & (kPackT - 1);
      if (i0 + i < rows && j0 + j < cols) dst[(i0 + i) * ldd + j0 + j] = t[j][i];
    }
  }
}

__global__ void __launch_bounds__(256) pack_rows_kernel(int64_t rows, int cols, const uint16_t* __restrict__ src,
                                                        int64_t lds, uint16_t* __restrict__ dst, int64_t ldd) {
  pdl_wait();
  pdl_trigger();
  pack_tile(rows, cols, src, lds, dst, ldd, blockIdx.x, blockIdx.y);
}

// Grouped column-panel packs (batched factorization): the CTAs walk the
// concatenated 64 x 64 tile lists of the tasks.
struct PackTask {
  const uint16_t* src;
  int64_t lds;
  uint16_t* dst;
  int64_t ldd;
  int64_t rows;
  int cols, tile_begin;
};
__global__ void __launch_bounds__(256) pack_grouped_kernel(const PackTask* __restrict__ tasks, int ntasks) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x;
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  const PackTask& k = tasks[lo];
  const int lt = t - k.tile_begin;
  const int64_t tr = cdiv<int64_t>(k.rows, kPackT);
  pack_tile(k.rows, k.cols, k.src, k.lds, k.dst, k.ldd, lt % tr, (int)(lt / tr));
}

// W_s = st(-Linv_ss L_{s,0:s}) into the first ws columns of the row-major
// operand Aop (row p, column q), fp32 accumulation over t ascending:
//   W[p][q] = -sum_t Linv[p][t] * L(s0 + t, k + q)
// Linv is Aop[p * ld + ws + t]; L(s0+t, k+q) = Lsub[t + q * ldlu].  Both runs
// of 128 values are contiguous and 16-byte aligned: loaded as 16-byte vectors
// before the multiply-adds.
__global__ void __launch_bounds__(128) make_w_kernel(int ws, uint16_t* aop, int64_t ld,
                                                     const uint16_t* __restrict__ Lsub, int64_t ldlu, int fmt) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (q >= ws) return;
  const uint4* li = reinterpret_cast<const uint4*>(aop + (int64_t)p * ld + ws);
  const uint4* lc = reinterpret_cast<const uint4*>(Lsub + (int64_t)q * ldlu);
  uint4 lv[16], cv[16];
#pragma unroll
  for (int k8 = 0; k8 < 16; ++k8) { lv[k8] = li[k8]; cv[k8] = lc[k8]; }
  float acc = 0.0f;
#pragma unroll
  for (int k8 = 0; k8 < 16; ++k8) {
    const uint32_t lw[4] = {lv[k8].x, lv[k8].y, lv[k8].z, lv[k8].w};
    const uint32_t cw[4] = {cv[k8].x, cv[k8].y, cv[k8].z, cv[k8].w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const uint16_t a16 = (uint16_t)(lw[h >> 1] >> ((h & 1) * 16));
      const uint16_t c16 = (uint16_t)(cw[h >> 1] >> ((h & 1) * 16));
      acc = __fmaf_rn(u16_to_f32(a16, fmt), u16_to_f32(c16, fmt), acc);
    }
  }
  aop[(int64_t)p * ld + q] = f32_to_u16(-acc, fmt);
}

// Z_s^T into the first zs columns of the row-major operand Bop (row p, column q):
//   Z[q][p] = -sum_t U(k + q, s0 + t) * Uinv[t][p]
// Uinv[t][p] = Bop[p * ld + zs + t] (contiguous, vector loads); U(k+q, s0+t) =
// Usub[q + t * ldlu] (coalesced across q), loaded 32 at a time before use.
__global__ void __launch_bounds__(128) make_z_kernel(int zs, uint16_t* bop, int64_t ld,
                                                     const uint16_t* __restrict__ Usub, int64_t ldlu, int fmt) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (q >= zs) return;
  const uint4* ui = reinterpret_cast<const uint4*>(bop + (int64_t)p * ld + zs);
  float acc = 0.0f;
#pragma unroll
  for (int t0 = 0; t0 < kB; t0 += 32) {
    uint16_t uv[32];
    uint4 iv[4];
#pragma unroll
    for (int u = 0; u < 32; ++u) uv[u] = Usub[q + (int64_t)(t0 + u) * ldlu];
#pragma unroll
    for (int k8 = 0; k8 < 4; ++k8) iv[k8] = ui[t0 / 8 + k8];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const uint32_t w = (u >> 3) == 0 ? (&iv[0].x)[(u & 7) >> 1]
                       : (u >> 3) == 1 ? (&iv[1].x)[(u & 7) >> 1]
                       : (u >> 3) == 2 ? (&iv[2].x)[(u & 7) >> 1] : (&iv[3].x)[(u & 7) >> 1];
      const uint16_t i16 = (uint16_t)(w >> ((u & 1) * 16));
      acc = __fmaf_rn(u16_to_f32(uv[u], fmt), u16_to_f32(i16, fmt), acc);
    }
  }
  bop[(int64_t)p * ld + q] = f32_to_u16(-acc, fmt);
}

// ---------------------------------------------------------------------------
// SIMT validation engine: the same products as the tensor-core engine with
// one fp32 fused multiply-add per term in ascending k (the oracle's order), so
// a factorization run on it is bit-identical to the oracle.  64 x 64 tiles,
// 256 threads, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
__device__ inline float e4m3_to_f32(uint8_t v) {
  const uint32_t s = (uint32_t)(v >> 7), e = (v >> 3) & 15, m = v & 7;
  float f;
  if (e == 0) f = (float)m * 0x1p-9f;                        // subnormal: m/8 * 2^-6
  else if (e == 15 && m == 7) f = __uint_as_float(0x7fc00000u);
  else f = __uint_as_float(((e + 120u) << 23) | (m << 20));  // (1 + m/8) 2^(e-7)
  return s ? -f : f;
}

// One CTA computes sub_m x sub_n tiles of 64 x 64 (sub_m = 2 when 64 < M <=
// 128, sub_n likewise): the panel products write their result over an operand
// (U12 over the B rows it reads, the row-major L21 copy over the A columns it
// reads), so a CTA must cover the whole 128-wide dimension and finish reading
// before it writes.  Each output's accumulation is the same in every case.
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmArgs g, int sub_m, int sub_n) {
  __shared__ float As[64][33], Bs[64][33];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t mb = (int64_t)blockIdx.y * 64 * sub_m, nb = (int64_t)blockIdx.x * 64 * sub_n;
  float acc[4][4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t >= sub_m * sub_n) break;
    const int64_t m0 = mb + 64 * (t % sub_m), n0 = nb + 64 * (t / sub_m);
    float accg[4][4];
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) acc[t][a][c] = 0.0f;
    for (int k0 = 0; k0 < g.K; k0 += 32) {
      if (g.fp8 && (k0 % 128) == 0) {
        for (int a = 0; a < 4; ++a)
          for (int c = 0; c < 4; ++c) accg[a][c] = 0.0f;
      }
      for (int idx = tid; idx < 64 * 32; idx += 256) {
        const int r = idx / 32, kk = idx % 32;
        const int64_t i = m0 + r, j = n0 + r;
        float av = 0.0f, bv = 0.0f;
        if (g.fp8) {
          if (i < g.M) av = e4m3_to_f32(((const uint8_t*)g.A)[i * g.lda + k0 + kk]);
          if (j < g.N) bv = e4m3_to_f32(((const uint8_t*)g.B)[j * g.ldb + k0 + kk]);
        } else {
          if (i < g.M) av = u16_to_f32(((const uint16_t*)g.A)[i * g.lda + k0 + kk], g.fmt);
          if (j < g.N) bv = u16_to_f32(((const uint16_t*)g.B)[j * g.ldb + k0 + kk], g.fmt);
        }
        As[r][kk] = av;
        Bs[r][kk] = bv;
      }
      __syncthreads();
      for (int kk = 0; kk < 32; ++kk)
        for (int a = 0; a < 4; ++a)
          for (int c = 0; c < 4; ++c) {
            if (g.fp8) accg[a][c] = __fmaf_rn(As[ty * 4 + a][kk], Bs[tx * 4 + c][kk], accg[a][c]);
            else acc[t][a][c] = __fmaf_rn(As[ty * 4 + a][kk], Bs[tx * 4 + c][kk], acc[t][a][c]);
          }
      __syncthreads();
      if (g.fp8 && ((k0 + 32) % 128) == 0) {
        const int kb = k0 / 128;
        for (int a = 0; a < 4; ++a)
          for (int c = 0; c < 4; ++c) {
            const int64_t i = min(m0 + ty * 4 + a, (int64_t)g.M - 1), j = min(n0 + tx * 4 + c, (int64_t)g.N - 1);
            const float sc = __fmul_rn(g.sA[(i / 128) * g.sa_ld + kb], g.sB[(j / 128) * g.sb_ld + kb]);
            acc[t][a][c] = __fmaf_rn(accg[a][c], sc, acc[t][a][c]);
          }
      }
    }
  }
  // every read of this CTA's operands is done (the loop ends on a barrier)
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t >= sub_m * sub_n) break;
    const int64_t m0 = mb + 64 * (t % sub_m), n0 = nb + 64 * (t / sub_m);
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        const int64_t i = m0 + ty * 4 + a, j = n0 + tx * 4 + c;
        if (i >= g.M || j >= g.N) continue;
        if (g.c32) {   // fp32 trailing matrix: one fp32 subtraction, no rounding to 16 bits
          float* cf = (float*)g.C + i + j * g.ldc;
          *cf = __fsub_rn(*cf, acc[t][a][c]);
          continue;
        }
        uint16_t* cp = g.C ? (uint16_t*)g.C + i + j * g.ldc : nullptr;
        float v;
        if (g.mode == kEpiSub) v = __fsub_rn(u16_to_f32(*cp, g.fmt), acc[t][a][c]);
        else v = g.sign * acc[t][a][c];
        const uint16_t h = f32_to_u16(v, g.fmt);
        if (cp) *cp = h;
        if (g.R) ((uint16_t*)g.R)[i * g.ldr + j] = h;
      }
  }
}

// ---------------------------------------------------------------------------
// FP8 variant of the Schur update (config with E4M3 operands): quantize the
// column panel (row-major, rows x b) and the row panel (column-major b x cols
// in the factor array) per 128 x 128 tile: s = fl32(amax / 448) (1 when the
// tile is zero), q = E4M3_satfinite(fl32(x / s)).  Outputs are K-major bytes:
// Lq[i * ldq + p], Uq[j * ldq + p], scales sL[(i/128) * ng + g], sU[(j/128) * ng + g].
// One CTA per tile.
// ---------------------------------------------------------------------------
__device__ inline uint8_t f32_to_e4m3_sat(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

__global__ void __launch_bounds__(256) quant_tile_kernel(const uint16_t* __restrict__ src, int64_t lds,
                                                        int rowmajor, int64_t rows, int b, int fmt,
                                                        uint8_t* __restrict__ q, int64_t ldq, float* scale,
                                                        int ng) {
  const int64_t a = blockIdx.x;   // 128-row (or column) tile of the long side
  const int gk = blockIdx.y;      // 128-deep slice
  const int tid = threadIdx.x;
  __shared__ float red[256];
  float amax = 0.0f;
  for (int idx = tid; idx < kB * kB; idx += 256) {
    const int64_t x = a * kB + idx / kB;
    const int p = gk * kB + idx % kB;
    if (x < rows && p < b) {
      const uint16_t h = rowmajor ? src[x * lds + p] : src[p + x * lds];
      amax = fmaxf(amax, fabsf(u16_to_f32(h, fmt)));
    }
  }
  red[tid] = amax;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) red[tid] = fmaxf(red[tid], red[tid + s]);
    __syncthreads();
  }
  amax = red[0];
  const float sc = amax == 0.0f ? 1.0f : __fdiv_rn(amax, 448.0f);
  for (int idx = tid; idx < kB * kB; idx += 256) {
    const int64_t x = a * kB + idx / kB;
    const int p = gk * kB + idx % kB;
    if (x < rows && p < b) {
      const uint16_t h = rowmajor ? src[x * lds + p] : src[p + x * lds];
      q[x * ldq + p] = f32_to_e4m3_sat(__fdiv_rn(u16_to_f32(h, fmt), sc));
    }
  }
  if (tid == 0) scale[a * ng + gk] = sc;
}

// ---------------------------------------------------------------------------
// Workspace layout of the factorization (all offsets 256-byte aligned).
// ---------------------------------------------------------------------------
struct FactorWs {
  uint32_t* status;
  uint16_t* Lp[2];   // packed column panel, row major, n x NB, by step parity
  uint16_t* Li;      // packed inner column panel, row major, NB x 128
  uint16_t* Aop[2];  // 4 row-panel operands [W_s | Linv_ss], 128 x NB each, by step parity
  uint16_t* Bop[2];  // 4 column-panel operands [Z_s^T | Uinv_ss^T], 128 x NB each, by step parity
  uint8_t* Lq[2];    // fp8 column panel, n x NB bytes, by step parity
  uint8_t* Uq[2];    // fp8 row panel, n x NB bytes (K-major per column)
  float* sL[2];      // fp8 scales, (n/128) x 4
  float* sU[2];
  float* W32;        // fp32 trailing matrix (TRAIL32 precisions), ld = ldw
  int64_t ldw;
  size_t bytes;
};

FactorWs carve(void* base, int64_t n, int prec, int NB) {
  FactorWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? (char*)base + off : nullptr;
    off += round_up<size_t>(bytes, 256);
    return p;
  };
  const int64_t nr = round_up<int64_t>(n, kB);
  w.status = (uint32_t*)take(256);
  for (int q = 0; q < 2; ++q) w.Lp[q] = (uint16_t*)take(sizeof(uint16_t) * nr * NB);
  w.Li = (uint16_t*)take(sizeof(uint16_t) * (size_t)NB * kB);
  for (int q = 0; q < 2; ++q) {
    w.Aop[q] = (uint16_t*)take(sizeof(uint16_t) * 4 * kB * NB);
    w.Bop[q] = (uint16_t*)take(sizeof(uint16_t) * 4 * kB * NB);
  }
  if (prec == HPMXP_FP8_E4M3) {
    for (int q = 0; q < 2; ++q) {
      w.Lq[q] = (uint8_t*)take((size_t)nr * NB);
      w.Uq[q] = (uint8_t*)take((size_t)nr * NB);
      w.sL[q] = (float*)take(sizeof(float) * (nr / kB) * 4);
      w.sU[q] = (float*)take(sizeof(float) * (nr / kB) * 4);
    }
  }
  if (trail32_of(prec)) {
    w.ldw = round_up<int64_t>(n, 8);
    w.W32 = (float*)take(sizeof(float) * (size_t)w.ldw * (size_t)n);
  }
  w.bytes = off;
  return w;
}

struct Factorizer {
  int64_t n;
  uint16_t* LU;
  int64_t ld;
  int fmt, prec, NB, engine;
  bool trail32 = false;   // Schur updates into the fp32 matrix w.W32; panels rounded from it

  // TRAIL32: block column [k, n) x [k, k+b) and block row [k, k+b) x [k+b, n)
  // of the fp32 matrix take their one rounding into the factor array
  void round_panel(int64_t k, int64_t b) {
    const float* W = w.W32;
    const int64_t ldw = w.ldw;
    round32_kernel<<<dim3((unsigned)cdiv<int64_t>(n - k, 256), (unsigned)std::min<int64_t>(b, 65535)), 256, 0, st>>>(
        n - k, b, W + k + k * ldw, ldw, at(k, k), ld, fmt);
    if (n - k - b > 0)
      round32_kernel<<<dim3((unsigned)cdiv<int64_t>(b, 256), (unsigned)std::min<int64_t>(n - k - b, 1024)), 256, 0,
                       st>>>(b, n - k - b, W + k + (k + b) * ldw, ldw, at(k, k + b), ld, fmt);
    count_launches(2);
    check(cudaGetLastError());
  }
  FactorWs w;
  cudaStream_t st;
  cudaError_t err = cudaSuccess;

  uint16_t* at(int64_t i, int64_t j) const { return LU + i + j * ld; }
  // the substitution operands of the current step's diagonal block (double
  // buffered by step parity: the look-ahead schedule's tail panels of step k
  // still read them while step k+1's diagonal block writes its own)
  int par = 0;
  uint16_t* aop(int s) const { return w.Aop[par] + (size_t)s * kB * NB; }
  uint16_t* bop(int s) const { return w.Bop[par] + (size_t)s * kB * NB; }

  void check(cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; }

  void gemm(GemmArgs g) {
    if (g.M <= 0 || g.N <= 0) return;
    g.fmt = fmt;
    g.status = w.status;
    check(engine == 1 ? gemm_simt(g, st) : gemm_tc(g, st));
  }

  // LU of the diagonal sub-block at (k, k), then its inverses (two CTAs)
  void getrf_base(int64_t k, int b, int slot) {
    void* tok = prof_begin(st);
    check(launch_pdl(getrf_lu_kernel, dim3(1), dim3(kGetrfThreads), kLuSmem, st, b, at(k, k), ld, fmt, w.status));
    check(launch_pdl(getrf_inv_kernel, dim3(2), dim3(kGetrfThreads), kInvSmem, st, b, (const uint16_t*)at(k, k), ld,
                     fmt, aop(slot) + slot * kB, NB, bop(slot) + slot * kB, NB));
    prof_end(tok, kProfGetrf, (double)b * b * b * 2.0, st);
    count_launches(2);
  }

  void pack(int64_t rows, int cols, const uint16_t* src, uint16_t* dst, int64_t ldd) {
    if (rows <= 0) return;
    dim3 grid((unsigned)cdiv<int64_t>(rows, kPackT), (unsigned)cdiv(cols, kPackT));
    void* tok = prof_begin(st);
    check(launch_pdl(pack_rows_kernel, grid, dim3(256), 0, st, rows, cols, src, ld, dst, ldd));
    prof_end(tok, kProfPanel, 4.0 * (double)rows * cols, st);
    count_launches(1);
  }

  // W_s = st(-Linv_ss L_{s,0:s}) and Z_s = st(-U_{0:s,s} Uinv_ss) of the
  // diagonal block at k (sub-block s > 0): they need only sub-block s's
  // inverses and the factors left of / above it, all final once getrf(s) ran.
  void make_w(int64_t k, int s) {
    const int64_t s0 = k + (int64_t)s * kB;
    void* tok = prof_begin(st);
    check(launch_pdl(make_w_kernel, dim3((unsigned)cdiv(s * kB, 128), kB), dim3(128), 0, st, s * kB, aop(s), NB,
                     (const uint16_t*)at(s0, k), ld, fmt));
    prof_end(tok, kProfPanel, 2.0 * s * kB * kB * kB, st);
    count_launches(1);
  }
  void make_z(int64_t k, int s) {
    const int64_t s0 = k + (int64_t)s * kB;
    void* tok = prof_begin(st);
    check(launch_pdl(make_z_kernel, dim3((unsigned)cdiv(s * kB, 128), kB), dim3(128), 0, st, s * kB, bop(s), NB,
                     (const uint16_t*)at(k, s0), ld, fmt));
    prof_end(tok, kProfPanel, 2.0 * s * kB * kB * kB, st);
    count_launches(1);
  }

  // Panels and Schur update of one sub-step inside a diagonal block wider than
  // 128: sub-block at kk (width 128) of the block ending at e.
  void inner_step(int64_t kk, int slot, int64_t e, int max_ctas) {
    const int64_t m = e - (kk + kB);
    if (m <= 0) return;
    GemmArgs u{};   // U12 = st(Linv A12), in place
    u.M = kB; u.N = (int)m; u.K = kB;
    u.A = aop(slot) + slot * kB; u.lda = NB;
    u.B = at(kk, kk + kB); u.ldb = ld;
    u.C = at(kk, kk + kB); u.ldc = ld;
    u.mode = kEpiStore; u.sign = 1.0f;
    u.max_ctas = max_ctas;
    fork();
    gemm(u);
    on_st3([&] {
      pack(m, kB, at(kk + kB, kk), w.Li, kB);
      GemmArgs l{};   // L21 = st(A21 Uinv): column major into LU, row major over the packed copy
      l.M = (int)m; l.N = kB; l.K = kB;
      l.A = w.Li; l.lda = kB;
      l.B = bop(slot) + slot * kB; l.ldb = NB;
      l.C = at(kk + kB, kk); l.ldc = ld;
      l.R = w.Li; l.ldr = kB;
      l.mode = kEpiStore; l.sign = 1.0f;
      l.max_ctas = max_ctas;
      gemm(l);
    });
    join();
    GemmArgs t{};   // A22 <- st(A22 - L21 U12)
    t.M = (int)m; t.N = (int)m; t.K = kB;
    t.A = w.Li; t.lda = kB;
    t.B = at(kk, kk + kB); t.ldb = ld;
    t.C = at(kk + kB, kk + kB); t.ldc = ld;
    t.mode = kEpiSub;
    t.max_ctas = max_ctas;
    gemm(t);
  }

  // Side streams of the look-ahead schedule (run_lookahead) and their events
  cudaStream_t st2 = nullptr, st4 = nullptr;
  cudaEvent_t evP = nullptr, evF = nullptr, evD = nullptr, evT = nullptr;
  int reserve = 0, sms = 0;
  // The row-panel (U12) and column-panel (L21) substitution chains depend on
  // nothing of each other: with a third stream the L21 chain runs on st3
  // between a fork and a join on `st`.
  cudaStream_t st3 = nullptr;
  cudaEvent_t evS = nullptr, evJ = nullptr;
  // W_s / Z_s run on their own lowest-priority stream: their CTAs must not
  // take the SMs the chain's GEMMs are waiting for
  cudaStream_t stw = nullptr;
  cudaEvent_t evW = nullptr, evW2 = nullptr;
  bool w_pending = false;
  void make_wz(int64_t k, int s) {
    if (!stw || !st3) { on_st3([&] { make_w(k, s); make_z(k, s); }); return; }
    check(cudaEventRecord(evW2, st3));   // after this sub-block's inner step (and so its getrf)
    check(cudaStreamWaitEvent(stw, evW2, 0));
    cudaStream_t keep = st;
    st = stw;
    make_w(k, s);
    make_z(k, s);
    st = keep;
    w_pending = true;
  }
  void join_wz() {   // the chains may use every W_s / Z_s made so far
    if (!w_pending) return;
    check(cudaEventRecord(evW, stw));
    check(cudaStreamWaitEvent(st, evW, 0));
    w_pending = false;
  }
  void fork() {
    if (!st3) return;
    check(cudaEventRecord(evS, st));
    check(cudaStreamWaitEvent(st3, evS, 0));
  }
  void join() {
    if (!st3) return;
    check(cudaEventRecord(evJ, st3));
    check(cudaStreamWaitEvent(st, evJ, 0));
  }
  template <class F>
  void on_st3(F&& f) {
    if (!st3) { f(); return; }
    cudaStream_t keep = st;
    st = st3;
    f();
    st = keep;
  }
  int64_t overlap_min = 8192;   // look-ahead only when the first step's trailing part is this wide

  // Diagonal block of step k (width b): getrf of each 128 sub-block and the
  // inner steps between them; beside it on stw the W_s / Z_s of the middle
  // sub-blocks (the last sub-block's are made by the caller).
  void diagonal_block(int64_t k, int64_t b, int64_t m, int panel_ctas) {
    const int nsub = (int)cdiv<int64_t>(b, kB);
    for (int s = 0; s < nsub; ++s) {
      const int64_t kk = k + (int64_t)s * kB;
      getrf_base(kk, (int)std::min<int64_t>(kB, k + b - kk), s);
      if (nsub > 1 && s + 1 < nsub) {
        inner_step(kk, s, k + b, panel_ctas);
        if (s > 0 && m > 0) make_wz(k, s);   // they feed only the panel chains
      }
    }
  }

  // One row-panel (U12 = [W_s | Linv_ss] [U12_{0:s}; A12_s]) and one
  // column-panel product of sub-block s, over columns [c0, c0 + N) of the
  // block row and rows [r0, r0 + M) of the block column (offsets from k + b).
  void u_panel(int64_t k, int64_t b, int s, int64_t c0, int64_t N, int max_ctas) {
    GemmArgs u{};
    u.M = kB; u.N = (int)N; u.K = (s + 1) * kB;
    u.A = aop(s); u.lda = NB;
    u.B = at(k, k + b + c0); u.ldb = ld;
    u.C = at(k + (int64_t)s * kB, k + b + c0); u.ldc = ld;
    u.mode = kEpiStore; u.sign = 1.0f;
    u.max_ctas = max_ctas;
    gemm(u);
  }
  void l_panel(int64_t k, int64_t b, int s, uint16_t* Lp, int64_t r0, int64_t M, int max_ctas) {
    GemmArgs l{};   // L21 column major into LU, row major over the packed copy
    l.M = (int)M; l.N = kB; l.K = (s + 1) * kB;
    l.A = Lp + r0 * NB; l.lda = NB;
    l.B = bop(s); l.ldb = NB;
    l.C = at(k + b + r0, k + (int64_t)s * kB); l.ldc = ld;
    l.R = Lp + r0 * NB + (int64_t)s * kB; l.ldr = NB;
    l.mode = kEpiStore; l.sign = 1.0f;
    l.max_ctas = max_ctas;
    gemm(l);
  }

  // FP8: per-tile E4M3 copies and scales of L21 rows [r0, r0 + M) and of U12
  // columns [c0, c0 + N) (tiles never straddle r0 or c0, multiples of 128)
  void quant_rows(int64_t b, int par_, const uint16_t* Lp, int64_t r0, int64_t M) {
    if (M <= 0) return;
    quant_tile_kernel<<<dim3((unsigned)cdiv<int64_t>(M, kB), (unsigned)cdiv<int64_t>(b, kB)), 256, 0, st>>>(
        Lp + r0 * NB, NB, 1, M, (int)b, fmt, w.Lq[par_] + r0 * NB, NB, w.sL[par_] + (r0 / kB) * 4, 4);
    count_launches(1);
    check(cudaGetLastError());
  }
  void quant_cols(int64_t k, int64_t b, int par_, int64_t c0, int64_t N) {
    if (N <= 0) return;
    quant_tile_kernel<<<dim3((unsigned)cdiv<int64_t>(N, kB), (unsigned)cdiv<int64_t>(b, kB)), 256, 0, st>>>(
        at(k, k + b + c0), ld, 0, N, (int)b, fmt, w.Uq[par_] + c0 * NB, NB, w.sU[par_] + (c0 / kB) * 4, 4);
    count_launches(1);
    check(cudaGetLastError());
  }

  // Schur update of step k (depth b) on rows [r0, r0 + M) x columns [c0, c0 + N)
  // of the trailing matrix (offsets from k + b): A22 <- st(A22 - L21 U12)
  void schur_part(int64_t k, int64_t b, int par_, const uint16_t* Lp, int64_t r0, int64_t M, int64_t c0,
                  int64_t N, int max_ctas) {
    if (M <= 0 || N <= 0) return;
    GemmArgs g{};
    g.M = (int)M; g.N = (int)N; g.K = (int)b;
    g.mode = kEpiSub;
    if (prec == HPMXP_FP8_E4M3) {
      g.fp8 = 1;
      g.lda = NB; g.ldb = NB;
      g.sa_ld = 4; g.sb_ld = 4;
      g.A = w.Lq[par_] + r0 * NB; g.B = w.Uq[par_] + c0 * NB;
      g.sA = w.sL[par_] + (r0 / kB) * 4; g.sB = w.sU[par_] + (c0 / kB) * 4;
    } else {
      g.lda = NB; g.ldb = ld;
      g.A = Lp + r0 * NB; g.B = at(k, k + b + c0);
    }
    if (trail32) {   // into the fp32 matrix, no rounding to 16 bits
      g.C = w.W32 + (k + b + r0) + (k + b + c0) * w.ldw;
      g.ldc = w.ldw;
      g.c32 = 1;
    } else {
      g.C = at(k + b + r0, k + b + c0);
      g.ldc = ld;
    }
    g.max_ctas = max_ctas;
    gemm(g);
  }

  template <class F>
  void on_st2(F&& f) {
    cudaStream_t keep = st;
    st = st2;
    f();
    st = keep;
  }

  void run() {
    if (st2) { run_lookahead(); return; }
    int step = 0;
    for (int64_t k = 0; k < n && err == cudaSuccess; k += NB, ++step) {
      const int64_t b = std::min<int64_t>(NB, n - k);
      const int nsub = (int)cdiv<int64_t>(b, kB);
      par = step & 1;
      uint16_t* Lp = w.Lp[par];
      const int64_t m = n - (k + b);
      if (trail32) round_panel(k, b);
      diagonal_block(k, b, m, 0);
      if (m <= 0) break;
      // row panel U12 (on st) and column panel L21 (on st3 when there is one),
      // block substitution over s; the chains meet before the update.  The
      // last sub-block's W_s / Z_s head its own chain's last product.
      join();
      join_wz();
      fork();
      on_st3([&] { pack(m, (int)b, at(k + b, k), Lp, NB); });
      for (int s = 0; s < nsub; ++s) {
        if (s > 0 && s == nsub - 1) make_w(k, s);
        u_panel(k, b, s, 0, m, 0);
        on_st3([&] {
          if (s > 0 && s == nsub - 1) make_z(k, s);
          l_panel(k, b, s, Lp, 0, m, 0);
        });
      }
      join();
      if (prec == HPMXP_FP8_E4M3) {
        quant_rows(b, par, Lp, 0, m);
        quant_cols(k, b, par, 0, m);
      }
      schur_part(k, b, par, Lp, 0, m, 0, m, 0);
    }
    join_wz();
  }

  // Look-ahead schedule.  The critical path of step k is the diagonal block,
  // then the "head" of the panels (the U12 columns and L21 rows of the next
  // diagonal block, b1 = min(NB, m) wide), then the update of the next
  // diagonal block alone, all on `st` (with the L21 head on st3).  The rest
  // runs beside it: the panels' "tail" (columns / rows past b1) on st4 as
  // soon as the diagonal block's operands exist (beside step k-1's far part
  // on st2), then on st2 the rest of the next block row and column ("near",
  // recorded as evN: step k+1's panels read it) and the far part of the
  // update (recorded as evF: step k+1's next-diagonal update reads it).  The
  // side streams' grids are held `reserve` SMs below the SM count, so the
  // critical chain always finds free SMs.  The packed L21 rows, the FP8
  // copies and the substitution operands read off the critical path are
  // double buffered by step parity: a buffer of parity p is written again two
  // steps later, after `st` has waited for evF of the step between, which
  // st2 records only after it has waited for that step's tails (evT).
  cudaEvent_t evN = nullptr;
  void run_lookahead() {
    const int cap = std::max(1, sms - reserve);
    bool prev = false;   // st2 holds work of the previous step (evN, evF recorded)
    int step = 0;
    for (int64_t k = 0; k < n && err == cudaSuccess; k += NB, ++step) {
      const int64_t b = std::min<int64_t>(NB, n - k);
      const int nsub = (int)cdiv<int64_t>(b, kB);
      par = step & 1;
      uint16_t* Lp = w.Lp[par];
      const int64_t m = n - (k + b);
      // (i) diagonal block k: updated in full by step k-1's critical path
      diagonal_block(k, b, m, 0);
      if (m <= 0) break;
      join();
      join_wz();
      if (nsub > 1) {   // the last sub-block's W_s / Z_s, read by head and tail
        fork();
        make_w(k, nsub - 1);
        on_st3([&] { make_z(k, nsub - 1); });
        join();
      }
      // block row / column k, written by step k-1's near part
      if (prev) check(cudaStreamWaitEvent(st, evN, 0));
      const int64_t b1 = std::min<int64_t>(NB, m), mt = m - b1;
      // (ii) tail of the panels on st4
      if (mt > 0) {
        check(cudaEventRecord(evD, st));
        check(cudaStreamWaitEvent(st4, evD, 0));
        cudaStream_t keep = st;
        st = st4;
        pack(mt, (int)b, at(k + b + b1, k), Lp + b1 * NB, NB);
        for (int s = 0; s < nsub; ++s) {
          u_panel(k, b, s, b1, mt, cap);
          l_panel(k, b, s, Lp, b1, mt, cap);
        }
        if (prec == HPMXP_FP8_E4M3) {
          quant_rows(b, par, Lp, b1, mt);
          quant_cols(k, b, par, b1, mt);
        }
        st = keep;
        check(cudaEventRecord(evT, st4));
      }
      // (iii) head of the panels
      fork();
      on_st3([&] { pack(b1, (int)b, at(k + b, k), Lp, NB); });
      for (int s = 0; s < nsub; ++s) {
        u_panel(k, b, s, 0, b1, 0);
        on_st3([&] { l_panel(k, b, s, Lp, 0, b1, 0); });
      }
      join();
      if (prec == HPMXP_FP8_E4M3) {
        quant_rows(b, par, Lp, 0, b1);
        quant_cols(k, b, par, 0, b1);
      }
      // (iv) the next diagonal block, after step k-1's far part (it lies there)
      if (prev) check(cudaStreamWaitEvent(st, evF, 0));
      if (mt > 0) check(cudaEventRecord(evP, st));   // heads (and their FP8 copies) done
      schur_part(k, b, par, Lp, 0, b1, 0, b1, 0);
      // (v) near and far parts on st2, after the heads and the tails
      if (mt > 0) {
        check(cudaStreamWaitEvent(st2, evP, 0));
        check(cudaStreamWaitEvent(st2, evT, 0));
        on_st2([&] {
          schur_part(k, b, par, Lp, b1, mt, 0, b1, cap);   // next block column below the diagonal block
          schur_part(k, b, par, Lp, 0, b1, b1, mt, cap);   // next block row right of it
          check(cudaEventRecord(evN, st2));
          schur_part(k, b, par, Lp, b1, mt, b1, mt, cap);  // far
          check(cudaEventRecord(evF, st2));
        });
        prev = true;
      } else {
        prev = false;   // nothing past the next diagonal block
      }
    }
    // every side-stream launch precedes the last event recorded on st2
    check(cudaEventRecord(evP, st2));
    check(cudaStreamWaitEvent(st, evP, 0));
    join_wz();
  }
};

}  // namespace

int gemm_engine() {
  const char* e = getenv("HPMXP_GEMM_ENGINE");
  return (e && strcmp(e, "simt") == 0) ? 1 : 0;
}

cudaError_t gemm_simt(const GemmArgs& g, cudaStream_t st) {
  const int sub_m = (g.M > 64 && g.M <= 128) ? 2 : 1, sub_n = (g.N > 64 && g.N <= 128) ? 2 : 1;
  dim3 grid((unsigned)cdiv(g.N, 64 * sub_n), (unsigned)cdiv(g.M, 64 * sub_m));
  gemm_simt_kernel<<<grid, 256, 0, st>>>(g, sub_m, sub_n);
  count_launches(1);
  return cudaGetLastError();
}

// Side stream and events of the look-ahead schedule, one set per device,
// created on first use and kept for the life of the process.
struct SideStream {
  std::mutex mu;   // one look-ahead factorization enqueues on this device at a time
  bool ok = false;
  cudaStream_t st = nullptr;    // near and far parts of the Schur update
  cudaStream_t st4 = nullptr;   // tails of the panels
  cudaStream_t st3 = nullptr;   // column-panel (L21) chain, beside the row-panel chain
  cudaStream_t stw = nullptr;   // W_s / Z_s of the diagonal block, lowest priority
  cudaEvent_t evP = nullptr, evF = nullptr, evN = nullptr, evD = nullptr, evT = nullptr, evS = nullptr,
              evJ = nullptr, evW = nullptr, evW2 = nullptr;
};

SideStream& side_stream(int dev) {
  static SideStream tab[64];
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  SideStream& s = tab[dev & 63];
  if (!s.ok) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&s.st, cudaStreamNonBlocking, lo) == cudaSuccess &&
        cudaStreamCreateWithPriority(&s.st3, cudaStreamNonBlocking, hi) == cudaSuccess &&
        cudaStreamCreateWithPriority(&s.stw, cudaStreamNonBlocking, lo) == cudaSuccess &&
        cudaStreamCreateWithPriority(&s.st4, cudaStreamNonBlocking, lo) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evD, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evT, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evW, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evW2, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evP, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evF, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evN, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evS, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&s.evJ, cudaEventDisableTiming) == cudaSuccess)
      s.ok = true;
  }
  return s;
}

cudaError_t launch_cast(int64_t n, const double* A, int64_t lda, void* out, int64_t ldo, int fmt, cudaStream_t st,
                        const double* rs, const double* cs) {
  void* tok = prof_begin(st);
  cast_kernel<<<dim3((unsigned)cdiv<int64_t>(n, kCastCols), (unsigned)cdiv<int64_t>(n, kCastRows)), 256, 0, st>>>(
      n, A, lda, (uint16_t*)out, ldo, fmt, rs, cs);
  prof_end(tok, kProfCast, 10.0 * (double)n * (double)n, st);
  count_launches(1);
  return cudaGetLastError();
}

size_t factor_ws_bytes(int64_t n, int prec, int nb) { return carve(nullptr, n, prec, nb).bytes; }

// ---------------------------------------------------------------------------
// Batched factorization: every system in lockstep at depth 128, one grouped
// launch per stage for all active systems.  Per step k (block width b = 128):
// getrf of each diagonal block (one CTA each), U12 = Linv A12 (grouped
// tcgen05, in place), pack of A21 (grouped), L21 = A21 Uinv with its
// row-major copy (grouped), A22 -= L21 U12 (grouped).  The same tiles as
// hpmxp_factor at nb = 128 without look-ahead, so the same bits.
// ---------------------------------------------------------------------------
namespace {
struct BatchLayout {
  uint32_t* status;        // count + 1 words: one per system, the last for the GEMM launches
  uint16_t** Lp;           // per system: packed column panel, row major, round_up(n, 128) x 128
  uint16_t** Aop;          // per system: Linv (K-major operand, 128 x 128)
  uint16_t** Bop;          // per system: Uinv^T
  GemmGroupItem* items;
  GetrfTask* getrf;
  PackTask* pack;
  size_t bytes;
};

struct BatchCounts { int64_t items = 0, getrf = 0, pack = 0; };

BatchCounts batch_counts(const hpmxp_problem* probs, int count) {
  BatchCounts c;
  for (int q = 0; q < count; ++q) {
    const int64_t steps = cdiv<int64_t>(probs[q].n, kB);
    c.getrf += steps;
    c.pack += steps - 1;
    c.items += 3 * (steps - 1);
  }
  return c;
}

BatchLayout carve_batch(void* base, const hpmxp_problem* probs, int count, std::vector<uint16_t*>* ptrs) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? (char*)base + off : nullptr;
    off += round_up<size_t>(bytes, 256);
    return p;
  };
  L.status = (uint32_t*)take(sizeof(uint32_t) * (count + 1));
  if (ptrs) ptrs->assign(3 * (size_t)count, nullptr);
  for (int q = 0; q < count; ++q) {
    const int64_t nr = round_up<int64_t>(probs[q].n, kB);
    uint16_t* lp = (uint16_t*)take(sizeof(uint16_t) * nr * kB);
    uint16_t* ao = (uint16_t*)take(sizeof(uint16_t) * kB * kB);
    uint16_t* bo = (uint16_t*)take(sizeof(uint16_t) * kB * kB);
    if (ptrs) { (*ptrs)[3 * q] = lp; (*ptrs)[3 * q + 1] = ao; (*ptrs)[3 * q + 2] = bo; }
  }
  const BatchCounts c = batch_counts(probs, count);
  L.items = (GemmGroupItem*)take(sizeof(GemmGroupItem) * std::max<int64_t>(c.items, 1));
  L.getrf = (GetrfTask*)take(sizeof(GetrfTask) * std::max<int64_t>(c.getrf, 1));
  L.pack = (PackTask*)take(sizeof(PackTask) * std::max<int64_t>(c.pack, 1));
  L.bytes = off;
  return L;
}
}  // namespace

size_t factor_batched_ws_bytes(const hpmxp_problem* probs, int count) {
  return carve_batch(nullptr, probs, count, nullptr).bytes;
}

hpmxp_status factor_batched(const hpmxp_problem* probs, int count, int prec, hpmxp_status* status_out, void* ws,
                            size_t ws_bytes, cudaStream_t st) {
  (void)ws_bytes;
  const int fmt = fmt_of(prec);
  std::vector<uint16_t*> ptr;
  const BatchLayout W = carve_batch(ws, probs, count, &ptr);
  int64_t nmax = 0;
  for (int q = 0; q < count; ++q) nmax = std::max(nmax, probs[q].n);
  const int64_t steps = cdiv<int64_t>(nmax, kB);
  const bool simt = gemm_engine() == 1;
  auto at = [&](int q, int64_t i, int64_t j) { return (uint16_t*)probs[q].LU + i + j * probs[q].ldlu; };

  // the whole plan, host side: per step the getrf tasks, pack tasks and the
  // three products' items, each step's part contiguous
  std::vector<GetrfTask> gt;
  std::vector<PackTask> pt;
  std::vector<GemmGroupItem> items;
  std::vector<GemmArgs> all_args;   // the products themselves (SIMT engine; flop counts)
  struct Step { int64_t g0, ng, p0, np, ptiles, u0, nu, tu, l0, nl, tl, s0, ns, ts; double fu, fl, fs; };
  std::vector<Step> plan(steps);
  GemmArgs proto{};
  proto.K = kB; proto.fmt = fmt; proto.status = W.status + count;
  for (int64_t s = 0; s < steps; ++s) {
    const int64_t k = s * kB;
    Step& S = plan[s];
    S = Step{};
    S.g0 = gt.size();
    for (int q = 0; q < count; ++q) {
      const int64_t n = probs[q].n;
      if (n <= k) continue;
      GetrfTask t{};
      t.b = (int)std::min<int64_t>(kB, n - k);
      t.D = at(q, k, k); t.ldd = probs[q].ldlu;
      t.linv = ptr[3 * q + 1]; t.ldl = kB;
      t.uinvT = ptr[3 * q + 2]; t.ldu = kB;
      t.status = W.status + q;
      gt.push_back(t);
    }
    S.ng = (int64_t)gt.size() - S.g0;
    // products of the systems with a trailing part
    std::vector<GemmArgs> U, Lg, Sg;
    S.p0 = pt.size();
    int ptiles = 0;
    for (int q = 0; q < count; ++q) {
      const int64_t n = probs[q].n, m = n - k - kB;
      if (m <= 0) continue;
      const int64_t ld = probs[q].ldlu;
      PackTask pk{};
      pk.src = at(q, k + kB, k); pk.lds = ld; pk.dst = ptr[3 * q]; pk.ldd = kB; pk.rows = m; pk.cols = kB;
      pk.tile_begin = ptiles;
      ptiles += (int)(cdiv<int64_t>(m, kPackT) * cdiv(kB, kPackT));
      pt.push_back(pk);
      GemmArgs u = proto;   // U12 = st(Linv A12), in place
      u.M = kB; u.N = (int)m; u.A = ptr[3 * q + 1]; u.lda = kB; u.B = at(q, k, k + kB); u.ldb = ld;
      u.C = at(q, k, k + kB); u.ldc = ld; u.mode = kEpiStore; u.sign = 1.0f;
      U.push_back(u);
      GemmArgs l = proto;   // L21 = st(A21 Uinv), column major into LU and row major over the packed copy
      l.M = (int)m; l.N = kB; l.A = ptr[3 * q]; l.lda = kB; l.B = ptr[3 * q + 2]; l.ldb = kB;
      l.C = at(q, k + kB, k); l.ldc = ld; l.R = ptr[3 * q]; l.ldr = kB; l.mode = kEpiStore; l.sign = 1.0f;
      Lg.push_back(l);
      GemmArgs t = proto;   // A22 <- st(A22 - L21 U12)
      t.M = (int)m; t.N = (int)m; t.A = ptr[3 * q]; t.lda = kB; t.B = at(q, k, k + kB); t.ldb = ld;
      t.C = at(q, k + kB, k + kB); t.ldc = ld; t.mode = kEpiSub;
      Sg.push_back(t);
    }
    S.np = (int64_t)pt.size() - S.p0;
    S.ptiles = ptiles;
    auto add = [&](std::vector<GemmArgs>& v, int64_t& first, int64_t& num, int64_t& tiles, double& flops) {
      first = items.size();
      num = v.size();
      tiles = 0;
      flops = 0.0;
      if (v.empty()) return true;
      items.resize(items.size() + v.size());
      int tt = 0;
      if (!gemm_group_encode(v.data(), (int)v.size(), items.data() + first, &tt)) return false;
      tiles = tt;
      for (const GemmArgs& g : v) flops += 2.0 * g.M * (double)g.N * g.K;
      all_args.insert(all_args.end(), v.begin(), v.end());
      return true;
    };
    if (!add(U, S.u0, S.nu, S.tu, S.fu) || !add(Lg, S.l0, S.nl, S.tl, S.fl) || !add(Sg, S.s0, S.ns, S.ts, S.fs))
      return HPMXP_EINVAL;
  }
  // one copy of the plan into the workspace
  cudaError_t e = cudaMemsetAsync(W.status, 0, sizeof(uint32_t) * (count + 1), st);
  if (e == cudaSuccess && !gt.empty())
    e = cudaMemcpyAsync(W.getrf, gt.data(), sizeof(GetrfTask) * gt.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !pt.empty())
    e = cudaMemcpyAsync(W.pack, pt.data(), sizeof(PackTask) * pt.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(W.items, items.data(), sizeof(GemmGroupItem) * items.size(), cudaMemcpyHostToDevice, st);
  for (int q = 0; q < count && e == cudaSuccess; ++q)
    e = launch_cast(probs[q].n, probs[q].A, probs[q].lda, probs[q].LU, probs[q].ldlu, fmt, st);
  static std::atomic<int> attr_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (e == cudaSuccess && attr_dev.load() != dev) {
    e = cudaFuncSetAttribute(getrf_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGetrfSmem);
    if (e == cudaSuccess) attr_dev.store(dev);
  }
  size_t ai = 0;   // index into all_args (SIMT engine)
  auto run_products = [&](int64_t first, int64_t num, int64_t tiles, double flops, const GemmArgs& kind) {
    if (num == 0 || e != cudaSuccess) return;
    if (simt) {
      for (int64_t c = 0; c < num && e == cudaSuccess; ++c) e = gemm_simt(all_args[ai + c], st);
    } else {
      double bytes = 0.0;
      for (int64_t c = 0; c < num; ++c) {
        const GemmArgs& g = all_args[ai + c];
        bytes += ((double)g.M + g.N) * g.K * 2.0 + (double)g.M * g.N * 2.0 * (kind.mode == kEpiSub ? 2.0 : 1.0) +
                 (g.R ? (double)g.M * g.N * 2.0 : 0.0);
      }
      e = gemm_tc_grouped(kind, W.items + first, (int)num, (int)tiles, st, flops, bytes);
    }
    ai += num;
  };
  for (int64_t s = 0; s < steps && e == cudaSuccess; ++s) {
    const Step& S = plan[s];
    void* tok = prof_begin(st);
    e = launch_pdl(getrf_grouped_kernel, dim3((unsigned)S.ng), dim3(kGetrfThreads), kGetrfSmem, st,
                   (const GetrfTask*)(W.getrf + S.g0), fmt);
    prof_end(tok, kProfGetrf, (double)S.ng * kB * kB * kB * 2.0, st);
    count_launches(1);
    if (S.np == 0) continue;
    GemmArgs ku = proto; ku.mode = kEpiStore; ku.sign = 1.0f;
    GemmArgs ks = proto; ks.mode = kEpiSub;
    run_products(S.u0, S.nu, S.tu, S.fu, ku);
    if (e == cudaSuccess) {
      void* tk = prof_begin(st);
      e = launch_pdl(pack_grouped_kernel, dim3((unsigned)S.ptiles), dim3(256), 0, st,
                     (const PackTask*)(W.pack + S.p0), (int)S.np);
      prof_end(tk, kProfPanel, 0.0, st);
      count_launches(1);
    }
    run_products(S.l0, S.nl, S.tl, S.fl, ku);
    run_products(S.s0, S.ns, S.ts, S.fs, ks);
  }
  if (e != cudaSuccess) return status_from_cuda(e);
  std::vector<uint32_t> words((size_t)count + 1);
  e = read_to_host(words.data(), W.status, sizeof(uint32_t) * (count + 1), st);
  if (e != cudaSuccess) return status_from_cuda(e);
  hpmxp_status first = status_from_word(words[count]);
  for (int q = 0; q < count; ++q) {
    const hpmxp_status sq = words[count] ? status_from_word(words[count]) : status_from_word(words[q]);
    if (status_out) status_out[q] = sq;
    if (first == HPMXP_OK) first = sq;
  }
  return first;
}

cudaError_t launch_balance(int64_t n, const double* A, int64_t lda, int prec, double* rs, double* cs,
                           cudaStream_t st) {
  void* tok = prof_begin(st);
  cudaError_t e = cudaMemsetAsync(rs, 0, sizeof(double) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  dim3 g1((unsigned)cdiv<int64_t>(n, kBalRows), (unsigned)cdiv<int64_t>(n, kBalChunk));
  row_absmax_kernel<<<g1, 256, 0, st>>>(n, A, lda, reinterpret_cast<unsigned long long*>(rs));
  row_scale_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, rs);
  col_scale_kernel<<<(unsigned)cdiv<int64_t>(n, kBalCols), 256, 0, st>>>(n, A, lda, rs, cs);
  const double s = fmt_of(prec) == kFP16 ? 4096.0 : 1.0;
  if (s != 1.0) {
    format_scale_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, rs, s);
    count_launches(1);
  }
  prof_end(tok, kProfBalance, 16.0 * (double)n * (double)n, st);
  count_launches(3);
  return cudaGetLastError();
}

hpmxp_status factor(int64_t n, const double* A, int64_t lda, int prec, int nb, void* LU,
                    int64_t ldlu, void* ws, size_t ws_bytes, cudaStream_t st, const double* rs,
                    const double* cs) {
  static std::atomic<int> attr_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev.load() != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(getrf_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLuSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(getrf_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvSmem);
    if (e != cudaSuccess) return status_from_cuda(e);
    attr_dev.store(dev);
  }
  Factorizer f;
  f.n = n; f.LU = (uint16_t*)LU; f.ld = ldlu;
  f.prec = prec; f.fmt = fmt_of(prec);
  f.trail32 = trail32_of(prec);
  f.NB = nb; f.engine = gemm_engine();
  f.w = carve(ws, n, prec, nb);
  f.st = st;
  f.check(cudaMemsetAsync(f.w.status, 0, sizeof(uint32_t), st));
  if (f.trail32) {
    void* tok = prof_begin(st);
    cast32_kernel<<<dim3((unsigned)n, (unsigned)cdiv<int64_t>(n, 256)), 256, 0, st>>>(n, A, lda, f.w.W32, f.w.ldw,
                                                                                      rs, cs);
    prof_end(tok, kProfCast, 12.0 * (double)n * (double)n, st);
    count_launches(1);
    f.check(cudaGetLastError());
  } else {
    f.check(launch_cast(n, A, lda, LU, ldlu, f.fmt, st, rs, cs));
  }
  const hpmxp_tuning tune = tuning();
  if (tune.overlap_min > 0) f.overlap_min = tune.overlap_min;
  // the largest far part is n - 2 nb (first step); below overlap_min the
  // schedule never uses the side stream, so it is not taken (concurrent
  // factorizations of small systems on other streams then do not serialize)
  std::unique_lock<std::mutex> lk;
  if (!f.trail32 && n - 2 * (int64_t)nb >= std::max<int64_t>(f.overlap_min, 1) &&
      getenv("HPMXP_NO_LOOKAHEAD") == nullptr) {
    SideStream& ss = side_stream(dev);
    if (ss.ok) {
      lk = std::unique_lock<std::mutex>(ss.mu);
      f.st2 = ss.st;
      f.st3 = ss.st3;
      f.evP = ss.evP;
      f.evF = ss.evF;
      f.evN = ss.evN;
      f.st4 = ss.st4;
      f.evD = ss.evD;
      f.evT = ss.evT;
      f.evS = ss.evS;
      f.evJ = ss.evJ;
      f.stw = ss.stw;
      f.evW = ss.evW;
      f.evW2 = ss.evW2;
      cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev);
      f.reserve = std::max(4, f.sms / 16);
      if (tune.reserve_sms > 0) f.reserve = std::max(1, std::min(f.sms - 1, tune.reserve_sms));
    }
  }
  f.run();
  if (lk.owns_lock()) lk.unlock();
  if (f.err != cudaSuccess) return status_from_cuda(f.err);
  uint32_t word = 0;
  cudaError_t e = read_to_host(&word, f.w.status, sizeof(word), st);
  if (e != cudaSuccess) return status_from_cuda(e);
  return status_from_word(word);
}

}  // namespace hpmxp
