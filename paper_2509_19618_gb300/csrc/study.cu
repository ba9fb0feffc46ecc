// FP64 LU without pivoting and its triangular solves, for the pivot-growth
// and residual-norm study of section "Experimental Results" (Figs. 2-4): the
// 64-bit factorization without pivoting whose largest pivot and residual
// norms the paper compares with partial pivoting.
//
// Right-looking, block width 64, fp64 storage and arithmetic, in the plain
// order of Fig. 1's algorithm: at every diagonal block D = [k, k+64)
//   (i)   D factored unblocked (l = a / pivot, then a -= l u by fused
//         multiply-add, pivots ascending) in shared memory, one CTA;
//   (ii)  U12 = L11^{-1} A12 by forward substitution, one thread per column,
//         terms t ascending; L21 = A21 U11^{-1} by substitution, one thread
//         per row, terms t ascending, then one division by u_cc;
//   (iii) A22 <- A22 - L21 U12, one fp64 accumulation per entry over the 64
//         terms in ascending order, then one subtraction (SIMT tiles: GB300's
//         fp64 rate is the bound, not the tensor cores, which have no
//         useful fp64 path on this part).
// The triangular solves go by 64-row blocks: the diagonal block by
// substitution in one CTA, then a fp64 GEMV of the solved block into the
// rows after it.
#include "internal.h"

#include <algorithm>

namespace hpmxp {
namespace {

constexpr int kQ = 64;        // block width
constexpr int kQP = kQ + 1;   // shared pitch (doubles)

// (i) the b x b diagonal block at D (b <= 64), 256 threads.
__global__ void __launch_bounds__(256) lu64_diag_kernel(int b, double* D, int64_t ld, uint32_t* status) {
  __shared__ double a[kQ * kQP];   // a[j * kQP + i]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < b * b; idx += 256) {
    const int i = idx % b, j = idx / b;
    a[j * kQP + i] = D[i + (int64_t)j * ld];
  }
  __syncthreads();
  for (int p = 0; p < b; ++p) {
    const double piv = a[p * kQP + p];
    if (tid == 0 && !(isfinite(piv) && piv != 0.0)) atomicOr(status, kErrPivot);
    for (int i = p + 1 + tid; i < b; i += 256) a[p * kQP + i] = a[p * kQP + i] / piv;
    __syncthreads();
    const int r = b - p - 1;
    for (int idx = tid; idx < r * r; idx += 256) {
      const int i = p + 1 + idx % r, j = p + 1 + idx / r;
      a[j * kQP + i] = __fma_rn(-a[p * kQP + i], a[j * kQP + p], a[j * kQP + i]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < b * b; idx += 256) {
    const int i = idx % b, j = idx / b;
    D[i + (int64_t)j * ld] = a[j * kQP + i];
  }
}

// (ii) U12 = L11^{-1} A12 for the m columns after the block: one thread per
// column, the column in registers.
__global__ void __launch_bounds__(128) lu64_row_panel_kernel(const double* __restrict__ L11, int64_t ld,
                                                             double* __restrict__ A12, int64_t m) {
  __shared__ double L[kQ * kQP];   // L[t * kQP + r] = L11(r, t)
  for (int idx = threadIdx.x; idx < kQ * kQ; idx += 128) {
    const int r = idx % kQ, t = idx / kQ;
    L[t * kQP + r] = L11[r + (int64_t)t * ld];
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (j >= m) return;
  double* col = A12 + j * ld;
  double x[kQ];
#pragma unroll
  for (int r = 0; r < kQ; ++r) x[r] = col[r];
#pragma unroll
  for (int r = 1; r < kQ; ++r) {
    double acc = x[r];
#pragma unroll
    for (int t = 0; t < r; ++t) acc = __fma_rn(-L[t * kQP + r], x[t], acc);
    x[r] = acc;
  }
#pragma unroll
  for (int r = 0; r < kQ; ++r) col[r] = x[r];
}

// (ii') L21 = A21 U11^{-1} for the m rows after the block: one thread per row
// (consecutive rows per warp: each column access is coalesced).
__global__ void __launch_bounds__(128) lu64_col_panel_kernel(const double* __restrict__ U11, int64_t ld,
                                                             double* __restrict__ A21, int64_t m) {
  __shared__ double U[kQ * kQP];   // U[c * kQP + t] = U11(t, c)
  for (int idx = threadIdx.x; idx < kQ * kQ; idx += 128) {
    const int t = idx % kQ, c = idx / kQ;
    U[c * kQP + t] = U11[t + (int64_t)c * ld];
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (i >= m) return;
  double y[kQ];
#pragma unroll
  for (int c = 0; c < kQ; ++c) y[c] = A21[i + (int64_t)c * ld];
#pragma unroll
  for (int c = 0; c < kQ; ++c) {
    double acc = y[c];
#pragma unroll
    for (int t = 0; t < c; ++t) acc = __fma_rn(-y[t], U[c * kQP + t], acc);
    y[c] = acc / U[c * kQP + c];
  }
#pragma unroll
  for (int c = 0; c < kQ; ++c) A21[i + (int64_t)c * ld] = y[c];
}

// (iii) C <- C - L U over an m x m trailing block, K = 64: 64 x 64 output
// tiles, 256 threads with 4 x 4 entries each (thread rows fastest, so every
// column access of a warp covers 64 consecutive rows).  The operands go
// through shared memory in two 32-deep halves; each entry's 64 terms are still
// accumulated in ascending order.
constexpr int kH = 32;
__global__ void __launch_bounds__(256) lu64_update_kernel(const double* __restrict__ Lp,
                                                          const double* __restrict__ Up, double* __restrict__ C,
                                                          int64_t ld, int64_t m) {
  __shared__ double Ls[kH * kQP];        // Ls[p * kQP + i] = L(i0 + i, h + p)
  __shared__ double Us[kQ * (kH + 1)];   // Us[j * (kH + 1) + p] = U(h + p, j0 + j)
  const int64_t i0 = (int64_t)blockIdx.x * kQ, j0 = (int64_t)blockIdx.y * kQ;
  const int tid = threadIdx.x;
  const int ti = (tid % 16) * 4, tj = (tid / 16) * 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  for (int h = 0; h < kQ; h += kH) {
    for (int idx = tid; idx < kQ * kH; idx += 256) {
      const int i = idx % kQ, p = idx / kQ;
      Ls[p * kQP + i] = i0 + i < m ? Lp[i0 + i + (int64_t)(h + p) * ld] : 0.0;
      const int pp = idx % kH, j = idx / kH;
      Us[j * (kH + 1) + pp] = j0 + j < m ? Up[h + pp + (j0 + j) * ld] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < kH; ++p) {
      double l[4], u[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) l[a] = Ls[p * kQP + ti + a];
#pragma unroll
      for (int c = 0; c < 4; ++c) u[c] = Us[(tj + c) * (kH + 1) + p];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = __fma_rn(l[a], u[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t j = j0 + tj + c;
    if (j >= m) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + ti + a;
      if (i < m) C[i + j * ld] = C[i + j * ld] - acc[a][c];
    }
  }
}

// Triangular solves, 64-row blocks.  Diagonal block: one CTA of 64 threads,
// one column of B per thread (nrhs <= 64); lower: unit diagonal, forward;
// upper: backward with one division per row.
template <bool kLower>
__global__ void __launch_bounds__(64) trsv64_diag_kernel(int b, const double* __restrict__ D, int64_t ld,
                                                         double* __restrict__ X, int64_t ldx, int64_t nrhs) {
  __shared__ double T[kQ * kQP];   // T[c * kQP + r] = D(r, c)
  for (int idx = threadIdx.x; idx < b * b; idx += 64) {
    const int r = idx % b, c = idx / b;
    T[c * kQP + r] = D[r + (int64_t)c * ld];
  }
  __syncthreads();
  const int64_t k = threadIdx.x;
  if (k >= nrhs) return;
  double* x = X + k * ldx;
  if (kLower) {
    for (int r = 1; r < b; ++r) {
      double acc = x[r];
      for (int t = 0; t < r; ++t) acc = __fma_rn(-T[t * kQP + r], x[t], acc);
      x[r] = acc;
    }
  } else {
    for (int r = b - 1; r >= 0; --r) {
      double acc = x[r];
      for (int t = r + 1; t < b; ++t) acc = __fma_rn(-T[t * kQP + r], x[t], acc);
      x[r] = acc / T[r * kQP + r];
    }
  }
}

// Y(rows) -= M(rows, 0:b) X(0:b) for `rows` rows (M column major), one thread
// per (row, rhs).
__global__ void __launch_bounds__(256) trsv64_update_kernel(int64_t rows, int b, const double* __restrict__ M,
                                                            int64_t ld, const double* __restrict__ X,
                                                            double* __restrict__ Y, int64_t ldx, int64_t nrhs) {
  const int64_t g = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (g >= rows * nrhs) return;
  const int64_t i = g % rows, k = g / rows;
  double acc = 0.0;
  for (int t = 0; t < b; ++t) acc = __fma_rn(M[i + (int64_t)t * ld], X[t + k * ldx], acc);
  Y[i + k * ldx] -= acc;
}

}  // namespace

cudaError_t lu_f64(int64_t n, double* A, int64_t ld, uint32_t* status, cudaStream_t st) {
  for (int64_t k = 0; k < n; k += kQ) {
    const int b = (int)std::min<int64_t>(kQ, n - k);
    double* D = A + k + k * ld;
    lu64_diag_kernel<<<1, 256, 0, st>>>(b, D, ld, status);
    count_launches(1);
    const int64_t m = n - k - b;
    if (m <= 0) break;
    const unsigned g = (unsigned)cdiv<int64_t>(m, 128);
    lu64_row_panel_kernel<<<g, 128, 0, st>>>(D, ld, D + b * ld, m);
    lu64_col_panel_kernel<<<g, 128, 0, st>>>(D, ld, D + b, m);
    const unsigned t = (unsigned)cdiv<int64_t>(m, kQ);
    lu64_update_kernel<<<dim3(t, t), 256, 0, st>>>(D + b, D + b * ld, D + b + b * ld, ld, m);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t lu_solve_f64(int64_t n, const double* LU, int64_t ld, double* X, int64_t ldx, int64_t nrhs,
                         cudaStream_t st) {
  const int64_t nb = cdiv<int64_t>(n, kQ);
  for (int64_t c = 0; c < nb; ++c) {   // forward: L y = b
    const int64_t r0 = c * kQ;
    const int b = (int)std::min<int64_t>(kQ, n - r0);
    trsv64_diag_kernel<true><<<1, 64, 0, st>>>(b, LU + r0 + r0 * ld, ld, X + r0, ldx, nrhs);
    const int64_t rows = n - r0 - b;
    if (rows > 0)
      trsv64_update_kernel<<<(unsigned)cdiv<int64_t>(rows * nrhs, 256), 256, 0, st>>>(
          rows, b, LU + r0 + b + r0 * ld, ld, X + r0, X + r0 + b, ldx, nrhs);
    count_launches(rows > 0 ? 2 : 1);
  }
  for (int64_t c = nb - 1; c >= 0; --c) {   // backward: U x = y
    const int64_t r0 = c * kQ;
    const int b = (int)std::min<int64_t>(kQ, n - r0);
    trsv64_diag_kernel<false><<<1, 64, 0, st>>>(b, LU + r0 + r0 * ld, ld, X + r0, ldx, nrhs);
    if (r0 > 0)
      trsv64_update_kernel<<<(unsigned)cdiv<int64_t>(r0 * nrhs, 256), 256, 0, st>>>(
          r0, b, LU + r0 * ld, ld, X + r0, X, ldx, nrhs);
    count_launches(r0 > 0 ? 2 : 1);
  }
  return cudaGetLastError();
}

}  // namespace hpmxp
