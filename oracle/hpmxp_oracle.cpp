// HPL-MxP CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, sequential restatement of what the solver path computes, used
// only by the tests, by the smoke check and by the benchmark's CPU-baseline
// leg.  It shares no code, header, table or constant generator with the CUDA
// library and must never be called from the product path.
//
// Every function cites the passage of the paper (Dongarra & Luszczek,
// "HPL-MxP Benchmark: Mixed-Precision Algorithms, Iterative Refinement, and
// Scalable Data Generation", arXiv 2509.19618) it restates.  Where the paper is
// silent, the reading used is stated next to the code.
//
// Precision conventions (section "Algorithmic Framework", Fig. 1):
//   * storage of the factors and of the trailing matrix: a low-precision format
//     (BF16, FP16) emulated by software round-to-nearest-even of an fp64 value;
//   * panel arithmetic (diagonal getrf, triangular inverses) in fp32;
//   * every product of two low-precision operands is accumulated in fp32 with
//     one fused multiply-add per term, terms taken in ascending index order;
//   * refinement (GMRES-IR) in fp64.
// Compile with -ffp-contract=off: every fused multiply-add here is explicit.
//
// Parity status of each function is listed in its comment; all are pinned by
// tests/test_oracle_*.py except where the comment says "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

namespace {

// ---------------------------------------------------------------------------
// Low-precision formats, rounding to nearest, ties to even (IEEE 754 2019,
// section 4.3.1).  A format is given by its significand width p (including the
// implicit bit), its smallest normal exponent emin and its largest finite
// value.  Overflow gives +-inf for the IEEE formats and saturates for OCP E4M3
// (which has no infinity).  Subnormals are handled by clamping the quantum.
// ---------------------------------------------------------------------------
enum Fmt { FMT_BF16 = 0, FMT_FP16 = 1, FMT_E4M3 = 2, FMT_FP32 = 3, FMT_FP64 = 4 };

struct FmtDesc {
  int p;          // significand bits including the implicit one
  int emin;       // exponent of the smallest normal number
  double maxval;  // largest finite value
  bool saturate;  // overflow saturates to maxval instead of giving infinity
};

FmtDesc fmt_desc(int f) {
  switch (f) {
    case FMT_BF16: return {8, -126, std::ldexp(255.0, 120), false};   // (2-2^-7)*2^127
    case FMT_FP16: return {11, -14, 65504.0, false};
    case FMT_E4M3: return {4, -6, 448.0, true};
    case FMT_FP32: return {24, -126, std::ldexp(16777215.0, 104), false};
    default: return {53, -1022, 0.0, false};
  }
}

double round_fmt(double x, int f) {
  if (f == FMT_FP64) return x;
  if (std::isnan(x)) return x;
  const FmtDesc d = fmt_desc(f);
  if (std::isinf(x)) return d.saturate ? std::copysign(d.maxval, x) : x;
  if (x == 0.0) return x;
  const double ax = std::fabs(x);
  int e;
  std::frexp(ax, &e);            // ax = m * 2^e, m in [0.5, 1): leading bit at 2^(e-1)
  const int lead = e - 1;
  const int quantum = std::max(lead, d.emin) - (d.p - 1);
  const double scaled = std::ldexp(ax, -quantum);   // exact: power-of-two scaling
  const double r = std::nearbyint(scaled);           // default mode: to nearest, ties to even
  double y = std::ldexp(r, quantum);
  if (y > d.maxval) y = d.saturate ? d.maxval : INFINITY;
  return std::copysign(y, x);
}

// ---------------------------------------------------------------------------
// Scalable generator (section "Matrix Generation"): every entry is reachable
// from the seed in O(log t) steps, so any tile of an arbitrarily large matrix
// can be produced independently.  The paper fixes no generator; the reading is
// a 64-bit linear congruential generator with Knuth's MMIX multiplier and
// increment, and F. Brown's 1994 arbitrary-stride jump for the skip-ahead.
// ---------------------------------------------------------------------------
const uint64_t kLcgMul = 6364136223846793005ULL;
const uint64_t kLcgAdd = 1442695040888963407ULL;

// Affine map s -> a*s + c (mod 2^64) equal to k applications of one step.
void lcg_jump(uint64_t k, uint64_t* out_a, uint64_t* out_c) {
  uint64_t acc_a = 1, acc_c = 0;         // identity map
  uint64_t sq_a = kLcgMul, sq_c = kLcgAdd;  // the step map raised to 2^bit
  while (k != 0) {
    if (k & 1) {
      acc_a = acc_a * sq_a;
      acc_c = acc_c * sq_a + sq_c;
    }
    sq_c = (sq_a + 1) * sq_c;
    sq_a = sq_a * sq_a;
    k >>= 1;
  }
  *out_a = acc_a;
  *out_c = acc_c;
}

// Draw t (t >= 0) of the stream seeded with `seed` uses state s_{t+1}.
// Mapping: the top 52 bits u of the state give the odd integer
// q = 2u + 1 - 2^52, |q| < 2^52, and the value q * 2^-53, exact in fp64 and in
// the open interval (-0.5, 0.5).
inline int64_t state_to_q(uint64_t s) {
  const int64_t u = (int64_t)(s >> 12);
  return 2 * u + 1 - (int64_t(1) << 52);
}
inline double q_to_value(int64_t q) { return std::ldexp((double)q, -53); }

// Exact unsigned 128-bit integer -> fp64, rounding to nearest, ties to even
// (the compiler's conversion follows the IEEE default rounding mode).
inline double u128_to_double(u128 v) { return (double)v; }

enum DiagMode { DIAG_DOMINANT = 0, DIAG_SQRTN = 1, DIAG_NONE = 2, DIAG_DEPARTURE = 3 };

// Diagonal of row i from its exact off-diagonal magnitude sum S (an integer
// number of 2^-53 units), the raw draw q_ii and the mode.
//  * DOMINANT: a_ii = fl(fl(S) * 2^-53 + margin): the row's absolute sum plus
//    the margin, so A is strictly row diagonally dominant by `margin`.
//  * SQRTN: a_ii = fl(q_ii 2^-53 + sign(q_ii) * fl(c * fl(sqrt(n)))) with
//    c = margin: the sqrt(n) diagonal scaling the experiments section
//    recommends (c = 1) and its 5/8 sqrt(n) curve (c = 5/8).
//  * NONE: the raw draw (uniform entries without diagonal scaling).
//  * DEPARTURE: a_ii = fl(fl(S) * 2^-53 * rho), rho = margin: the "departure
//    from diagonal dominance" of section "Matrix Generation", whose formula
//    the paper does not print; reading: the diagonal is the fraction rho of
//    the row's off-diagonal absolute sum (rho < 1 departs from dominance).
double diag_value(int mode, u128 S, int64_t q_ii, double margin, int64_t n) {
  switch (mode) {
    case DIAG_DOMINANT: return std::ldexp(u128_to_double(S), -53) + margin;
    case DIAG_DEPARTURE: return std::ldexp(u128_to_double(S), -53) * margin;
    case DIAG_SQRTN: {
      const double r = margin * std::sqrt((double)n);
      return q_to_value(q_ii) + (q_ii > 0 ? r : -r);
    }
    default: return q_to_value(q_ii);
  }
}

// ---------------------------------------------------------------------------
// Low-precision blocked right-looking LU without pivoting (section
// "Algorithmic Framework", Fig. 1 and the paragraph after it).
//
// The matrix is factored in place; every stored value is rounded to the
// storage format after each step.  Reading of the paper's scheme used here
// (the paper permits a custom mixed-precision scheme):
//   (i)   the diagonal block is factored in fp32 arithmetic (blocks wider
//         than 128 recursively, with the same algorithm at depth 128);
//   (ii)  the triangular solves multiply by explicitly inverted 128x128
//         diagonal sub-blocks (inverses formed in fp32 arithmetic), so the
//         panel work is products of low-precision operands with fp32
//         accumulation, like the Schur update;
//   (iii) the Schur complement A22 <- A22 - A21 A11^{-1} A12 is one product of
//         low-precision operands accumulated in fp32 over the whole panel
//         width, rounded once into storage.
// Template parameter T is the arithmetic type (float for the method; double
// together with FMT_FP64 storage gives the exact-arithmetic special case used
// as a pin against the textbook factorization).
// ---------------------------------------------------------------------------
const int kBase = 128;  // width of the diagonal sub-blocks factored unblocked

template <class T>
inline T fma_t(T a, T b, T c);
template <>
inline float fma_t<float>(float a, float b, float c) { return std::fmaf(a, b, c); }
template <>
inline double fma_t<double>(double a, double b, double c) { return std::fma(a, b, c); }

template <class T>
struct LowPrecLU {
  int64_t n;
  int fmt;                  // storage format of factors and trailing matrix
  int fmt_update;           // operand format of the Schur update (FMT_E4M3 = fp8 variant)
  bool trail32 = false;     // 32-bit trailing matrix: top-level Schur results stay fp32, a block
                            // column / row is rounded to fmt once, when it becomes the panel
  std::vector<double> M;    // working matrix, column major, ld = n
  // inverses of the 128-wide diagonal sub-blocks, indexed by block start / 128
  std::vector<std::vector<double>> Linv, Uinv;  // column major, ld = 128

  double& at(int64_t i, int64_t j) { return M[(size_t)i + (size_t)j * (size_t)n]; }
  double st(double v) const { return round_fmt(v, fmt); }

  // (i) unblocked right-looking factorization of the b x b block at (k, k),
  // b <= 128, in arithmetic T; l = a / pivot, then rank-1 updates, pivots in
  // ascending order.  Followed by the inverses of the stored unit-lower L and
  // upper U factors of the block.  Returns false on a zero or non-finite pivot.
  bool getrf_base(int64_t k, int64_t b) {
    std::vector<T> a((size_t)b * b);
    for (int64_t j = 0; j < b; ++j)
      for (int64_t i = 0; i < b; ++i) a[i + j * b] = (T)at(k + i, k + j);
    bool ok = true;
    for (int64_t p = 0; p < b; ++p) {
      const T piv = a[p + p * b];
      if (!(std::isfinite((double)piv)) || piv == T(0)) ok = false;
      for (int64_t i = p + 1; i < b; ++i) a[i + p * b] = a[i + p * b] / piv;
      for (int64_t j = p + 1; j < b; ++j)
        for (int64_t i = p + 1; i < b; ++i)
          a[i + j * b] = fma_t<T>(-a[i + p * b], a[p + j * b], a[i + j * b]);
    }
    for (int64_t j = 0; j < b; ++j)
      for (int64_t i = 0; i < b; ++i) at(k + i, k + j) = st((double)a[i + j * b]);

    // Inverse of the unit lower factor X = L^{-1} (from the stored values):
    // X[r][c] = -sum_{t=c}^{r-1} L[r][t] X[t][c], t ascending, X[c][c] = 1.
    std::vector<double> li((size_t)kBase * kBase, 0.0), ui((size_t)kBase * kBase, 0.0);
    for (int64_t c = 0; c < b; ++c) {
      std::vector<T> x(b, T(0));
      x[c] = T(1);
      for (int64_t r = c + 1; r < b; ++r) {
        T acc = T(0);
        for (int64_t t = c; t < r; ++t) acc = fma_t<T>(-(T)at(k + r, k + t), x[t], acc);
        x[r] = acc;
      }
      for (int64_t r = 0; r < b; ++r) li[r + c * kBase] = st((double)x[r]);
    }
    // Inverse of the upper factor Y = U^{-1}: Y[c][c] = 1 / U[c][c] and, for
    // r < c, Y[r][c] = (-sum_{t=c}^{r+1} U[r][t] Y[t][c]) / U[r][r] with t
    // descending from c.
    for (int64_t c = 0; c < b; ++c) {
      std::vector<T> y(b, T(0));
      y[c] = T(1) / (T)at(k + c, k + c);
      for (int64_t r = c - 1; r >= 0; --r) {
        T acc = T(0);
        for (int64_t t = c; t > r; --t) acc = fma_t<T>((T)at(k + r, k + t), y[t], acc);
        y[r] = -acc / (T)at(k + r, k + r);
      }
      for (int64_t r = 0; r < b; ++r) ui[r + c * kBase] = st((double)y[r]);
    }
    Linv[(size_t)(k / kBase)] = li;
    Uinv[(size_t)(k / kBase)] = ui;
    return ok;
  }

  // (ii) U12 = L_D^{-1} A12 for the diagonal block D = [k, k+b) and columns
  // [c0, c1), by block forward substitution over the 128-wide sub-blocks s of
  // D:  U_s = st( W_s U_{0:s} + Linv_ss A_s ) with W_s = st(-Linv_ss L_{s,0:s}),
  // one fp32 accumulation over the rows of D in ascending order.
  void trsm_row_panel(int64_t k, int64_t b, int64_t c0, int64_t c1) {
    for (int64_t s0 = k; s0 < k + b; s0 += kBase) {
      const int64_t bs = std::min<int64_t>(kBase, k + b - s0);
      const std::vector<double>& li = Linv[(size_t)(s0 / kBase)];
      // W (bs x (s0-k)), column major
      const int64_t wk = s0 - k;
      std::vector<double> W((size_t)bs * std::max<int64_t>(wk, 1));
      for (int64_t q = 0; q < wk; ++q)
        for (int64_t p = 0; p < bs; ++p) {
          T acc = T(0);
          for (int64_t t = 0; t < bs; ++t)
            acc = fma_t<T>((T)li[p + t * kBase], (T)at(s0 + t, k + q), acc);
          W[p + q * bs] = st(-(double)acc);
        }
      std::vector<double> out((size_t)bs);
      for (int64_t j = c0; j < c1; ++j) {
        for (int64_t p = 0; p < bs; ++p) {
          T acc = T(0);
          for (int64_t q = 0; q < wk; ++q) acc = fma_t<T>((T)W[p + q * bs], (T)at(k + q, j), acc);
          for (int64_t t = 0; t < bs; ++t)
            acc = fma_t<T>((T)li[p + t * kBase], (T)at(s0 + t, j), acc);
          out[p] = st((double)acc);
        }
        for (int64_t p = 0; p < bs; ++p) at(s0 + p, j) = out[p];
      }
    }
  }

  // (ii') L21 = A21 U_D^{-1} for rows [r0, r1), by block substitution over the
  // 128-wide sub-blocks s of D: L_s = st( L_{0:s} Z_s + A_s Uinv_ss ) with
  // Z_s = st(-U_{0:s,s} Uinv_ss), one fp32 accumulation over the columns of D
  // in ascending order.
  void trsm_col_panel(int64_t k, int64_t b, int64_t r0, int64_t r1) {
    for (int64_t s0 = k; s0 < k + b; s0 += kBase) {
      const int64_t bs = std::min<int64_t>(kBase, k + b - s0);
      const std::vector<double>& ui = Uinv[(size_t)(s0 / kBase)];
      const int64_t zk = s0 - k;
      std::vector<double> Z((size_t)std::max<int64_t>(zk, 1) * bs);  // zk x bs, column major
      for (int64_t p = 0; p < bs; ++p)
        for (int64_t q = 0; q < zk; ++q) {
          T acc = T(0);
          for (int64_t t = 0; t < bs; ++t)
            acc = fma_t<T>((T)at(k + q, s0 + t), (T)ui[t + p * kBase], acc);
          Z[q + p * zk] = st(-(double)acc);
        }
      std::vector<double> out((size_t)bs);
      for (int64_t i = r0; i < r1; ++i) {
        for (int64_t p = 0; p < bs; ++p) {
          T acc = T(0);
          for (int64_t q = 0; q < zk; ++q) acc = fma_t<T>((T)at(i, k + q), (T)Z[q + p * zk], acc);
          for (int64_t t = 0; t < bs; ++t)
            acc = fma_t<T>((T)at(i, s0 + t), (T)ui[t + p * kBase], acc);
          out[p] = st((double)acc);
        }
        for (int64_t p = 0; p < bs; ++p) at(i, s0 + p) = out[p];
      }
    }
  }

  // (iii) Schur update A22 <- st(A22 - L21 U12) over rows/cols [k+b, e) with
  // depth [k, k+b), fp32 accumulation in ascending p (Fig. 1).
  // `top` is false inside the recursive factorization of a diagonal block:
  // those updates are part of the diagonal-block factorization and keep the
  // storage format even in the FP8 variant.
  void schur_update(int64_t k, int64_t b, int64_t e, bool top) {
    if (top && fmt_update == FMT_E4M3) { schur_update_fp8(k, b, e); return; }
    const bool keep32 = top && trail32;
#pragma omp parallel for schedule(static)
    for (int64_t j = k + b; j < e; ++j)
      for (int64_t i = k + b; i < e; ++i) {
        T acc = T(0);
        for (int64_t p = k; p < k + b; ++p) acc = fma_t<T>((T)at(i, p), (T)at(p, j), acc);
        const double v = (double)((T)at(i, j) - acc);
        at(i, j) = keep32 ? round_fmt(v, FMT_FP32) : st(v);
      }
  }

  // 32-bit trailing matrix: block column [k, e) x [k, k+b) and block row
  // [k, k+b) x [k+b, e) rounded to the storage format when they become the panel
  void round_panel(int64_t k, int64_t b, int64_t e) {
    for (int64_t j = k; j < k + b; ++j)
      for (int64_t i = k; i < e; ++i) at(i, j) = st(at(i, j));
    for (int64_t j = k + b; j < e; ++j)
      for (int64_t i = k; i < k + b; ++i) at(i, j) = st(at(i, j));
  }

  // FP8 variant of (iii): the operands L21 and U12 are quantized per 128x128
  // tile to OCP E4M3 with an fp32 scale s = fl32(amax / 448) (s = 1 when the
  // tile is zero), q = E4M3(fl32(x / s)).  Tiles are aligned to the panel start
  // k: L tiles are [k+b+128a, +128) x [k+128g, +128), U tiles
  // [k+128g, +128) x [k+b+128c, +128).  For every 128-deep slice g the exact
  // E4M3 products are accumulated in fp32 (ascending p) into acc_g and folded
  // as acc = fma(acc_g, fl32(sL*sU), acc), g ascending; then A22 <- st(A22 - acc).
  void schur_update_fp8(int64_t k, int64_t b, int64_t e) {
    const int64_t m = e - (k + b);
    if (m <= 0) return;
    const int64_t nt = (m + kBase - 1) / kBase, ng = (b + kBase - 1) / kBase;
    std::vector<float> sL((size_t)nt * ng), sU((size_t)ng * nt);
    std::vector<float> qL((size_t)m * b), qU((size_t)b * m);  // qL row i col p (m x b, col major); qU (b x m)
    auto quant_tile = [&](bool isL, int64_t a, int64_t g) {
      const int64_t i0 = k + b + a * kBase, p0 = k + g * kBase;
      const int64_t ie = std::min<int64_t>(i0 + kBase, e), pe = std::min<int64_t>(p0 + kBase, k + b);
      float amax = 0.0f;
      for (int64_t x = i0; x < ie; ++x)
        for (int64_t p = p0; p < pe; ++p) {
          const float v = (float)(isL ? at(x, p) : at(p, x));
          amax = std::max(amax, std::fabs(v));
        }
      const float s = amax == 0.0f ? 1.0f : amax / 448.0f;
      for (int64_t x = i0; x < ie; ++x)
        for (int64_t p = p0; p < pe; ++p) {
          const float v = (float)(isL ? at(x, p) : at(p, x));
          const float q = (float)round_fmt((double)(v / s), FMT_E4M3);
          if (isL) qL[(size_t)(x - (k + b)) + (size_t)(p - k) * m] = q;
          else qU[(size_t)(p - k) + (size_t)(x - (k + b)) * b] = q;
        }
      if (isL) sL[(size_t)a * ng + g] = s; else sU[(size_t)g * nt + a] = s;
    };
    for (int64_t a = 0; a < nt; ++a)
      for (int64_t g = 0; g < ng; ++g) { quant_tile(true, a, g); quant_tile(false, a, g); }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j)
      for (int64_t i = 0; i < m; ++i) {
        float acc = 0.0f;
        for (int64_t g = 0; g < ng; ++g) {
          float ag = 0.0f;
          const int64_t pe = std::min<int64_t>((g + 1) * kBase, b);
          for (int64_t p = g * kBase; p < pe; ++p)
            ag = std::fmaf(qL[(size_t)i + (size_t)p * m], qU[(size_t)p + (size_t)j * b], ag);
          const float sc = sL[(size_t)(i / kBase) * ng + g] * sU[(size_t)g * nt + j / kBase];
          acc = std::fmaf(ag, sc, acc);
        }
        double& c = at(k + b + i, k + b + j);
        c = st((double)((float)c - acc));
      }
  }

  // ------------------------------------------------------------------------
  // Plain reading of Fig. 1 (no inverses): the nb x nb diagonal block is
  // factored unblocked in fp32 as one block, and the panels are formed by
  // fp32 forward / back substitution with the stored low-precision L11 / U11,
  // each panel entry rounded to storage once.  Used to measure how far the
  // method's inverse-based panels sit from the textbook substitution.
  // ------------------------------------------------------------------------
  bool getrf_plain(int64_t k, int64_t b) {
    std::vector<T> a((size_t)b * b);
    for (int64_t j = 0; j < b; ++j)
      for (int64_t i = 0; i < b; ++i) a[i + j * b] = (T)at(k + i, k + j);
    bool ok = true;
    for (int64_t p = 0; p < b; ++p) {
      const T piv = a[p + p * b];
      if (!(std::isfinite((double)piv)) || piv == T(0)) ok = false;
      for (int64_t i = p + 1; i < b; ++i) a[i + p * b] = a[i + p * b] / piv;
      for (int64_t j = p + 1; j < b; ++j)
        for (int64_t i = p + 1; i < b; ++i)
          a[i + j * b] = fma_t<T>(-a[i + p * b], a[p + j * b], a[i + j * b]);
    }
    for (int64_t j = 0; j < b; ++j)
      for (int64_t i = 0; i < b; ++i) at(k + i, k + j) = st((double)a[i + j * b]);
    return ok;
  }

  // U12 = L11^{-1} A12, column by column: u_r = a_r - sum_{t<r} l_rt u_t in T,
  // t ascending, then every u_r rounded to storage.
  void trsm_row_plain(int64_t k, int64_t b, int64_t c0, int64_t c1) {
    std::vector<T> u((size_t)b);
    for (int64_t j = c0; j < c1; ++j) {
      for (int64_t r = 0; r < b; ++r) {
        T acc = (T)at(k + r, j);
        for (int64_t t = 0; t < r; ++t) acc = fma_t<T>(-(T)at(k + r, k + t), u[t], acc);
        u[r] = acc;
      }
      for (int64_t r = 0; r < b; ++r) at(k + r, j) = st((double)u[r]);
    }
  }

  // L21 = A21 U11^{-1}, row by row: l_c = (a_c - sum_{t<c} l_t u_tc) / u_cc in
  // T, t ascending, then every l_c rounded to storage.
  void trsm_col_plain(int64_t k, int64_t b, int64_t r0, int64_t r1) {
    std::vector<T> l((size_t)b);
    for (int64_t i = r0; i < r1; ++i) {
      for (int64_t c = 0; c < b; ++c) {
        T acc = (T)at(i, k + c);
        for (int64_t t = 0; t < c; ++t) acc = fma_t<T>(-l[t], (T)at(k + t, k + c), acc);
        l[c] = acc / (T)at(k + c, k + c);
      }
      for (int64_t c = 0; c < b; ++c) at(i, k + c) = st((double)l[c]);
    }
  }

  bool lu_plain(int NB) {
    bool ok = true;
    for (int64_t k = 0; k < n; k += NB) {
      const int64_t b = std::min<int64_t>(NB, n - k);
      ok = getrf_plain(k, b) && ok;
      if (k + b >= n) break;
      trsm_row_plain(k, b, k + b, n);
      trsm_col_plain(k, b, k + b, n);
      schur_update(k, b, n, true);
    }
    return ok;
  }

  // Factor the square sub-matrix [k0, k0+size)^2 with update depth NB.
  bool lu_range(int64_t k0, int64_t size, int NB, bool top) {
    bool ok = true;
    const int64_t e = k0 + size;
    for (int64_t k = k0; k < e; k += NB) {
      const int64_t b = std::min<int64_t>(NB, e - k);
      if (top && trail32) round_panel(k, b, e);
      if (b <= kBase) ok = getrf_base(k, b) && ok;
      else ok = lu_range(k, b, kBase, false) && ok;
      if (k + b >= e) break;
      trsm_row_panel(k, b, k + b, e);
      trsm_col_panel(k, b, k + b, e);
      schur_update(k, b, e, top);
    }
    return ok;
  }
};

// ---------------------------------------------------------------------------
// Balancing and scaling (section "Algorithmic Framework": a Theta(n^2)
// balancing borrowed from the HPL harness and a scaling into the range of the
// low-precision format, both timed and undone at the end).  Reading: row then
// column equilibration by powers of two, rs_i = 2^-floor(log2 max_j |a_ij|),
// cs_j = 2^-floor(log2 max_i |rs_i a_ij|), the logarithms taken exactly (as
// integers, so no product can under- or overflow); a row or column that holds
// a non-finite entry, or only zeros, gets 1; then rs times the format's scale
// (2^12 for FP16, 1 otherwise).  The factorization then works on
// diag(rs) A diag(cs), and the preconditioner is
// M^{-1} = diag(cs) U^{-1} L^{-1} diag(rs), which undoes the balancing.
// ---------------------------------------------------------------------------
int floor_log2(double a) {   // finite a != 0
  int e;
  std::frexp(std::fabs(a), &e);   // |a| = f 2^e, f in [0.5, 1)
  return e - 1;
}

void balance(int64_t n, const double* A, int64_t lda, int fmt, double* rs, double* cs) {
  for (int64_t i = 0; i < n; ++i) {
    bool bad = false, any = false;
    int m = 0;
    for (int64_t j = 0; j < n; ++j) {
      const double a = A[i + j * lda];
      if (!std::isfinite(a)) bad = true;
      else if (a != 0.0) { m = any ? std::max(m, floor_log2(a)) : floor_log2(a); any = true; }
    }
    rs[i] = (bad || !any) ? 1.0 : std::ldexp(1.0, -m);
  }
  for (int64_t j = 0; j < n; ++j) {
    bool bad = false, any = false;
    int m = 0;
    for (int64_t i = 0; i < n; ++i) {
      const double a = A[i + j * lda];
      if (!std::isfinite(a)) { bad = true; continue; }
      if (a == 0.0) continue;
      const int l = floor_log2(a) + floor_log2(rs[i]);
      m = any ? std::max(m, l) : l;
      any = true;
    }
    cs[j] = (bad || !any) ? 1.0 : std::ldexp(1.0, -m);
  }
  const double s = fmt == FMT_FP16 ? 4096.0 : 1.0;
  for (int64_t i = 0; i < n; ++i) rs[i] *= s;
}

// ---------------------------------------------------------------------------
// fp64 refinement helpers (section "Algorithmic Framework": GMRES with the
// low-precision factors as a left preconditioner, fp64 working precision).
// ---------------------------------------------------------------------------

// z = U^{-1} L^{-1} v with the stored factors widened exactly; arithmetic Tp
// (double = the fp64 preconditioner; float = the fp32 option).
template <class Tp>
void precond_apply(int64_t n, const double* LU, int64_t ld, const double* v, double* z) {
  std::vector<Tp> y((size_t)n);
  for (int64_t i = 0; i < n; ++i) {   // forward, unit lower
    Tp acc = (Tp)v[i];
    for (int64_t j = 0; j < i; ++j) acc = fma_t<Tp>(-(Tp)LU[i + j * ld], y[j], acc);
    y[i] = acc;
  }
  for (int64_t i = n - 1; i >= 0; --i) {   // backward, upper
    Tp acc = y[i];
    for (int64_t j = i + 1; j < n; ++j) acc = fma_t<Tp>(-(Tp)LU[i + j * ld], y[j], acc);
    y[i] = acc / (Tp)LU[i + i * ld];
  }
  for (int64_t i = 0; i < n; ++i) z[i] = (double)y[i];
}

// w = A v with fp32 operands and accumulation: A_ij truncated toward zero to
// fp32, v_j rounded to nearest fp32, products accumulated by fused
// multiply-add in fp32, j ascending (the fp32 operator of GMRES when the
// preconditioner is applied in fp32).
void matvec_f32(int64_t n, const double* A, int64_t lda, const double* v, double* w) {
  std::vector<float> vf((size_t)n);
  for (int64_t j = 0; j < n; ++j) vf[j] = (float)v[j];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    float acc = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
      const double a = A[i + j * lda];
      float f = (float)a;
      if (std::fabs((double)f) > std::fabs(a)) f = std::nextafter(f, 0.0f);
      acc = std::fmaf(f, vf[j], acc);
    }
    w[i] = (double)acc;
  }
}

// r = b - A x, fp64, one fused multiply-add per term, j ascending.
void residual_vec(int64_t n, const double* A, int64_t lda, const double* x, const double* b,
                  double* r) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) acc = std::fma(A[i + j * lda], x[j], acc);
    r[i] = b[i] - acc;
  }
}

double norm_inf_vec(int64_t n, const double* v) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double a = std::fabs(v[i]);
    if (!(a <= m)) m = a;   // propagates NaN
  }
  return m;
}

double norm_inf_mat(int64_t n, const double* A, int64_t lda) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += std::fabs(A[i + j * lda]);
    if (!(s <= m)) m = s;
  }
  return m;
}

double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = std::fma(a[i], b[i], s);
  return s;
}

// HPL backward error (section "Algorithmic Framework"):
// ||Ax-b||_inf / ((||A||_inf ||x||_inf + ||b||_inf) * n * eps), eps = 2^-53.
double scaled_resid(double rn, double an, double xn, double bn, int64_t n) {
  return rn / ((an * xn + bn) * ((double)n * std::ldexp(1.0, -53)));
}

}  // namespace

// ===========================================================================
// C interface (ctypes)
// ===========================================================================
extern "C" {

double oracle_round(double x, int fmt) { return round_fmt(x, fmt); }

void oracle_round_array(const double* x, double* y, int64_t count, int fmt) {
  for (int64_t i = 0; i < count; ++i) y[i] = round_fmt(x[i], fmt);
}

void oracle_lcg_jump(uint64_t k, uint64_t* a, uint64_t* c) { lcg_jump(k, a, c); }

// State after t steps from `seed` (t = 0 gives the seed itself).
uint64_t oracle_lcg_state(uint64_t seed, uint64_t t) {
  uint64_t a, c;
  lcg_jump(t, &a, &c);
  return a * seed + c;
}

// Reference stepping (no skip-ahead): out[i] = state after i+1 steps.
void oracle_lcg_sequence(uint64_t seed, int64_t count, uint64_t* out) {
  uint64_t s = seed;
  for (int64_t i = 0; i < count; ++i) {
    s = kLcgMul * s + kLcgAdd;
    out[i] = s;
  }
}

double oracle_draw_value(uint64_t seed, uint64_t t) {
  uint64_t a, c;
  lcg_jump(t + 1, &a, &c);
  return q_to_value(state_to_q(a * seed + c));
}

// Full generation, sequential stepping through the stream: A (column major,
// entry (i,j) is draw i + j*n), then b (entry (i,r) is draw n*n + i + r*n).
// Returns 0, or -1 on bad arguments.
int oracle_generate(int64_t n, uint64_t seed, double margin, int mode, double* A, int64_t lda,
                    double* b, int64_t ldb, int64_t nrhs) {
  if (n < 1 || lda < n || (nrhs > 0 && ldb < n) || n > (int64_t(1) << 17)) return -1;
  if (mode < DIAG_DOMINANT || mode > DIAG_DEPARTURE || (mode == DIAG_DEPARTURE && !(margin > 0.0))) return -1;
  std::vector<u128> S((size_t)n, 0);
  std::vector<int64_t> qd((size_t)n, 0);
  uint64_t s = seed;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      s = kLcgMul * s + kLcgAdd;
      const int64_t q = state_to_q(s);
      A[i + j * lda] = q_to_value(q);
      if (i != j) S[(size_t)i] += (u128)(q < 0 ? -q : q);
      else qd[(size_t)i] = q;
    }
  for (int64_t i = 0; i < n; ++i) A[i + i * lda] = diag_value(mode, S[(size_t)i], qd[(size_t)i], margin, n);
  for (int64_t r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < n; ++i) {
      s = kLcgMul * s + kLcgAdd;
      b[i + r * ldb] = q_to_value(state_to_q(s));
    }
  return 0;
}

// Selected full rows of A (row-major out, nrows x n) by skip-ahead, for spot
// checks of matrices too large to generate on the host.
int oracle_generate_rows(int64_t n, uint64_t seed, double margin, int mode, const int64_t* rows,
                         int64_t nrows, double* out) {
  if (n < 1 || n > (int64_t(1) << 17)) return -1;
  if (mode < DIAG_DOMINANT || mode > DIAG_DEPARTURE || (mode == DIAG_DEPARTURE && !(margin > 0.0))) return -1;
  uint64_t an, cn;
  lcg_jump((uint64_t)n, &an, &cn);
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows[r];
    if (i < 0 || i >= n) return -1;
    uint64_t a1, c1;
    lcg_jump((uint64_t)i + 1, &a1, &c1);
    uint64_t s = a1 * seed + c1;   // draw i (column 0)
    u128 S = 0;
    int64_t qd = 0;
    for (int64_t j = 0; j < n; ++j) {
      const int64_t q = state_to_q(s);
      out[r * n + j] = q_to_value(q);
      if (j != i) S += (u128)(q < 0 ? -q : q);
      else qd = q;
      s = an * s + cn;
    }
    out[r * n + i] = diag_value(mode, S, qd, margin, n);
  }
  return 0;
}

// Low-precision LU.  LU (out, column major, ld = ldlu) receives the stored
// factor values widened to fp64 (unit-lower L below the diagonal, U on and
// above).  fmt: storage format (0 BF16, 1 FP16, 4 FP64 = exact special case,
// which also switches the arithmetic to fp64); fmt_update: 2 selects E4M3
// operands for the Schur update, anything else the storage format.
// Returns 0, 1 on a zero or non-finite pivot, -1 on bad arguments.
int oracle_factor_scheme(int64_t n, const double* A, int64_t lda, int fmt, int fmt_update, int nb,
                         double* LU, int64_t ldlu, int plain, const double* rs, const double* cs, int trail32);

int oracle_factor(int64_t n, const double* A, int64_t lda, int fmt, int fmt_update, int nb,
                  double* LU, int64_t ldlu) {
  return oracle_factor_scheme(n, A, lda, fmt, fmt_update, nb, LU, ldlu, 0, nullptr, nullptr, 0);
}

// The factorization in the method's scheme (plain = 0, above) or in the plain
// reading of Fig. 1 (plain = 1: unblocked fp32 diagonal block of width nb,
// fp32 substitution panels, no inverses; no fp8 update; with FP64 storage the
// arithmetic is fp64, the exact-arithmetic special case; nb may also be 64,
// the block width of the fp64 study factorization).
// rs, cs (both or neither): factor diag(rs) A diag(cs) instead of A (the
// powers of two are applied in fp64, exactly, before the one rounding).
// trail32 (method scheme, 16-bit fmt, no fp8 update): Fig. 1 with a 32-bit
// trailing matrix: the input rounded to fp32, the top-level Schur results
// kept in fp32, each block column / row rounded to fmt when it becomes the
// panel.
int oracle_factor_scheme(int64_t n, const double* A, int64_t lda, int fmt, int fmt_update, int nb,
                         double* LU, int64_t ldlu, int plain, const double* rs, const double* cs, int trail32) {
  if (trail32 && (plain || fmt == FMT_FP64 || fmt_update == FMT_E4M3)) return -1;
  if (n < 1 || lda < n || ldlu < n || !(nb == 128 || nb == 256 || nb == 512 || (plain && nb == 64))) return -1;
  if (plain && fmt_update == FMT_E4M3) return -1;
  bool ok;
  if (fmt == FMT_FP64) {
    LowPrecLU<double> f;
    f.n = n; f.fmt = fmt; f.fmt_update = FMT_FP64;
    f.M.resize((size_t)n * n);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) f.M[i + j * n] = rs ? A[i + j * lda] * rs[i] * cs[j] : A[i + j * lda];
    f.Linv.resize((size_t)(n + kBase - 1) / kBase);
    f.Uinv.resize(f.Linv.size());
    ok = plain ? f.lu_plain(nb) : f.lu_range(0, n, nb, true);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) LU[i + j * ldlu] = f.M[i + j * n];
  } else {
    LowPrecLU<float> f;
    f.n = n; f.fmt = fmt; f.fmt_update = fmt_update == FMT_E4M3 ? FMT_E4M3 : fmt;
    f.trail32 = trail32 != 0;
    f.M.resize((size_t)n * n);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i)
        f.M[i + j * n] = round_fmt(rs ? A[i + j * lda] * rs[i] * cs[j] : A[i + j * lda], trail32 ? FMT_FP32 : fmt);
    f.Linv.resize((size_t)(n + kBase - 1) / kBase);
    f.Uinv.resize(f.Linv.size());
    ok = plain ? f.lu_plain(nb) : f.lu_range(0, n, nb, true);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) LU[i + j * ldlu] = f.M[i + j * n];
  }
  return ok ? 0 : 1;
}

// The fp32 Arnoldi product of the inner GMRES alone: w = A v with A truncated
// toward zero to fp32, v rounded to fp32, fp32 fused multiply-adds, j
// ascending (matvec_f32 above).
void oracle_matvec_f32(int64_t n, const double* A, int64_t lda, const double* v, double* w) {
  matvec_f32(n, A, lda, v, w);
}

// Apply the preconditioner z = U^{-1} L^{-1} v (prec 0: fp64, 1: fp32).
void oracle_precond(int64_t n, const double* LU, int64_t ld, const double* v, double* z, int prec) {
  if (prec == 1) precond_apply<float>(n, LU, ld, v, z);
  else precond_apply<double>(n, LU, ld, v, z);
}

// With the factors of diag(rs) A diag(cs): z = diag(cs) U^{-1} L^{-1} diag(rs) v
// (rs, cs NULL: no balancing).
void oracle_precond_scaled(int64_t n, const double* LU, int64_t ld, const double* v, double* z, int prec,
                           const double* rs, const double* cs) {
  if (!rs) { oracle_precond(n, LU, ld, v, z, prec); return; }
  std::vector<double> w((size_t)n);
  for (int64_t i = 0; i < n; ++i) w[i] = v[i] * rs[i];
  oracle_precond(n, LU, ld, w.data(), z, prec);
  for (int64_t i = 0; i < n; ++i) z[i] *= cs[i];
}

// Balancing scales of A for the format fmt (see balance above).
void oracle_balance(int64_t n, const double* A, int64_t lda, int fmt, double* rs, double* cs) {
  balance(n, A, lda, fmt, rs, cs);
}

void oracle_residual_vec(int64_t n, const double* A, int64_t lda, const double* x,
                         const double* b, double* r) {
  residual_vec(n, A, lda, x, b, r);
}

// Scaled residual of every right-hand side (section "Algorithmic Framework").
void oracle_scaled_residual(int64_t n, const double* A, int64_t lda, const double* X, int64_t ldx,
                            const double* B, int64_t ldb, int64_t nrhs, double* out) {
  std::vector<double> r((size_t)n);
  const double an = norm_inf_mat(n, A, lda);
  for (int64_t c = 0; c < nrhs; ++c) {
    residual_vec(n, A, lda, X + c * ldx, B + c * ldb, r.data());
    out[c] = scaled_resid(norm_inf_vec(n, r.data()), an, norm_inf_vec(n, X + c * ldx),
                          norm_inf_vec(n, B + c * ldb), n);
  }
}

// Per right-hand side outcome of the refinement.
struct oracle_ir_info {
  int32_t iters;       // total inner (Arnoldi) steps over all restarts
  int32_t outer;       // restart cycles started
  double scaled_resid; // at exit
  int32_t status;      // 0 ok, 4 no convergence in max_iters, 5 breakdown (non-finite)
};

// GMRES-based iterative refinement (section "Algorithmic Framework"):
//   x0 = U^{-1} L^{-1} b from the low-precision factors; then repeat
//     r = b - A x (fp64);  stop when the scaled residual < accept;
//     fail when max_iters inner steps are spent (the 50-iteration rule);
//     restarted GMRES(restart) on M^{-1} A d = M^{-1} r with M = LU (left
//     preconditioner), modified Gram-Schmidt Arnoldi, Givens rotations;
//     x += V y.
// The inner loop of a cycle stops when the least-squares residual estimate
// |g_{j+1}| <= beta * max(inner_tol, theta * accept / sr0), sr0 being the
// scaled residual at the start of the cycle (theta = 0 disables the adaptive
// term).  Arithmetic: fp64; with pprec 1 the preconditioner of the inner
// GMRES is applied in fp32, with mprec 1 its matrix-vector product A v_j, while
// the outer residual, orthogonalization, rotations and update stay fp64.
// Reading: "iterations" in the 50 cap are inner Arnoldi steps summed over
// restarts.  With bal_r, bal_c (the balancing scales rs, cs of the factors,
// both or neither) the preconditioner is diag(cs) U^{-1} L^{-1} diag(rs) and everything else is in
// the space of the input system.
int oracle_solve_ir(int64_t n, const double* A, int64_t lda, const double* LU, int64_t ldlu,
                    const double* B, int64_t ldb, double* X, int64_t ldx, int64_t nrhs, int restart,
                    int max_iters, double inner_tol, double theta, double accept, int pprec,
                    int mprec, const double* bal_r, const double* bal_c, oracle_ir_info* info) {
  if (n < 1 || restart < 1 || max_iters < 0) return -1;
  const double an = norm_inf_mat(n, A, lda);
  const int m = restart;
  int worst = 0;
  std::vector<double> r(n), z(n), w(n), V((size_t)n * (m + 1)), H((size_t)(m + 1) * m), cs(m), sn(m),
      g(m + 1), y(m);
  for (int64_t c = 0; c < nrhs; ++c) {
    const double* b = B + c * ldb;
    double* x = X + c * ldx;
    const double bn = norm_inf_vec(n, b);
    oracle_precond_scaled(n, LU, ldlu, b, x, pprec, bal_r, bal_c);
    int iters = 0, outer = 0, status = 0;
    double sr = 0.0;
    for (;;) {
      residual_vec(n, A, lda, x, b, r.data());
      sr = scaled_resid(norm_inf_vec(n, r.data()), an, norm_inf_vec(n, x), bn, n);
      if (!std::isfinite(sr)) { status = 5; break; }
      if (sr < accept) { status = 0; break; }
      if (iters >= max_iters) { status = 4; break; }
      ++outer;
      oracle_precond_scaled(n, LU, ldlu, r.data(), z.data(), pprec, bal_r, bal_c);
      const double beta = std::sqrt(dot(n, z.data(), z.data()));
      if (!std::isfinite(beta) || beta == 0.0) { status = 5; break; }
      for (int64_t i = 0; i < n; ++i) V[i] = z[i] / beta;
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      const double tol = beta * std::max(inner_tol, theta > 0.0 ? theta * accept / sr : 0.0);
      int k = 0;
      bool bad = false;
      for (int j = 0; j < m && iters < max_iters; ++j) {
        std::vector<double> Av(n);
        std::vector<double> zero(n, 0.0);
        // w = M^{-1} (A v_j): the residual routine with b = 0 gives -A v_j
        if (mprec == 1) {
          matvec_f32(n, A, lda, &V[(size_t)j * n], Av.data());
        } else {
          residual_vec(n, A, lda, &V[(size_t)j * n], zero.data(), Av.data());
          for (int64_t i = 0; i < n; ++i) Av[i] = -Av[i];
        }
        oracle_precond_scaled(n, LU, ldlu, Av.data(), w.data(), pprec, bal_r, bal_c);
        for (int i = 0; i <= j; ++i) {            // modified Gram-Schmidt
          const double h = dot(n, w.data(), &V[(size_t)i * n]);
          H[i + j * (m + 1)] = h;
          for (int64_t t = 0; t < n; ++t) w[t] = std::fma(-h, V[(size_t)i * n + t], w[t]);
        }
        const double hn = std::sqrt(dot(n, w.data(), w.data()));
        H[(j + 1) + j * (m + 1)] = hn;
        for (int i = 0; i < j; ++i) {             // previous rotations
          const double a0 = H[i + j * (m + 1)], a1 = H[(i + 1) + j * (m + 1)];
          H[i + j * (m + 1)] = cs[i] * a0 + sn[i] * a1;
          H[(i + 1) + j * (m + 1)] = -sn[i] * a0 + cs[i] * a1;
        }
        const double hj = H[j + j * (m + 1)];
        const double den = std::hypot(hj, hn);
        if (!std::isfinite(den) || den == 0.0) { bad = true; break; }
        cs[j] = hj / den;
        sn[j] = hn / den;
        H[j + j * (m + 1)] = den;
        H[(j + 1) + j * (m + 1)] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++iters;
        k = j + 1;
        if (hn == 0.0) break;                      // exact (happy) breakdown
        for (int64_t t = 0; t < n; ++t) V[(size_t)(j + 1) * n + t] = w[t] / hn;
        if (std::fabs(g[j + 1]) <= tol) break;
      }
      if (bad) { status = 5; break; }
      for (int i = k - 1; i >= 0; --i) {          // y = H^{-1} g
        double acc = g[i];
        for (int t = i + 1; t < k; ++t) acc = std::fma(-H[i + t * (m + 1)], y[t], acc);
        y[i] = acc / H[i + i * (m + 1)];
      }
      for (int i = 0; i < k; ++i)                  // x += V y
        for (int64_t t = 0; t < n; ++t) x[t] = std::fma(V[(size_t)i * n + t], y[i], x[t]);
    }
    info[c].iters = iters;
    info[c].outer = outer;
    info[c].scaled_resid = sr;
    info[c].status = status;
    worst = std::max(worst, status);
  }
  return worst;
}

int oracle_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Threads used by the oracle's parallel loops from now on (k >= 1); returns
// the number in effect afterwards.
int oracle_set_num_threads(int k) {
#ifdef _OPENMP
  if (k >= 1) omp_set_num_threads(k);
  return omp_get_max_threads();
#else
  (void)k;
  return 1;
#endif
}

}  // extern "C"
