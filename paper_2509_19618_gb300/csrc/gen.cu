// Scalable matrix/RHS generator (section "Matrix Generation").
//
// Entry (i, j) of A is draw t = i + j*n and b(i, r) is draw n*n + i + r*n of a
// 64-bit LCG; draw t uses the state after t+1 steps.  Each thread reaches its
// first state by skip-ahead (affine-map doubling, F. Brown 1994) and then
// steps by n along its row, so every write of a warp is one contiguous run of
// a column (coalesced) and any tile of an arbitrarily large matrix is produced
// independently.  The off-diagonal magnitudes of each row are summed exactly:
// 64-bit per-thread partial sums (at most 512 terms below 2^52 each) folded
// into a 128-bit accumulator per row with carry-propagating atomics, which are
// associative, so the diagonal is bit-for-bit independent of scheduling.
#include "internal.h"

#include <mutex>

namespace hpmxp {
namespace {

constexpr uint64_t kMul = 6364136223846793005ULL;  // Knuth, MMIX
constexpr uint64_t kInc = 1442695040888963407ULL;

struct Affine { uint64_t a, c; };

// The step map applied k times: s -> a s + c (mod 2^64).
__host__ __device__ inline Affine lcg_power(uint64_t k) {
  Affine acc{1, 0}, sq{kMul, kInc};
  while (k) {
    if (k & 1) { acc.c = acc.c * sq.a + sq.c; acc.a = acc.a * sq.a; }
    sq.c = (sq.a + 1) * sq.c;
    sq.a = sq.a * sq.a;
    k >>= 1;
  }
  return acc;
}

// Odd integer q = 2u + 1 - 2^52 from the top 52 bits u of a state.
__device__ inline int64_t state_q(uint64_t s) {
  return (int64_t)((s >> 12) << 1) + 1 - (int64_t(1) << 52);
}
// q * 2^-53 (exact: |q| < 2^53).
__device__ inline double q_value(int64_t q) { return (double)q * 0x1p-53; }

// 128-bit accumulator (lo, hi) += v.  The add that wraps the low word is the
// one that sees old + v < old, so every carry is counted exactly once.
__device__ inline void atomic_add_u128(unsigned long long* p, unsigned long long v) {
  const unsigned long long old = atomicAdd(p, v);
  if (old + v < old) atomicAdd(p + 1, 1ull);
}

// Exact 128-bit unsigned integer -> fp64, round to nearest even.  The top 64
// bits after normalization are rounded by the hardware conversion; a nonzero
// remainder below them is folded into their last bit as a sticky bit, which
// can only break an exact tie, never create one.
__device__ inline double u128_to_f64(unsigned long long hi, unsigned long long lo) {
  if (hi == 0) return __ull2double_rn(lo);
  const int sh = __clzll((long long)hi);
  const unsigned long long top = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
  const unsigned long long rest = lo << sh;
  const double d = __ull2double_rn(top | (rest != 0 ? 1ull : 0ull));
  // exact scaling by 2^(64 - sh)
  return d * __longlong_as_double((long long)(1023 + 64 - sh) << 52);
}

constexpr int kRows = 128;      // rows per CTA (one per thread)
constexpr int kChunk = 512;     // columns per CTA; 512 * 2^52 < 2^64

// Phase 1: values of A for a 128-row x 512-column tile, per-row partial sums
// of the off-diagonal |q| into the 128-bit accumulators sums[2i], sums[2i+1].
__global__ void __launch_bounds__(kRows) gen_matrix_kernel(int64_t n, uint64_t seed, double* A,
                                                           int64_t lda, unsigned long long* sums,
                                                           Affine stride_n) {
  const int64_t i = (int64_t)blockIdx.x * kRows + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * kChunk;
  if (i >= n) return;
  const int64_t j1 = min(j0 + (int64_t)kChunk, n);
  const Affine start = lcg_power((uint64_t)(i + j0 * n) + 1);
  uint64_t s = start.a * seed + start.c;
  unsigned long long part = 0;
  double* col = A + i + j0 * lda;
  for (int64_t j = j0; j < j1; ++j) {
    const int64_t q = state_q(s);
    *col = q_value(q);
    col += lda;
    if (j != i) part += (unsigned long long)(q < 0 ? -q : q);
    s = stride_n.a * s + stride_n.c;
  }
  if (part) atomic_add_u128(sums + 2 * i, part);
}

// Phase 2: the diagonal (section "Matrix Generation": diagonal dominance and
// its "departure"; the c sqrt(n) variants from section "Experimental Results").
//   DOMINANT   a_ii = fl(fl(S_i) 2^-53 + margin)
//   SQRTN      a_ii = fl(q_ii 2^-53 + sign(q_ii) fl(margin fl(sqrt(n))))   (margin = c)
//   NONE       a_ii = q_ii 2^-53
//   DEPARTURE  a_ii = fl(fl(S_i) 2^-53 margin)                            (margin = rho)
__global__ void gen_diag_kernel(int64_t n, uint64_t seed, double margin, int mode, double* A,
                                int64_t lda, const unsigned long long* sums) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v;
  if (mode == HPMXP_DIAG_DOMINANT || mode == HPMXP_DIAG_DEPARTURE) {
    const double S = u128_to_f64(sums[2 * i + 1], sums[2 * i]);
    v = mode == HPMXP_DIAG_DOMINANT ? __dadd_rn(S * 0x1p-53, margin) : __dmul_rn(S * 0x1p-53, margin);
  } else {
    const Affine p = lcg_power((uint64_t)(i + i * n) + 1);
    const int64_t q = state_q(p.a * seed + p.c);
    const double r = __dmul_rn(margin, __dsqrt_rn((double)n));
    v = mode == HPMXP_DIAG_SQRTN ? __dadd_rn(q_value(q), q > 0 ? r : -r) : q_value(q);
  }
  A[i + i * lda] = v;
}

// Right-hand sides: b(i, r) = draw n*n + i + r*n; each thread makes 64
// consecutive entries of one column.
__global__ void gen_rhs_kernel(int64_t n, int64_t nrhs, uint64_t seed, double* b, int64_t ldb) {
  const int64_t per = 64;
  const int64_t tiles = cdiv(n, per);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= tiles * nrhs) return;
  const int64_t r = g / tiles, i0 = (g % tiles) * per;
  const int64_t i1 = min(i0 + per, n);
  const Affine p = lcg_power((uint64_t)(n * n + i0 + r * n) + 1);
  uint64_t s = p.a * seed + p.c;
  for (int64_t i = i0; i < i1; ++i) {
    b[i + r * ldb] = q_value(state_q(s));
    s = kMul * s + kInc;
  }
}

}  // namespace

cudaError_t launch_generate(int64_t n, uint64_t seed, double margin, int mode, double* A,
                            int64_t lda, double* b, int64_t ldb, int64_t nrhs,
                            unsigned long long* sums, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * 2 * (size_t)n, st);
  if (e != cudaSuccess) return e;
  const Affine stride = lcg_power((uint64_t)n);
  dim3 grid((unsigned)cdiv<int64_t>(n, kRows), (unsigned)cdiv<int64_t>(n, kChunk));
  gen_matrix_kernel<<<grid, kRows, 0, st>>>(n, seed, A, lda, sums, stride);
  gen_diag_kernel<<<(unsigned)cdiv<int64_t>(n, 256), 256, 0, st>>>(n, seed, margin, mode, A, lda, sums);
  if (nrhs > 0) {
    const int64_t work = cdiv<int64_t>(n, 64) * nrhs;
    gen_rhs_kernel<<<(unsigned)cdiv<int64_t>(work, 128), 128, 0, st>>>(n, nrhs, seed, b, ldb);
    count_launches(1);
  }
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace hpmxp

// ---------------------------------------------------------------------------
// Generation with library-held scratch (hpmxp_generate_noalloc).  The 128-bit
// row sums live in a fixed array of this module instead of caller memory; the
// arithmetic and the kernels are those of hpmxp_generate.

namespace hpmxp {
namespace {

constexpr int64_t kNoallocMaxN = int64_t(1) << 17;   // 131072 rows: 2 MiB per GPU

// Two 64-bit words (low, high) per row; must be zero when gen_matrix_kernel
// starts, and keeps the previous call's sums afterwards.
static __device__ __align__(256) unsigned long long g_row_sums[2 * kNoallocMaxN];

constexpr int kMaxDevices = 256;
std::mutex g_sums_mutex;
void* g_sums_ptr[kMaxDevices];   // device address of g_row_sums, per device

// The device address of g_row_sums on the current device.  Host code cannot
// use the symbol itself (it names a host-side stand-in), so the address is
// asked for once per device, with that device current, and kept.
cudaError_t row_sums_address(unsigned long long** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_sums_mutex);
  if (!g_sums_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_row_sums);
    if (e != cudaSuccess) return e;
    if (!ptr) return cudaErrorInvalidSymbol;
    g_sums_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned long long*>(g_sums_ptr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace hpmxp

extern "C" hpmxp_status hpmxp_generate_noalloc(int64_t n, uint64_t seed, double margin, int diag_mode,
                                               double* A, int64_t lda, double* b, int64_t ldb, int64_t nrhs,
                                               void* stream) {
  using namespace hpmxp;
  if (n > kNoallocMaxN) return HPMXP_ENOMEM;
  if (n < 1 || !A || lda < n || nrhs < 0 || (nrhs > 0 && (!b || ldb < n))) return HPMXP_EINVAL;
  if (diag_mode < HPMXP_DIAG_DOMINANT || diag_mode > HPMXP_DIAG_DEPARTURE) return HPMXP_EINVAL;
  if (diag_mode == HPMXP_DIAG_DEPARTURE && !(margin > 0.0)) return HPMXP_EINVAL;
  unsigned long long* sums = nullptr;
  cudaError_t e = row_sums_address(&sums);
  if (e != cudaSuccess) return status_from_cuda(e);
  // launch_generate clears the first 2n words on `stream` before the sums are made
  e = launch_generate(n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, sums, (cudaStream_t)stream);
  return status_from_cuda(e);
}
