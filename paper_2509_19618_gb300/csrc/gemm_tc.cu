// Tensor-core product engine for the LU's panel and Schur-update products
// (section "Algorithmic Framework", Fig. 1: low-precision operands, fp32
// accumulation).  sm_103a: operands are staged into shared memory by TMA
// (128-byte swizzle, K-major), multiplied by tcgen05.mma issued from one
// thread with the fp32 accumulator in tensor memory, and read back with
// tcgen05.ld by four epilogue warps that apply C - acc (or +-acc) and round to
// the 16-bit storage format.
//
// CTA = 6 warps: warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs,
// warps 2..5 run the epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
// Tile 128 x 128, K staged 128 bytes per row per stage.  The E4M3 variant
// keeps one TMEM accumulator per 128-deep K slice and folds them with the
// per-tile scales in the epilogue.
//
// Every wait is bounded (kSpinLimit polls, kWaitNs of wall time); a wait that runs out sets
// kErrTimeout in the status word, skips the remaining work and still frees
// tensor memory before the CTA exits.
#include "internal.h"

#include <cudaTypedefs.h>

#include <mutex>

namespace hpmxp {
namespace {

constexpr int kBM = 128, kBN = 128;
constexpr int kRowBytes = 128;                       // K bytes per row per stage (one swizzle atom)
constexpr int kStageA = kBM * kRowBytes;             // 16 KiB
constexpr int kStageB = kBN * kRowBytes;             // 16 KiB
constexpr int kThreads = 192;

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 1; i < kSpinLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ inline void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ inline void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
}
__device__ inline void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Arrive on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ inline void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ inline void tc_mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ inline void tc_mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane.  The wait takes the
// registers as operands so no use of them can be scheduled before it.
__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), leading byte
// offset unused for this layout (set to 16 bytes), descriptor version 1.
__device__ inline uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: fp32 accumulator, K-major A and B, M = 128, N = 128.
// Operand format code: kind::f16 -> 0 F16, 1 BF16; kind::f8f6f4 -> 0 E4M3.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt_code) {
  return (1u << 4) | (fmt_code << 7) | (fmt_code << 10) | ((uint32_t)(kBN >> 3) << 17) |
         ((uint32_t)(kBM >> 4) << 24);
}

struct TcParams {
  int M, N, nkb;        // rows, columns, K stages (128 bytes of K each)
  int mode;
  float sign;
  int fmt;
  int fp8;              // E4M3 operands: one accumulator per stage (= 128-deep slice)
  uint32_t ncols;       // TMEM columns allocated
  uint16_t* C; int64_t ldc;
  uint16_t* R; int64_t ldr;
  const float* sA; int sa_ld;
  const float* sB; int sb_ld;
  uint32_t* status;
};

template <int kStages>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);   // swizzle atoms need 1024-byte alignment
  const uint32_t sA = smem_u32(smem);
  const uint32_t sB = sA + kStages * kStageA;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * (kStageA + kStageB));
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(kStages + s); };
  const uint32_t done = bar0 + 8u * (uint32_t)(2 * kStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
    mbar_init(done, 1);
    fence_mbar_init();
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), p.ncols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: stage s holds K bytes [128 kb, 128 kb + 128) of A and B
      const int kx = kRowBytes / 2;   // the maps count K in 16-bit units: 64 per 128-byte stage
      int issued = 0;
      bool ok = true;
      for (int kb = 0; kb < p.nkb && ok; ++kb) {
        const int s = kb % kStages, use = kb / kStages;
        if (use > 0 && !mbar_wait(empty(s), (uint32_t)((use - 1) & 1))) { ok = false; break; }
        mbar_expect_tx(full(s), kStageA + kStageB);
        tma_load_2d(sA + s * kStageA, &tmA, kb * kx, m0, full(s));
        tma_load_2d(sB + s * kStageB, &tmB, kb * kx, n0, full(s));
        ++issued;
      }
      if (!ok) atomicOr(p.status, kErrTimeout);
      // drain: the last load of every stage has landed before the CTA can exit
      for (int kb = max(0, issued - kStages); kb < issued; ++kb)
        if (!mbar_wait(full(kb % kStages), (uint32_t)((kb / kStages) & 1))) atomicOr(p.status, kErrTimeout);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = p.fp8 ? make_idesc(0) : make_idesc(p.fmt == kBF16 ? 1u : 0u);
      bool ok = true;
      for (int kb = 0; kb < p.nkb; ++kb) {
        const int s = kb % kStages, use = kb / kStages;
        if (!mbar_wait(full(s), (uint32_t)(use & 1))) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (p.fp8 ? (uint32_t)(kb * kBN) : 0u);
        for (int kk = 0; kk < 4; ++kk) {   // 4 MMAs of 32 bytes of K each
          const uint64_t a = sdesc_sw128(sA + s * kStageA + kk * 32);
          const uint64_t b = sdesc_sw128(sB + s * kStageB + kk * 32);
          const uint32_t acc = p.fp8 ? (kk > 0) : (kb > 0 || kk > 0);
          if (p.fp8) tc_mma_f8(d, a, b, idesc, acc);
          else tc_mma_f16(d, a, b, idesc, acc);
        }
        tc_commit(empty(s));   // the stage is free once these MMAs have read it
      }
      if (!ok) atomicOr(p.status, kErrTimeout);
      tc_commit(done);
    }
  } else {
    // epilogue: this warp's 32 TMEM lanes are rows m0 + 32 q + lane
    const int q = warp & 3;
    const int64_t row = (int64_t)m0 + 32 * q + lane;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0));   // warp-uniform for tcgen05.ld
    tc_fence_after();
    if (!ok) {
      if (lane == 0) atomicOr(p.status, kErrTimeout);
    } else {
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
      float sc[4] = {1.0f, 1.0f, 1.0f, 1.0f};
      if (p.fp8)
        for (int g = 0; g < p.nkb && g < 4; ++g)
          sc[g] = __fmul_rn(p.sA[(m0 / 128) * p.sa_ld + g], p.sB[(n0 / 128) * p.sb_ld + g]);
      for (int c0 = 0; c0 < kBN; c0 += 16) {
        float acc[16];
        uint32_t r[16];
        if (p.fp8) {
          for (int v = 0; v < 16; ++v) acc[v] = 0.0f;
          for (int g = 0; g < p.nkb; ++g) {
            tmem_ld16(lane_addr + (uint32_t)(g * kBN + c0), r);
            for (int v = 0; v < 16; ++v) acc[v] = __fmaf_rn(__uint_as_float(r[v]), sc[g], acc[v]);
          }
        } else {
          tmem_ld16(lane_addr + (uint32_t)c0, r);
          for (int v = 0; v < 16; ++v) acc[v] = __uint_as_float(r[v]);
        }
        if (row < p.M) {
          for (int v = 0; v < 16; ++v) {
            const int64_t col = (int64_t)n0 + c0 + v;
            if (col >= p.N) break;
            uint16_t* cp = p.C ? p.C + row + col * p.ldc : nullptr;
            float out;
            if (p.mode == kEpiSub) out = __fsub_rn(u16_to_f32(*cp, p.fmt), acc[v]);
            else out = p.sign * acc[v];
            const uint16_t h = f32_to_u16(out, p.fmt);
            if (cp) *cp = h;
            if (p.R) p.R[row * p.ldr + col] = h;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, p.ncols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 2-D K-major operand: `rows` rows of `k_bytes` bytes, consecutive rows
// `ld_bytes` apart; box = 128 rows x 128 bytes, 128-byte swizzle, zero fill
// outside the operand.
bool make_operand_map(CUtensorMap* tm, const void* base, uint64_t k_bytes, uint64_t rows, uint64_t ld_bytes) {
  auto fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) || (ld_bytes & 15) || (k_bytes % kRowBytes)) return false;
  cuuint64_t dims[2] = {k_bytes / 2, rows};
  cuuint64_t strides[1] = {ld_bytes};
  cuuint32_t box[2] = {kRowBytes / 2, 128};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int kStages>
size_t smem_bytes_for() { return 1024 + (size_t)kStages * (kStageA + kStageB) + 8 * (2 * kStages + 1) + 16; }

template <int kStages>
cudaError_t launch(const CUtensorMap& a, const CUtensorMap& b, const TcParams& p, size_t smem, double flops,
                   cudaStream_t st) {
  static int configured_for = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_for != dev) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(200 * 1024));
    if (e != cudaSuccess) return e;
    configured_for = dev;
  }
  dim3 grid((unsigned)cdiv(p.N, kBN), (unsigned)cdiv(p.M, kBM));
  void* tok = prof_begin(st);
  gemm_tc_kernel<kStages><<<grid, kThreads, smem, st>>>(a, b, p);
  prof_end(tok, kProfGemm, flops, st);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_tc(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const int esz = g.fp8 ? 1 : 2;
  const uint64_t kbytes = (uint64_t)g.K * esz;
  if (kbytes % kRowBytes) return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_operand_map(&ta, g.A, kbytes, (uint64_t)g.M, (uint64_t)g.lda * esz) ||
      !make_operand_map(&tb, g.B, kbytes, (uint64_t)g.N, (uint64_t)g.ldb * esz))
    return cudaErrorInvalidValue;
  TcParams p{};
  p.M = g.M; p.N = g.N; p.nkb = (int)(kbytes / kRowBytes);
  p.mode = g.mode; p.sign = g.sign; p.fmt = g.fmt; p.fp8 = g.fp8;
  p.C = (uint16_t*)g.C; p.ldc = g.ldc; p.R = (uint16_t*)g.R; p.ldr = g.ldr;
  p.sA = g.sA; p.sa_ld = g.sa_ld; p.sB = g.sB; p.sb_ld = g.sb_ld;
  p.status = g.status;
  if (g.fp8) {
    if (p.nkb > 4) return cudaErrorInvalidValue;   // one 128-column accumulator per slice
    p.ncols = p.nkb <= 1 ? 128u : (p.nkb <= 2 ? 256u : 512u);
  } else {
    p.ncols = 128u;
  }
  // Shared memory also caps residency so that resident CTAs never ask for
  // more than the 512 TMEM columns of an SM at once.
  const int max_res = (int)(512u / p.ncols);
  const size_t floor_smem = max_res >= 3 ? 0 : (max_res == 2 ? 100 * 1024 : 120 * 1024);
  const double flops = 2.0 * g.M * (double)g.N * g.K;
  if (p.nkb <= 2) {
    const size_t smem = std::max(smem_bytes_for<2>(), floor_smem);
    return launch<2>(ta, tb, p, smem, flops, st);
  }
  const size_t smem = std::max(smem_bytes_for<4>(), floor_smem);
  return launch<4>(ta, tb, p, smem, flops, st);
}

}  // namespace hpmxp
