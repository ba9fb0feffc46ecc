// Tensor-core product engine for the LU's panel and Schur-update products
// (section "Algorithmic Framework", Fig. 1: low-precision operands, fp32
// accumulation).  sm_103a: operands are staged into shared memory by TMA
// (128-byte swizzle, K-major), multiplied by tcgen05.mma issued from one
// thread with fp32 accumulators in tensor memory, and read back with
// tcgen05.ld by four epilogue warps.
//
// Persistent kernel, one CTA per SM, TI x 128 output tiles (TI = 128, or 256
// for the large 16-bit products) in a static round-robin order.  The MMA
// computes the TRANSPOSED tile (TMEM lane = output column j, TMEM column =
// output row i) so each epilogue thread owns consecutive rows of one column of
// the column-major output: the C tile is moved by TMA between HBM and
// 128-byte-swizzled shared boxes of 64 rows and the epilogue touches them with
// 16-byte, bank-conflict-free accesses.
//
// Roles: warp 0 TMA producer of the operand ring; warp 1 TMEM owner and MMA
// issuer; warps 2..9 epilogue in two groups of four (warp w reads TMEM lanes
// 32*(w%4)..+31; group g takes rows TI/2 g .. of the tile), which also
// prefetch C tiles ahead and issue the TMA stores.
// Accumulators are double buffered in TMEM (single buffered for 4-slice FP8),
// so the epilogue of one tile overlaps the MMAs of the next.  The E4M3
// variant keeps one accumulator per 128-deep K slice and folds them with the
// per-tile scales in the epilogue.
//
// Every wait is bounded (a poll count and a global-timer limit passed in
// TcParams); a wait that runs out sets kErrTimeout in the status word, skips
// the remaining work and still drains its copies and tensor-core work (with
// the default bound) and frees tensor memory before the CTA exits.  The four
// warps of an epilogue group take each tile's go / give-up decision together,
// so none of them is left waiting at the group's named barrier.
#include "internal.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace hpmxp {
namespace {

constexpr int kTJ = 128;                      // output columns per tile (MMA M, TMEM lanes)
constexpr int kRowBytes = 128;                // K bytes per operand row per stage (one swizzle atom)
constexpr int kStageA = kTJ * kRowBytes;      // MMA A operand: rows j (16 KiB)
constexpr int kCBox = kTJ * 128;              // one C box: 128 bytes of rows x 128 columns (16 KiB)
constexpr int kEpiGroups = 2;                 // epilogue groups, one per half of the tile's rows
constexpr int kEpiThreads = 128;              // threads per epilogue group (one warp per TMEM lane quarter)
constexpr int kThreads = 64 + kEpiGroups * kEpiThreads;

// Tile height TI (output rows i per tile = MMA N): 128, or 256 for the large
// 16-bit products, where every operand byte an SM receives feeds twice the
// flops (the SM's operand intake is what bounds this kernel at K >= 256).
// CB: bytes per C element, 2 (the 16-bit factor storage) or 4 (an fp32
// trailing matrix: C = fl32(C - acc), 128-row tiles only).
template <int TI, int CB = 2>
struct TileCfg {
  static constexpr int kStages = TI == 128 ? 4 : 3;
  static constexpr int kStageB = TI * kRowBytes;            // MMA B operand: rows i (16 or 32 KiB)
  static constexpr int kBoxRows = 128 / CB;                 // rows of one 128-byte C box: 64 or 32
  static constexpr int kBoxes = TI / 2 / kBoxRows;          // C boxes per epilogue group
  static constexpr int kCTile = kEpiGroups * kBoxes * kCBox;  // 32, 64 KiB (16-bit) or 64 KiB (fp32)
  // C tile buffers: with three, one is in the epilogue, one being stored and
  // one loading; the 256-row and the fp32 tiles have room for one only
  static constexpr int kCBufs = (TI == 128 && CB == 2) ? 3 : 1;
  static constexpr int kAhead = kCBufs >= 2 ? kCBufs - 1 : 1;   // C prefetch distance (local tiles)
  static constexpr int kReadWait = kCBufs >= 2 ? kCBufs - 2 : 0; // stores allowed to be still reading
  static constexpr size_t kSmem = 1024 + (size_t)kStages * (kStageA + kStageB) + (size_t)kCBufs * kCTile +
                                  8 * (2 * kStages + 5 + 2 * kCBufs) + 16;
};
// 227 KB of dynamic shared memory per CTA; two TI-column fp32 accumulators in
// the 512 TMEM columns; a TMA box is at most 256 rows
static_assert(TileCfg<128>::kSmem <= 232448 && TileCfg<256>::kSmem <= 232448 && TileCfg<128, 4>::kSmem <= 232448,
              "shared memory per CTA");
template <int TI>
constexpr bool tile_fits() { return 2 * TI <= 512 && TI <= 256 && TI % 128 == 0; }
static_assert(tile_fits<128>() && tile_fits<256>(), "two accumulators in TMEM, one TMA box per stage");

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
// Bounded wait for the phase with the given parity to complete: at most
// `polls` polls and `ns` nanoseconds (the defaults for the drain waits).
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, long long polls = kSpinLimit,
                                 unsigned long long ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 1; i < polls; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 0 && global_ns() - t0 > ns) return false;
  }
  return false;
}

__device__ inline void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ inline void tma_store_2d(const CUtensorMap* tm, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"((uint64_t)tm), "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ inline void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ inline void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ inline void epi_barrier(int group) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "n"(kEpiThreads) : "memory");
}
// True for every thread of the epilogue group when v is true for all of them
// (a barrier of the group's four warps with an AND reduction).
__device__ inline bool epi_all(int group, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + group), "n"(kEpiThreads)
      : "memory");
  return r != 0;
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

// 64 consecutive fp32 columns: two x32 loads in flight, one wait.
__device__ inline void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
#define HPMXP_LD32(OFF, B)                                                                                       \
  asm volatile(                                                                                                \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, " \
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"            \
      : "=r"(r[B + 0]), "=r"(r[B + 1]), "=r"(r[B + 2]), "=r"(r[B + 3]), "=r"(r[B + 4]), "=r"(r[B + 5]),         \
        "=r"(r[B + 6]), "=r"(r[B + 7]), "=r"(r[B + 8]), "=r"(r[B + 9]), "=r"(r[B + 10]), "=r"(r[B + 11]),       \
        "=r"(r[B + 12]), "=r"(r[B + 13]), "=r"(r[B + 14]), "=r"(r[B + 15]), "=r"(r[B + 16]), "=r"(r[B + 17]),   \
        "=r"(r[B + 18]), "=r"(r[B + 19]), "=r"(r[B + 20]), "=r"(r[B + 21]), "=r"(r[B + 22]), "=r"(r[B + 23]),   \
        "=r"(r[B + 24]), "=r"(r[B + 25]), "=r"(r[B + 26]), "=r"(r[B + 27]), "=r"(r[B + 28]), "=r"(r[B + 29]),   \
        "=r"(r[B + 30]), "=r"(r[B + 31])                                                                        \
      : "r"(taddr + OFF))
  HPMXP_LD32(0u, 0);
  HPMXP_LD32(32u, 32);
#undef HPMXP_LD32
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]),
                 "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]), "+r"(r[42]),
                 "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]), "+r"(r[49]),
                 "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]), "+r"(r[56]),
                 "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])
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

// Instruction descriptor: fp32 accumulator, K-major A and B, M = 128, N = TI.
// Operand format code: kind::f16 -> 0 F16, 1 BF16; kind::f8f6f4 -> 0 E4M3.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt_code, int ti) {
  return (1u << 4) | (fmt_code << 7) | (fmt_code << 10) | ((uint32_t)(ti >> 3) << 17) |
         ((uint32_t)(kTJ >> 4) << 24);
}

struct TcParams {
  int M, N, nkb;          // output rows, columns, K stages (128 bytes of K each)
  int tiles_i, ntiles;
  int mode;
  float sign;
  int fmt;
  int fp8;                // E4M3 operands: one accumulator per stage (= 128-deep slice)
  int nbuf;               // TMEM accumulator buffers (1 or 2)
  uint32_t acc_cols;      // TMEM columns per accumulator buffer
  uint32_t ncols;         // TMEM columns allocated
  int has_c;              // write (and for kEpiSub read) the column-major C through tmC
  uint16_t* R; int64_t ldr;
  const float* sA; int sa_ld;
  const float* sB; int sb_ld;
  uint32_t* status;
  long long wait_polls;            // bound of the pipeline waits (the drain waits keep the defaults)
  unsigned long long wait_ns;
  // measurement: [0] the earliest CTA start after the stream dependency, [1]
  // all-ones minus the latest CTA end (global timer, ns; both kept by
  // atomicMin from all-ones), NULL when not measured
  unsigned long long* span;
};

// Two floats rounded to nearest even into one 32-bit word of 16-bit values (lo
// in the low half): one packed conversion instruction.
__device__ inline uint32_t pack16x2(float lo, float hi, int fmt) {
  uint32_t r;
  if (fmt == kBF16) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Where tile t of the launch is: its product's tensor maps, its output origin
// and that product's bounds (one product, or the items of a grouped launch).
struct TileLoc {
  const CUtensorMap* a;
  const CUtensorMap* b;
  const CUtensorMap* c;
  int i0, j0, M, N;
  uint16_t* R;
  int64_t ldr;
};

template <int TI, int CB>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, TcParams p, const GemmGroupItem* __restrict__ items,
               int nitems) {
  using Cfg = TileCfg<TI, CB>;
  constexpr int kStages = Cfg::kStages, kStageB = Cfg::kStageB, kCTile = Cfg::kCTile, kCBufs = Cfg::kCBufs;
  constexpr int kBoxes = Cfg::kBoxes, kBoxRows = Cfg::kBoxRows;
  constexpr int kSegs = TI / 128;   // 64-row segments of an epilogue group's TI/2 rows
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);   // swizzle atoms need 1024-byte alignment
  const uint32_t sOpA = smem_u32(smem);                            // [kStages][rows j][128 B]
  const uint32_t sOpB = sOpA + kStages * kStageA;                  // [kStages][rows i][128 B]
  const uint32_t sC = sOpB + kStages * kStageB;                    // [kCBufs][group][box][cols j][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * (kStageA + kStageB) + kCBufs * kCTile);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(kStages + s); };
  auto acc_full = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kStages + b); };
  auto acc_empty = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kStages + 2 + b); };
  auto c_full = [&](int b, int h) { return bar0 + 8u * (uint32_t)(2 * kStages + 4 + 2 * b + h); };
  const uint32_t mma_drain = bar0 + 8u * (uint32_t)(2 * kStages + 4 + 2 * kCBufs);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5 + 2 * kCBufs);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // tile t -> its product (grouped launch: the last item starting at or before t)
  auto locate = [&](int t) {
    TileLoc L;
    if (items == nullptr) {
      L.a = &tmA; L.b = &tmB; L.c = &tmC;
      L.i0 = (t % p.tiles_i) * TI; L.j0 = (t / p.tiles_i) * kTJ;
      L.M = p.M; L.N = p.N; L.R = p.R; L.ldr = p.ldr;
    } else {
      int lo = 0, hi = nitems - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
      }
      const GemmGroupItem& g = items[lo];
      const int lt = t - g.tile_begin;
      L.a = reinterpret_cast<const CUtensorMap*>(g.maps[0]);
      L.b = reinterpret_cast<const CUtensorMap*>(g.maps[1]);
      L.c = reinterpret_cast<const CUtensorMap*>(g.maps[2]);
      L.i0 = (lt % g.tiles_i) * TI; L.j0 = (lt / g.tiles_i) * kTJ;
      L.M = g.M; L.N = g.N; L.R = (uint16_t*)g.R; L.ldr = g.ldr;
    }
    return L;
  };
  // the items' tensor maps were written to global memory before the launch:
  // acquire them for the tensor-map proxy before the first TMA through them
  auto acquire_maps = [&](int which) {
    for (int it = 0; items != nullptr && it < nitems; ++it)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)items[it].maps[which])
                   : "memory");
  };

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), kEpiGroups * kEpiThreads / 32);
    }
    for (int b = 0; b < kCBufs; ++b) {
      mbar_init(c_full(b, 0), 1);
      mbar_init(c_full(b, 1), 1);
    }
    mbar_init(mma_drain, 1);
    fence_mbar_init();
    if (items == nullptr) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      if (p.has_c) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmC) : "memory");
    }
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), p.ncols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // the setup above may run while the previous kernel of the stream finishes;
  // no global memory is touched before it has completed
  pdl_wait();
  pdl_trigger();
  if (p.span && threadIdx.x == 0) atomicMin(p.span, global_ns());

  if (warp == 0) {
    if (lane == 0) {
      // operand ring: stage s holds K bytes [128 kb, +128) of the tile's rows j (A) and rows i (B)
      long long pos = 0;   // ring position over all tiles of this CTA
      bool ok = true;
      acquire_maps(0);
      acquire_maps(1);
      for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
        const TileLoc L = locate(t);
        const int i0 = L.i0, j0 = L.j0;
        for (int kb = 0; kb < p.nkb; ++kb, ++pos) {
          const int s = (int)(pos % kStages);
          const long long use = pos / kStages;
          if (use > 0 && !mbar_wait(empty(s), (uint32_t)((use - 1) & 1), p.wait_polls, p.wait_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full(s), kStageA + kStageB);
          tma_load_2d(sOpA + s * kStageA, L.b, kb * (kRowBytes / 2), j0, full(s));
          tma_load_2d(sOpB + s * kStageB, L.a, kb * (kRowBytes / 2), i0, full(s));
        }
      }
      if (!ok) atomicOr(p.status, kErrTimeout);
      // drain: the last load of every stage has landed before the CTA can exit
      for (long long q = (pos > kStages ? pos - kStages : 0); q < pos; ++q)
        if (!mbar_wait(full((int)(q % kStages)), (uint32_t)((q / kStages) & 1))) atomicOr(p.status, kErrTimeout);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = p.fp8 ? make_idesc(0, TI) : make_idesc(p.fmt == kBF16 ? 1u : 0u, TI);
      long long pos = 0;
      bool ok = true;
      int local = 0;
      for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x, ++local) {
        const int ab = local % p.nbuf, ause = local / p.nbuf;
        if (ause > 0 && !mbar_wait(acc_empty(ab), (uint32_t)((ause - 1) & 1), p.wait_polls, p.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)ab * p.acc_cols;
        for (int kb = 0; kb < p.nkb; ++kb, ++pos) {
          const int s = (int)(pos % kStages);
          if (!mbar_wait(full(s), (uint32_t)((pos / kStages) & 1), p.wait_polls, p.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = d0 + (p.fp8 ? (uint32_t)(kb * TI) : 0u);
          for (int kk = 0; kk < 4; ++kk) {   // 4 MMAs of 32 bytes of K each
            const uint64_t a = sdesc_sw128(sOpA + s * kStageA + kk * 32);
            const uint64_t b = sdesc_sw128(sOpB + s * kStageB + kk * 32);
            const uint32_t acc = p.fp8 ? (kk > 0) : (kb > 0 || kk > 0);
            if (p.fp8) tc_mma_f8(d, a, b, idesc, acc);
            else tc_mma_f16(d, a, b, idesc, acc);
          }
          tc_commit(empty(s));   // the stage is free once these MMAs have read it
        }
        tc_commit(acc_full(ab));
      }
      if (!ok) atomicOr(p.status, kErrTimeout);
      // every MMA issued has completed before TMEM is freed, also when an
      // epilogue group gave up before the last accumulator was written
      tc_commit(mma_drain);
      if (!mbar_wait(mma_drain, 0)) atomicOr(p.status, kErrTimeout);
    }
  } else {
    // epilogue: group g = (warp - 2) / 4 owns rows i0 + (TI/2) g .. + TI/2 - 1 of the
    // tile, as kBoxes C boxes of 64 rows; thread = output column j = j0 + jl,
    // jl = 32 q + lane (its TMEM lane)
    const int q = warp & 3;
    const int g = (warp - 2) >> 2;
    const int jl = 32 * q + lane;
    const bool leader = ((warp - 2) & 3) == 0 && lane == 0;
    const bool load_c = p.has_c && p.mode == kEpiSub;
    // C tile buffers rotate over local tiles: tile l uses buffer l % kCBufs.
    // With three buffers the C of tile l + 2 is loaded into the buffer of tile
    // l - 1 as soon as the store of tile l - 1 has been read, which is checked
    // one tile later, when it is long done, so the epilogue never waits on its
    // own store; with one buffer the C of tile l + 1 follows the store of l.
    int issued_c[kCBufs];         // local tile whose C load is outstanding in each buffer
    for (int b = 0; b < kCBufs; ++b) issued_c[b] = -1;
    auto load_c_tile = [&](int tt, int b) {   // this group's boxes of tile tt's C into buffer b
      const TileLoc Lc = locate(tt);
      mbar_expect_tx(c_full(b, g), kBoxes * kCBox);
#pragma unroll
      for (int h = 0; h < kBoxes; ++h)
        tma_load_2d(sC + b * kCTile + (g * kBoxes + h) * kCBox, Lc.c, Lc.i0 + (TI / 2) * g + kBoxRows * h, Lc.j0,
                    c_full(b, g));
    };
    if (leader && p.has_c) acquire_maps(2);
    if (leader && load_c) {       // prefetch the C of the first kAhead local tiles
      int local = 0;
      for (int t = blockIdx.x; t < p.ntiles && local < Cfg::kAhead; t += gridDim.x, ++local) {
        load_c_tile(t, local % kCBufs);
        issued_c[local % kCBufs] = local;
      }
    }
    bool ok = true;
    int local = 0;
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++local) {
      const TileLoc L = locate(t);
      const int i0 = L.i0, j0 = L.j0;
      const int cb = local % kCBufs, ab = local % p.nbuf;
      bool w = true;
      if (load_c) w = mbar_wait(c_full(cb, g), (uint32_t)((local / kCBufs) & 1), p.wait_polls, p.wait_ns);
      w = w && mbar_wait(acc_full(ab), (uint32_t)((local / p.nbuf) & 1), p.wait_polls, p.wait_ns);
      // one decision for the whole group (warp-uniform for tcgen05.ld, and no
      // warp of the group left behind at its named barrier)
      w = epi_all(g, w);
      if (!w) { ok = false; break; }
      if (leader) issued_c[cb] = -1;
      tc_fence_after();
      const uint32_t lane_base = tmem + (uint32_t)ab * p.acc_cols + ((uint32_t)(32 * q) << 16) + (TI / 2) * g;
      float sc[4] = {1.0f, 1.0f, 1.0f, 1.0f};
      if (p.fp8)
        for (int s2 = 0; s2 < p.nkb && s2 < 4; ++s2)
          sc[s2] = __fmul_rn(p.sA[(i0 / 128) * p.sa_ld + s2], p.sB[(j0 / 128) * p.sb_ld + s2]);
      const int64_t j = (int64_t)j0 + jl;
      // one buffer, no C to load: the buffer's previous store was read (the
      // leader waited for it before it reached this barrier)
      if (kCBufs == 1 && p.has_c && !load_c) epi_barrier(g);
#pragma unroll 1
      for (int h = 0; h < kSegs; ++h) {   // 64-row segments of the group's rows
        const uint32_t lane_addr = lane_base + 64u * h;
        float acc[64];
        {
          uint32_t r[64];
          if (p.fp8) {
#pragma unroll
            for (int v = 0; v < 64; ++v) acc[v] = 0.0f;
            for (int s2 = 0; s2 < p.nkb; ++s2) {
              tmem_ld64(lane_addr + (uint32_t)(s2 * TI), r);
#pragma unroll
              for (int v = 0; v < 64; ++v) acc[v] = __fmaf_rn(__uint_as_float(r[v]), sc[s2], acc[v]);
            }
          } else {
            tmem_ld64(lane_addr, r);
#pragma unroll
            for (int v = 0; v < 64; ++v) acc[v] = __uint_as_float(r[v]);
          }
        }
        if (h == kSegs - 1) {
          // accumulator buffer free for the MMA warp as soon as it is in registers
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty(ab));
        }
        if constexpr (CB == 4) {
          // fp32 C: two 32-row boxes; rows 32 q + 4 c8 .. +3 of column j in chunk c8 of box q
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const uint32_t row_addr = sC + cb * kCTile + (g * kBoxes + 2 * h + q) * kCBox + jl * 128;
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
              const uint32_t ad = row_addr + ((c8 ^ (jl & 7)) << 4);
              float cf[4];
              asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                           : "=f"(cf[0]), "=f"(cf[1]), "=f"(cf[2]), "=f"(cf[3]) : "r"(ad) : "memory");
#pragma unroll
              for (int v = 0; v < 4; ++v) cf[v] = __fsub_rn(cf[v], acc[32 * q + 4 * c8 + v]);
              asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                           ::"r"(ad), "f"(cf[0]), "f"(cf[1]), "f"(cf[2]), "f"(cf[3]) : "memory");
            }
          }
        } else {
        // rows i0 + (TI/2) g + 64 h + 8 ch .. +7 of column j: eight 16-byte chunks of the swizzled box
        const uint32_t cbox = sC + cb * kCTile + (g * kBoxes + h) * kCBox;
        const uint32_t row_addr = cbox + jl * 128;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const uint32_t ad = row_addr + ((ch ^ (jl & 7)) << 4);
          uint32_t outw[4];
          if (p.mode == kEpiSub) {
            uint32_t cw[4];
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(cw[0]), "=r"(cw[1]), "=r"(cw[2]), "=r"(cw[3]) : "r"(ad) : "memory");
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const float lo = __fsub_rn(u16_to_f32((uint16_t)(cw[v] & 0xffffu), p.fmt), acc[8 * ch + 2 * v]);
              const float hi = __fsub_rn(u16_to_f32((uint16_t)(cw[v] >> 16), p.fmt), acc[8 * ch + 2 * v + 1]);
              outw[v] = pack16x2(lo, hi, p.fmt);
            }
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              outw[v] = pack16x2(p.sign * acc[8 * ch + 2 * v], p.sign * acc[8 * ch + 2 * v + 1], p.fmt);
          }
          if (p.has_c)
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                         ::"r"(ad), "r"(outw[0]), "r"(outw[1]), "r"(outw[2]), "r"(outw[3]) : "memory");
          if (L.R && j < L.N) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const int64_t i = (int64_t)i0 + (TI / 2) * g + 64 * h + 8 * ch + v;
              if (i < L.M) L.R[i * L.ldr + j] = (uint16_t)((outw[v >> 1] >> ((v & 1) * 16)) & 0xffffu);
            }
          }
        }
        }
      }
      if (p.has_c) {
        fence_async_smem();
        epi_barrier(g);
        if (leader) {
#pragma unroll
          for (int h = 0; h < kBoxes; ++h)
            tma_store_2d(L.c, i0 + (TI / 2) * g + kBoxRows * h, j0, sC + cb * kCTile + (g * kBoxes + h) * kCBox);
          bulk_commit();
          // the stores issued kCBufs - 1 tiles ago (one buffer: this tile's)
          // have finished reading their buffer, which now receives the C of
          // the tile kAhead ahead
          asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(Cfg::kReadWait) : "memory");
          const int t2 = t + Cfg::kAhead * (int)gridDim.x;
          if (load_c && t2 < p.ntiles) {
            const int b2 = (local + Cfg::kAhead) % kCBufs;
            load_c_tile(t2, b2);
            issued_c[b2] = local + Cfg::kAhead;
          }
        }
      }
    }
    if (!ok && lane == 0) atomicOr(p.status, kErrTimeout);
    if (leader) {
      bulk_wait0();
      // C loads issued for tiles this CTA did not reach (error path) land before exit
      for (int b = 0; b < kCBufs; ++b)
        if (issued_c[b] >= 0 && !mbar_wait(c_full(b, g), (uint32_t)((issued_c[b] / kCBufs) & 1)))
          atomicOr(p.status, kErrTimeout);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, p.ncols);
  }
  if (p.span && threadIdx.x == 0) atomicMin(p.span + 1, ~global_ns());
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

// 2-D map over 16-bit (or, with u32, 32-bit) units: `rows` rows of `inner`
// units, consecutive rows `ld_bytes` apart, box = box_inner x box_rows,
// 128-byte swizzle, zero fill outside the matrix.
bool make_map(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t rows, uint64_t ld_bytes,
              uint32_t box_inner, uint32_t box_rows, bool u32 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) || (ld_bytes & 15) || inner == 0 || rows == 0) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld_bytes};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, u32 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base),
            dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// persistent grid size: the SM count, or the calling thread's SM budget
int grid_cap() {
  const int b = sm_budget();
  return b > 0 ? std::min(b, num_sms()) : num_sms();
}

}  // namespace

namespace {

template <int TI, int CB = 2>
cudaError_t gemm_tc_tiles(const GemmArgs& g, cudaStream_t st) {
  using Cfg = TileCfg<TI, CB>;
  static_assert(CB == 2 || TI == 128, "fp32 C on 128-row tiles only");
  if (CB == 4 && (g.mode != kEpiSub || g.R || !g.C)) return cudaErrorInvalidValue;
  const int esz = g.fp8 ? 1 : 2;
  const uint64_t kbytes = (uint64_t)g.K * esz;
  if (kbytes % kRowBytes) return cudaErrorInvalidValue;
  CUtensorMap ta, tb, tc;
  if (!make_map(&ta, g.A, kbytes / 2, (uint64_t)g.M, (uint64_t)g.lda * esz, kRowBytes / 2, TI) ||
      !make_map(&tb, g.B, kbytes / 2, (uint64_t)g.N, (uint64_t)g.ldb * esz, kRowBytes / 2, kTJ))
    return cudaErrorInvalidValue;
  TcParams p{};
  p.has_c = g.C != nullptr;
  if (p.has_c) {
    // column-major C: inner = rows; box = 128 bytes of rows (64 16-bit or 32 fp32) x 128 columns
    if (!make_map(&tc, g.C, (uint64_t)g.M, (uint64_t)g.N, (uint64_t)g.ldc * CB, Cfg::kBoxRows, kTJ, CB == 4))
      return cudaErrorInvalidValue;
  } else {
    tc = ta;   // never dereferenced
  }
  p.M = g.M; p.N = g.N; p.nkb = (int)(kbytes / kRowBytes);
  p.tiles_i = cdiv(g.M, TI);
  p.ntiles = p.tiles_i * cdiv(g.N, kTJ);
  p.mode = g.mode; p.sign = g.sign; p.fmt = g.fmt; p.fp8 = g.fp8;
  p.R = (uint16_t*)g.R; p.ldr = g.ldr;
  p.sA = g.sA; p.sa_ld = g.sa_ld; p.sB = g.sB; p.sb_ld = g.sb_ld;
  p.status = g.status;
  const WaitBudget wb = wait_budget();
  p.wait_polls = wb.polls;
  p.wait_ns = wb.ns;
  if (g.fp8) {
    if (TI != 128 || p.nkb > 4) return cudaErrorInvalidValue;   // one 128-column accumulator per slice
    p.acc_cols = (uint32_t)(TI * p.nkb);
  } else {
    p.acc_cols = TI;
  }
  p.nbuf = (2 * p.acc_cols <= 512u) ? 2 : 1;
  uint32_t need = p.acc_cols * (uint32_t)p.nbuf, ncols = 32;
  while (ncols < need) ncols <<= 1;
  p.ncols = ncols;

  static std::atomic<int> configured_for{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_for.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<TI, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    configured_for.store(dev);
  }
  const int grid = std::min(p.ntiles, g.max_ctas > 0 ? std::min(g.max_ctas, grid_cap()) : grid_cap());
  const double flops = 2.0 * g.M * (double)g.N * g.K;
  // algorithmic DRAM bytes: both operands once, C read (subtract mode) and
  // written once, the optional row-major copy written once
  const double mn = (double)g.M * (double)g.N;
  const double bytes = ((double)g.M + (double)g.N) * (double)g.K * esz +
                       (p.has_c ? mn * CB * (g.mode == kEpiSub ? 2.0 : 1.0) : 0.0) + (g.R ? mn * 2.0 : 0.0);
  void* tok = prof_begin(st);
  p.span = prof_device_span(tok);
  const cudaError_t e =
      launch_pdl(gemm_tc_kernel<TI, CB>, dim3(grid), dim3(kThreads), Cfg::kSmem, st, ta, tb, tc, p,
                 (const GemmGroupItem*)nullptr, 0);
  prof_end(tok, g.mode == kEpiSub ? kProfGemm : kProfGemmStore, flops, st, bytes);
  count_launches(1);
  return e;
}

}  // namespace

bool gemm_group_encode(const GemmArgs* gs, int count, GemmGroupItem* items, int* total_tiles) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  int tiles = 0;
  for (int c = 0; c < count; ++c) {
    const GemmArgs& g = gs[c];
    if (g.fp8 || g.c32 || g.K <= 0 || g.K >= 256 || (g.K % 128) || g.K != gs[0].K || g.mode != gs[0].mode ||
        (!g.R) != (!gs[0].R) || !g.C || g.M <= 0 || g.N <= 0)
      return false;
    const uint64_t kbytes = (uint64_t)g.K * 2;
    CUtensorMap* ta = reinterpret_cast<CUtensorMap*>(items[c].maps[0]);
    CUtensorMap* tb = reinterpret_cast<CUtensorMap*>(items[c].maps[1]);
    CUtensorMap* tc = reinterpret_cast<CUtensorMap*>(items[c].maps[2]);
    if (!make_map(ta, g.A, kbytes / 2, (uint64_t)g.M, (uint64_t)g.lda * 2, kRowBytes / 2, 128) ||
        !make_map(tb, g.B, kbytes / 2, (uint64_t)g.N, (uint64_t)g.ldb * 2, kRowBytes / 2, kTJ) ||
        !make_map(tc, g.C, (uint64_t)g.M, (uint64_t)g.N, (uint64_t)g.ldc * 2, 64, kTJ))
      return false;
    items[c].M = g.M;
    items[c].N = g.N;
    items[c].tiles_i = cdiv(g.M, 128);
    items[c].tile_begin = tiles;
    items[c].R = g.R;
    items[c].ldr = g.ldr;
    tiles += items[c].tiles_i * cdiv(g.N, kTJ);
  }
  *total_tiles = tiles;
  return true;
}

cudaError_t gemm_tc_grouped(const GemmArgs& g, const GemmGroupItem* dev_items, int nitems, int total_tiles,
                            cudaStream_t st, double flops, double bytes) {
  using Cfg = TileCfg<128, 2>;
  if (nitems <= 0 || total_tiles <= 0) return cudaSuccess;
  TcParams p{};
  p.has_c = 1;
  p.nkb = (int)((uint64_t)g.K * 2 / kRowBytes);
  p.tiles_i = 1;
  p.ntiles = total_tiles;
  p.mode = g.mode; p.sign = g.sign; p.fmt = g.fmt; p.fp8 = 0;
  p.status = g.status;
  const WaitBudget wb = wait_budget();
  p.wait_polls = wb.polls;
  p.wait_ns = wb.ns;
  p.acc_cols = 128;
  p.nbuf = 2;
  p.ncols = 256;
  static std::atomic<int> configured_for{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_for.load() != dev) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    configured_for.store(dev);
  }
  const int grid = std::min(total_tiles, g.max_ctas > 0 ? std::min(g.max_ctas, grid_cap()) : grid_cap());
  CUtensorMap none;
  memset(&none, 0, sizeof(none));   // the items' maps are used instead
  void* tok = prof_begin(st);
  p.span = prof_device_span(tok);
  const cudaError_t e = launch_pdl(gemm_tc_kernel<128, 2>, dim3(grid), dim3(kThreads), Cfg::kSmem, st, none, none,
                                   none, p, dev_items, nitems);
  prof_end(tok, g.mode == kEpiSub ? kProfGemm : kProfGemmStore, flops, st, bytes);
  count_launches(1);
  return e;
}

namespace {

// A tile height of 128 (hpmxp_set_tuning or HPMXP_GEMM_TILE=128) keeps every
// product on the 128-row tile.
bool wide_tiles_enabled() { return tuning().gemm_tile != 128; }

}  // namespace

cudaError_t gemm_tc(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.c32) return g.fp8 ? cudaErrorInvalidValue : gemm_tc_tiles<128, 4>(g, st);
  // 256-row tiles for the 16-bit products that fill them (M >= 256) and have
  // enough depth (K >= 256) for one C buffer to keep up
  if (!g.fp8 && g.M >= 256 && g.K >= 256 && wide_tiles_enabled()) return gemm_tc_tiles<256>(g, st);
  return gemm_tc_tiles<128>(g, st);
}

}  // namespace hpmxp
