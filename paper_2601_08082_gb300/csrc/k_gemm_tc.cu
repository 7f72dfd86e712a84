// FP16 tensor-core GEMM for the low-precision off-diagonal levels (Sec. 3.3):
// C_master -= scale * X Y^T with X, Y read from the row-major FP16 shadow of L by TMA,
// multiplied by tcgen05.mma (kind::f16, FP32 accumulation in TMEM) and applied to the
// FP64 master in the epilogue.  This is Alg. 2's GEMM update of B2 by B1 L21^T and Alg. 3's
// update of C21 by A2 A1^T at an FP16 level; with
// `lower` it is the leaf SYRK of Alg. 3 (entries above the diagonal are skipped, and
// tiles entirely above it are never computed).
//
// The same kernels run the FP32 levels on tensor cores by the error-corrected
// TF32 split (Ootomo and Yokota, 2022): each FP32 operand is stored as hi = tf32(x) and
// lo = tf32(x - hi) (row-major FP32 arrays written once per finished block of L); per K
// slice the MMA warp issues hi hi^T into one TMEM accumulator and hi lo^T + lo hi^T into a
// second (kind::tf32, FP32 accumulation), and the epilogue subtracts their sum in FP64.
// Keeping the small correction terms in their own accumulator keeps them from being
// rounded away against the large one.
//
// One CTA computes one 128 x BN tile.  Warp roles: warp 0 issues TMA loads into a
// STAGES-deep ring of 128B-swizzled K-major tiles, warp 1 owns the TMEM allocation and
// issues the MMAs (one elected thread), warps 2-5 read the accumulator back with
// tcgen05.ld and update the master.  Every mbarrier wait is bounded by %globaltimer and
// reports DEV_ERR_TIMEOUT instead of spinning forever.
#include <algorithm>
#include <cstdio>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_ROW_BYTES = 128;  // one 128-byte swizzle row of K: 64 fp16 or 32 fp32 (tf32)
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 192;
// operand kinds: FP16 (kind::f16), TF32 split (kind::tf32, two operand tiles and two
// accumulators), E4M3 with one power-of-two scale per 128 x 128 tile (kind::mxf8f6f4 with UE8M0
// block scales)
constexpr int KIND_F16 = 0, KIND_TF32X3 = 1, KIND_F8 = 2;
template <int KIND> struct TcElem { static constexpr int BK = 64; };      // K elements per stage
template <> struct TcElem<KIND_TF32X3> { static constexpr int BK = 32; };
template <> struct TcElem<KIND_F8> { static constexpr int BK = 128; };
// E4M3 scales: tile_exp[I * ntile_ld + J] = exponent of the 128 x 128 tile (I, J) of L; the
// operands' first row tiles (xt0, yt0) and first K tile (kt0) on that grid
struct F8Scales {
  const int* tile_exp;
  int ntile_ld, xt0, yt0, kt0;
};
__host__ __device__ constexpr uint32_t tmem_cols_pow2(uint32_t c) {
  return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after kWaitTimeoutNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  if (mbar_try_wait(addr, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(addr, parity)) return true;
    if (globaltimer() - t0 > kWaitTimeoutNs) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128B swizzle,
// 8-row core-matrix groups 1024 bytes apart (SBO), descriptor version 1 (bits 46-48).
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = F16 (0), both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// kind::tf32: A = B = TF32 (2) at bits 7-9 and 10-12, D = F32; K = 8 per instruction.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// Block-scaled kind::mxf8f6f4: A = B = E4M3 (0) at bits 7-9 and 10-12, scale factors UE8M0
// (bit 23), scale-factor IDs 0 (bits 4-5, 29-30), N >> 3 at 17-22, M >> 4 at 24-28; D = F32,
// K = 32 per instruction with one scale per row and 32 K elements (scale_vec::1X).
__host__ __device__ constexpr uint32_t idesc_f8bs(int M, int N) {
  return ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f8bs(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate));
}
// Shared-memory descriptor of a scale-factor source for tcgen05.cp .32x128b: 32 rows of 16
// bytes, 8-row core matrices 128 bytes apart, no swizzle.  The sources hold one byte value
// throughout (1 KB each), so every row and column the copy reads carries the tile's scale.
__device__ __forceinline__ uint64_t sf_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(128 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// 32 lanes x 128 bits from shared memory into the TMEM columns at taddr, replicated into the
// four lane quarters (tcgen05 pipeline: ordered before the MMAs this thread issues next)
__device__ __forceinline__ void sf_copy(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}
// The MMAs of one 128-byte K slice (4 instructions of 32 bytes each) into the accumulator
// set at `acc` (TF32 split: hi hi^T at acc, hi lo^T + lo hi^T at acc + BN; E4M3: the slice's
// scale factors are first copied from sf (A at 0, B at 1 KB) into TMEM columns sf_t .. + 7).
template <int BN, int KIND>
__device__ __forceinline__ void mma_slice(uint32_t acc, const uint8_t* a, const uint8_t* b, size_t a_tile,
                                          size_t b_tile, bool first, const uint8_t* sf = nullptr,
                                          uint32_t sf_t = 0) {
  const uint64_t ad = sw128_desc(a), bd = sw128_desc(b);
  if constexpr (KIND == KIND_F16) {
    constexpr uint32_t idesc = idesc_f16(TC_BM, BN);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)                 // K = 16 per instruction: +32 bytes
      mma_f16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (!first || kk > 0) ? 1u : 0u);
  } else if constexpr (KIND == KIND_F8) {
    constexpr uint32_t idesc = idesc_f8bs(TC_BM, BN);
    sf_copy(sf_t, sf_desc(sf));
    sf_copy(sf_t + 4, sf_desc(sf + 1024));
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)                 // K = 32 per instruction: +32 bytes
      mma_f8bs(acc, ad + 2 * kk, bd + 2 * kk, idesc, sf_t, sf_t + 4, (!first || kk > 0) ? 1u : 0u);
  } else {
    constexpr uint32_t idesc = idesc_tf32(TC_BM, BN);
    const uint64_t adl = sw128_desc(a + a_tile), bdl = sw128_desc(b + b_tile);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {               // K = 8 per instruction: +32 bytes
      const uint32_t accum = (!first || kk > 0) ? 1u : 0u;
      mma_tf32(acc, ad + 2 * kk, bd + 2 * kk, idesc, accum);
      mma_tf32(acc + BN, ad + 2 * kk, bdl + 2 * kk, idesc, accum);
      mma_tf32(acc + BN, adl + 2 * kk, bd + 2 * kk, idesc, 1u);
    }
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// TF32 split: two operand tiles (hi, lo) per matrix and stage, and two accumulators per tile.
// E4M3: per stage two 1 KB scale-factor sources in shared memory and 8 TMEM columns (A: 4,
// B: 4) after the accumulators.
template <int BN, int KIND = KIND_F16>
struct TcLayout {
  static_assert(KIND != KIND_F8 || BN <= 128, "an E4M3 column tile lies within one 128-row scale tile");
  static constexpr int ops = KIND == KIND_TF32X3 ? 2 : 1;
  static constexpr int stages = KIND == KIND_TF32X3 && BN >= 128 ? 3 : TC_STAGES;
  static constexpr size_t a_tile = (size_t)TC_BM * TC_ROW_BYTES;
  static constexpr size_t b_tile = (size_t)BN * TC_ROW_BYTES;
  static constexpr size_t a_stage = ops * a_tile;
  static constexpr size_t b_stage = ops * b_tile;
  static constexpr size_t sf_stage = KIND == KIND_F8 ? 2048 : 0;
  static constexpr uint32_t acc_cols = KIND == KIND_TF32X3 ? 2 * BN : BN;   // TMEM columns of one tile
  static constexpr uint32_t sf_cols = KIND == KIND_F8 ? 8 * stages : 0;
  static constexpr size_t bars = 1024;  // barriers + tmem slot, padded
  static constexpr size_t bytes = 1024 /*alignment slack*/ + stages * (a_stage + b_stage + sf_stage) + bars;
};

// E4M3 tile exponents of the A and B tiles at K tiles kb0 .. kb0 + 31: lane l loads those of
// K tile kb0 + l (one load latency per 32 stages; each stage takes its pair by a shuffle)
__device__ __forceinline__ void f8_exponents(const F8Scales& f8, int at, int bt, int kb0, int nk, int& ea, int& eb) {
  const int kt = kb0 + (threadIdx.x & 31);
  ea = kt < nk ? f8.tile_exp[(size_t)(f8.xt0 + at) * f8.ntile_ld + f8.kt0 + kt] : 0;
  eb = kt < nk ? f8.tile_exp[(size_t)(f8.yt0 + bt) * f8.ntile_ld + f8.kt0 + kt] : 0;
}
// E4M3 producer step (warp 0, all lanes): fill the stage's two scale-factor sources with the
// UE8M0 codes 127 + e of the A and B tiles at K tile kb (exponents from f8_exponents, held by
// lane kb % 32), then (lane 0) the operand loads.  Returns false (all lanes) when the wait
// for a free stage expired.
template <int BN>
__device__ __forceinline__ bool f8_produce(int ea_l, int eb_l, int kb, uint8_t* sf, uint64_t* empty_s, uint32_t ph,
                                           uint64_t* full_s, uint8_t* a, uint8_t* b, const CUtensorMap* tmX,
                                           const CUtensorMap* tmY, int xk, int xm, int yn, unsigned* err) {
  const int lane = threadIdx.x & 31;
  int ea = __shfl_sync(0xffffffffu, ea_l, kb & 31) + 127;
  int eb = __shfl_sync(0xffffffffu, eb_l, kb & 31) + 127;
  bool ok = true;
  if (lane == 0) ok = mbar_wait(empty_s, ph ^ 1);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  if (!ok) return false;
  if (ea < 0 || ea > 254 || eb < 0 || eb > 254) {
    if (lane == 0) atomicOr(err, DEV_ERR_RANGE);
    ea = min(max(ea, 0), 254);
    eb = min(max(eb, 0), 254);
  }
  const uint32_t wa = 0x01010101u * (uint32_t)ea, wb = 0x01010101u * (uint32_t)eb;
  uint4* pa = reinterpret_cast<uint4*>(sf);
  uint4* pb = reinterpret_cast<uint4*>(sf + 1024);
  pa[lane] = make_uint4(wa, wa, wa, wa);
  pa[lane + 32] = make_uint4(wa, wa, wa, wa);
  pb[lane] = make_uint4(wb, wb, wb, wb);
  pb[lane + 32] = make_uint4(wb, wb, wb, wb);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    mbar_arrive_expect_tx(full_s, (uint32_t)(TcLayout<BN, KIND_F8>::a_stage + TcLayout<BN, KIND_F8>::b_stage));
    tma_load_2d(a, tmX, xk, xm, full_s);
    tma_load_2d(b, tmY, xk, yn, full_s);
  }
  return true;
}

template <int BN, int KIND>
__device__ __forceinline__ void gemm_tc_tile(const CUtensorMap* tmX, const CUtensorMap* tmY, const CUtensorMap* tmXl,
                                             const CUtensorMap* tmYl, double* __restrict__ C, int ldc, int m, int n,
                                             int k, int lower, double scale, unsigned* __restrict__ err,
                                             F8Scales f8 = F8Scales{}) {
  using Lay = TcLayout<BN, KIND>;
  constexpr int STAGES = Lay::stages;
  constexpr int BK = TcElem<KIND>::BK;
  constexpr uint32_t TMEM_COLS = tmem_cols_pow2(Lay::acc_cols + Lay::sf_cols);
  extern __shared__ unsigned char smem_raw[];
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  if (lower && m0 + TC_BM - 1 < n0) return;          // tile strictly above the diagonal

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * Lay::a_stage;
  uint8_t* sSF = sB + STAGES * Lay::b_stage;
  uint64_t* full = reinterpret_cast<uint64_t*>(sSF + STAGES * Lay::sf_stage);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (k + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if constexpr (KIND == KIND_F8) {
      if (lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmX)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmY)) : "memory");
      }
      int ea = 0, eb = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if ((kb & 31) == 0) f8_exponents(f8, blockIdx.x, n0 / TC_BM, kb, nk, ea, eb);
        if (!f8_produce<BN>(ea, eb, kb, sSF + s * Lay::sf_stage, &empty[s], (kb / STAGES) & 1, &full[s],
                            sA + s * Lay::a_stage, sB + s * Lay::b_stage, tmX, tmY, kb * BK, m0, n0, err)) {
          if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
    } else if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmY)) : "memory");
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1)) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
        mbar_arrive_expect_tx(&full[s], (uint32_t)(Lay::a_stage + Lay::b_stage));
        tma_load_2d(sA + s * Lay::a_stage, tmX, kb * BK, m0, &full[s]);
        tma_load_2d(sB + s * Lay::b_stage, tmY, kb * BK, n0, &full[s]);
        if constexpr (KIND == KIND_TF32X3) {
          tma_load_2d(sA + s * Lay::a_stage + Lay::a_tile, tmXl, kb * BK, m0, &full[s]);
          tma_load_2d(sB + s * Lay::b_stage + Lay::b_tile, tmYl, kb * BK, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&full[s], ph)) { atomicOr(err, DEV_ERR_TIMEOUT); ok = false; break; }
        tc_fence_after();
        mma_slice<BN, KIND>(tmem, sA + s * Lay::a_stage, sB + s * Lay::b_stage, Lay::a_tile, Lay::b_tile, kb == 0,
                            sSF + s * Lay::sf_stage, tmem + Lay::acc_cols + (uint32_t)(8 * s));
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(accum);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (its accessible sub-partition)
    const int q = warp & 3;
    const bool ok = mbar_wait(accum, 0);
    if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
      const int row = m0 + q * 32 + lane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= n) break;                       // uniform across the warp
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        uint32_t r[32];
        tmem_ld32(taddr, r);
        uint32_t r2[KIND == KIND_TF32X3 ? 32 : 1];
        if constexpr (KIND == KIND_TF32X3) tmem_ld32(taddr + BN, r2);
        if (row < m) {
          // all 32 loads first (independent, in flight together), then the 32 stores
          double* base_p = C + (size_t)(n0 + c0) * ldc + row;
          double cv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            cv[j] = (col < n && (!lower || row >= col)) ? __ldcs(base_p + (size_t)j * ldc) : 0.0;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            double v = (double)__uint_as_float(r[j]);
            if constexpr (KIND == KIND_TF32X3) v += (double)__uint_as_float(r2[j]);
            if (col < n && (!lower || row >= col)) __stcs(base_p + (size_t)j * ldc, cv[j] - scale * v);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, BN <= 64 ? 2 : 1)
gemm_f16_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                   double* __restrict__ C, int ldc, int m, int n, int k, int lower, double scale,
                   unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tile<BN, KIND_F16>(&tmX, &tmY, nullptr, nullptr, C, ldc, m, n, k, lower, scale, err);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_tf32x3_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                      const __grid_constant__ CUtensorMap tmXl, const __grid_constant__ CUtensorMap tmYl,
                      double* __restrict__ C, int ldc, int m, int n, int k, int lower, unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tile<BN, KIND_TF32X3>(&tmX, &tmY, &tmXl, &tmYl, C, ldc, m, n, k, lower, 1.0, err);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, BN <= 64 ? 2 : 1)
gemm_f8_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                  double* __restrict__ C, int ldc, int m, int n, int k, int lower, F8Scales f8,
                  unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tile<BN, KIND_F8>(&tmX, &tmY, nullptr, nullptr, C, ldc, m, n, k, lower, 1.0, err, f8);
}

// Persistent variant for products with more tiles than SMs: each CTA walks the active
// tiles (column-major over the tile grid, tiles above the diagonal skipped when `lower`)
// with stride gridDim.x.  The TMEM accumulator is double-buffered (2 x BN columns): the MMA
// warp fills buffer (t & 1) for tile t while the four epilogue warps drain the other one,
// so the FP64 read-modify-write of tile t overlaps the MMAs of tile t + 1.  The operand ring
// (STAGES slots) runs on across tiles.  acc_full[b]: MMAs of the tile in buffer b done
// (tcgen05.commit); acc_empty[b]: its epilogue has read it (one arrival per epilogue warp).
// All waits are bounded; on a timeout every role stops after its current tile.
template <int BN>
__device__ __forceinline__ bool tile_of(int idx, int gm, int gn, bool lower, int& mt, int& nt) {
  for (int j = 0; j < gn; ++j) {
    const int first = lower ? (j * BN) / TC_BM : 0;
    const int cnt = gm - first;
    if (cnt <= 0) continue;
    if (idx < cnt) {
      mt = first + idx;
      nt = j;
      return true;
    }
    idx -= cnt;
  }
  return false;
}

template <int BN, int KIND>
__device__ __forceinline__ void gemm_tc_tiles(const CUtensorMap* tmX, const CUtensorMap* tmY, const CUtensorMap* tmXl,
                                              const CUtensorMap* tmYl, double* __restrict__ C, int ldc, int m, int n,
                                              int k, int lower, double scale, int ntiles, unsigned* __restrict__ err,
                                              F8Scales f8 = F8Scales{}) {
  using Lay = TcLayout<BN, KIND>;
  constexpr int STAGES = Lay::stages;
  constexpr int BK = TcElem<KIND>::BK;
  constexpr uint32_t ACC = Lay::acc_cols;
  constexpr uint32_t TMEM_COLS = tmem_cols_pow2(2 * ACC + Lay::sf_cols);
  extern __shared__ unsigned char smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * Lay::a_stage;
  uint8_t* sSF = sB + STAGES * Lay::b_stage;
  uint64_t* full = reinterpret_cast<uint64_t*>(sSF + STAGES * Lay::sf_stage);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;             // [2]
  uint64_t* acc_empty = acc_full + 2;              // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (k + BK - 1) / BK;
  const int gm = (m + TC_BM - 1) / TC_BM, gn = (n + BN - 1) / BN;

  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmX)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmY)) : "memory");
    }
    if (KIND == KIND_F8 || lane == 0) {
      long long kb_all = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // E4M3: all 32 lanes run this loop, so the abort decision is lane 0's, broadcast
        int stop = *abort_flag;
        if constexpr (KIND == KIND_F8) stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop) break;
        int mt, nt;
        if (!tile_of<BN>(t, gm, gn, lower != 0, mt, nt)) break;
        bool ok = true;
        int ea = 0, eb = 0;
        for (int kb = 0; kb < nk; ++kb, ++kb_all) {
          const int q = (int)(kb_all % STAGES);
          const uint32_t ph = (uint32_t)((kb_all / STAGES) & 1);
          if constexpr (KIND == KIND_F8) {
            if ((kb & 31) == 0) f8_exponents(f8, mt, (nt * BN) / TC_BM, kb, nk, ea, eb);
            if (!f8_produce<BN>(ea, eb, kb, sSF + q * Lay::sf_stage, &empty[q], ph, &full[q], sA + q * Lay::a_stage,
                                sB + q * Lay::b_stage, tmX, tmY, kb * BK, mt * TC_BM, nt * BN, err)) {
              ok = false;
              break;
            }
          } else {
            if (!mbar_wait(&empty[q], ph ^ 1)) { ok = false; break; }
            mbar_arrive_expect_tx(&full[q], (uint32_t)(Lay::a_stage + Lay::b_stage));
            tma_load_2d(sA + q * Lay::a_stage, tmX, kb * BK, mt * TC_BM, &full[q]);
            tma_load_2d(sB + q * Lay::b_stage, tmY, kb * BK, nt * BN, &full[q]);
            if constexpr (KIND == KIND_TF32X3) {
              tma_load_2d(sA + q * Lay::a_stage + Lay::a_tile, tmXl, kb * BK, mt * TC_BM, &full[q]);
              tma_load_2d(sB + q * Lay::b_stage + Lay::b_tile, tmYl, kb * BK, nt * BN, &full[q]);
            }
          }
        }
        if (!ok) {
          if (lane == 0) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            *abort_flag = 1;
          }
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long kb_all = 0;
      int it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t acc = tmem + (uint32_t)b * ACC;
        if (!mbar_wait(&acc_empty[b], (uint32_t)(((it >> 1) & 1) ^ 1))) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++kb_all) {
          const int q = (int)(kb_all % STAGES);
          const uint32_t ph = (uint32_t)((kb_all / STAGES) & 1);
          if (!mbar_wait(&full[q], ph)) { atomicOr(err, DEV_ERR_TIMEOUT); ok = false; break; }
          tc_fence_after();
          mma_slice<BN, KIND>(acc, sA + q * Lay::a_stage, sB + q * Lay::b_stage, Lay::a_tile, Lay::b_tile, kb == 0,
                              sSF + q * Lay::sf_stage, tmem + 2 * ACC + (uint32_t)(8 * q));
          mma_commit(&empty[q]);
        }
        if (!ok) { *abort_flag = 1; break; }
        mma_commit(&acc_full[b]);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (its accessible sub-partition)
    const int qd = warp & 3;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      int mt, nt;
      if (!tile_of<BN>(t, gm, gn, lower != 0, mt, nt)) break;
      const int b = it & 1;
      const bool ok = mbar_wait(&acc_full[b], (uint32_t)((it >> 1) & 1));
      if (!ok) { atomicOr(err, DEV_ERR_TIMEOUT); *abort_flag = 1; break; }
      tc_fence_after();
      const int m0 = mt * TC_BM, n0 = nt * BN;
      const int row = m0 + qd * 32 + lane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= n) break;                       // uniform across the warp
        const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)b * ACC + (uint32_t)c0;
        uint32_t r[32];
        tmem_ld32(taddr, r);
        uint32_t r2[KIND == KIND_TF32X3 ? 32 : 1];
        if constexpr (KIND == KIND_TF32X3) tmem_ld32(taddr + BN, r2);
        if (row < m) {
          double* base_p = C + (size_t)(n0 + c0) * ldc + row;
          double cv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            cv[j] = (col < n && (!lower || row >= col)) ? __ldcs(base_p + (size_t)j * ldc) : 0.0;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            double v = (double)__uint_as_float(r[j]);
            if constexpr (KIND == KIND_TF32X3) v += (double)__uint_as_float(r2[j]);
            if (col < n && (!lower || row >= col)) __stcs(base_p + (size_t)j * ldc, cv[j] - scale * v);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
      if (*abort_flag) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_f16_tc_persistent(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                       double* __restrict__ C, int ldc, int m, int n, int k, int lower, double scale,
                       int ntiles, unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tiles<BN, KIND_F16>(&tmX, &tmY, nullptr, nullptr, C, ldc, m, n, k, lower, scale, ntiles, err);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_tf32x3_tc_persistent(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                          const __grid_constant__ CUtensorMap tmXl, const __grid_constant__ CUtensorMap tmYl,
                          double* __restrict__ C, int ldc, int m, int n, int k, int lower, int ntiles,
                          unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tiles<BN, KIND_TF32X3>(&tmX, &tmY, &tmXl, &tmYl, C, ldc, m, n, k, lower, 1.0, ntiles, err);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_f8_tc_persistent(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                      double* __restrict__ C, int ldc, int m, int n, int k, int lower, int ntiles, F8Scales f8,
                      unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  gemm_tc_tiles<BN, KIND_F8>(&tmX, &tmY, nullptr, nullptr, C, ldc, m, n, k, lower, 1.0, ntiles, err, f8);
}

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled_t get_encode() {
  static PFN_encodeTiled_t fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled_t>(p);
  }
  return fn;
}

// 2-D map over a rows x cols block of a row-major e4m3 (bytes), fp16 or fp32 matrix (leading
// dimension ld elements), box = box_rows x 128 bytes of K, 128B swizzle, zero fill outside.
template <typename T>
bool make_map(CUtensorMap* map, const T* base, int rows, int cols, int ld, int box_rows) {
  static_assert(sizeof(T) == 1 || sizeof(T) == 2 || sizeof(T) == 4, "e4m3, fp16 or fp32 operands");
  PFN_encodeTiled_t enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
  cuuint32_t box[2] = {(cuuint32_t)(TC_ROW_BYTES / sizeof(T)), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(map, dt, 2, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_persistent(double* C, int ldc, const __half* S, int lds, int xr0, int yr0, int k0, int m, int n,
                              int k, bool lower, double scale, long long ntiles, int sms, unsigned* dev_err,
                              cudaStream_t s) {
  CUtensorMap mx, my;
  if (!make_map(&mx, S + (size_t)xr0 * lds + k0, m, k, lds, TC_BM)) return cudaErrorInvalidValue;
  if (!make_map(&my, S + (size_t)yr0 * lds + k0, n, k, lds, BN)) return cudaErrorInvalidValue;
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_tc_persistent<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TcLayout<BN>::bytes);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  const int cap = launch_ctx().max_ctas > 0 ? std::min(sms, launch_ctx().max_ctas) : sms;
  const int grid = (int)std::min<long long>(ntiles, cap);
  (void)launch_pdl(gemm_f16_tc_persistent<BN>, dim3(grid), dim3(TC_THREADS), TcLayout<BN>::bytes, s, mx, my, C, ldc, m, n, k, lower ? 1 : 0,
                                                                          scale, (int)ntiles, dev_err);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_bn(double* C, int ldc, const __half* S, int lds, int xr0, int yr0, int k0, int m, int n, int k,
                      bool lower, double scale, unsigned* dev_err, cudaStream_t s) {
  CUtensorMap mx, my;
  if (!make_map(&mx, S + (size_t)xr0 * lds + k0, m, k, lds, TC_BM)) return cudaErrorInvalidValue;
  if (!make_map(&my, S + (size_t)yr0 * lds + k0, n, k, lds, BN)) return cudaErrorInvalidValue;
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(gemm_f16_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TcLayout<BN>::bytes);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  dim3 grid((m + TC_BM - 1) / TC_BM, (n + BN - 1) / BN);
  (void)launch_pdl(gemm_f16_tc_kernel<BN>, dim3(grid), dim3(TC_THREADS), TcLayout<BN>::bytes, s, mx, my, C, ldc, m, n, k, lower ? 1 : 0,
                                                                        scale, dev_err);
  return cudaGetLastError();
}

// TF32 split: hi / lo row-major FP32 arrays with the same layout (leading dimension ldh)
template <int BN>
cudaError_t launch_split(double* C, int ldc, const float* H, const float* Lo, int ldh, int xr0, int yr0, int k0,
                         int m, int n, int k, bool lower, long long ntiles, int sms, bool persistent,
                         unsigned* dev_err, cudaStream_t s) {
  CUtensorMap mx, my, mxl, myl;
  const size_t xo = (size_t)xr0 * ldh + k0, yo = (size_t)yr0 * ldh + k0;
  if (!make_map(&mx, H + xo, m, k, ldh, TC_BM) || !make_map(&my, H + yo, n, k, ldh, BN) ||
      !make_map(&mxl, Lo + xo, m, k, ldh, TC_BM) || !make_map(&myl, Lo + yo, n, k, ldh, BN))
    return cudaErrorInvalidValue;
  using Lay = TcLayout<BN, true>;
  static unsigned long long attr_mask[2] = {0, 0};
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask[persistent] & attr_bit)) {
    cudaError_t e = persistent ? cudaFuncSetAttribute(gemm_tf32x3_tc_persistent<BN>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes)
                               : cudaFuncSetAttribute(gemm_tf32x3_tc_kernel<BN>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
    if (e != cudaSuccess) return e;
    attr_mask[persistent] |= attr_bit;
  }
  if (persistent) {
    const int cap = launch_ctx().max_ctas > 0 ? std::min(sms, launch_ctx().max_ctas) : sms;
    const int grid = (int)std::min<long long>(ntiles, cap);
    (void)launch_pdl(gemm_tf32x3_tc_persistent<BN>, dim3(grid), dim3(TC_THREADS), Lay::bytes, s, mx, my, mxl, myl, C,
                     ldc, m, n, k, lower ? 1 : 0, (int)ntiles, dev_err);
  } else {
    dim3 grid((m + TC_BM - 1) / TC_BM, (n + BN - 1) / BN);
    (void)launch_pdl(gemm_tf32x3_tc_kernel<BN>, grid, dim3(TC_THREADS), Lay::bytes, s, mx, my, mxl, myl, C, ldc, m, n,
                     k, lower ? 1 : 0, dev_err);
  }
  return cudaGetLastError();
}

// E4M3 codes (row-major bytes, ld lds) with per-tile exponents: block-scaled FP8 MMAs
template <int BN>
cudaError_t launch_f8(double* C, int ldc, const uint8_t* S, int lds, int xr0, int yr0, int k0, int m, int n, int k,
                      bool lower, const int* tile_exp, int ntile_ld, long long ntiles, int sms, bool persistent,
                      unsigned* dev_err, cudaStream_t s) {
  CUtensorMap mx, my;
  if (!make_map(&mx, S + (size_t)xr0 * lds + k0, m, k, lds, TC_BM) || !make_map(&my, S + (size_t)yr0 * lds + k0, n, k, lds, BN))
    return cudaErrorInvalidValue;
  const F8Scales f8{tile_exp, ntile_ld, xr0 / TC_BM, yr0 / TC_BM, k0 / TC_BM};
  using Lay = TcLayout<BN, KIND_F8>;
  static unsigned long long attr_mask[2] = {0, 0};
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask[persistent] & attr_bit)) {
    cudaError_t e = persistent ? cudaFuncSetAttribute(gemm_f8_tc_persistent<BN>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes)
                               : cudaFuncSetAttribute(gemm_f8_tc_kernel<BN>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
    if (e != cudaSuccess) return e;
    attr_mask[persistent] |= attr_bit;
  }
  if (persistent) {
    const int cap = launch_ctx().max_ctas > 0 ? std::min(sms, launch_ctx().max_ctas) : sms;
    const int grid = (int)std::min<long long>(ntiles, cap);
    (void)launch_pdl(gemm_f8_tc_persistent<BN>, dim3(grid), dim3(TC_THREADS), Lay::bytes, s, mx, my, C, ldc, m, n, k,
                     lower ? 1 : 0, (int)ntiles, f8, dev_err);
  } else {
    dim3 grid((m + TC_BM - 1) / TC_BM, (n + BN - 1) / BN);
    (void)launch_pdl(gemm_f8_tc_kernel<BN>, grid, dim3(TC_THREADS), Lay::bytes, s, mx, my, C, ldc, m, n, k,
                     lower ? 1 : 0, f8, dev_err);
  }
  return cudaGetLastError();
}

// tiles of a BN-wide grid that hold work (tiles wholly above the diagonal are skipped)
long long active_tiles(int m, int n, bool lower, int bn) {
  const int gm = (m + TC_BM - 1) / TC_BM, gn = (n + bn - 1) / bn;
  if (!lower) return (long long)gm * gn;
  long long t = 0;
  for (int j = 0; j < gn; ++j) {
    const int first = (j * bn) / TC_BM;          // first M-tile reaching the diagonal of column tile j
    t += gm > first ? gm - first : 0;
  }
  return t;
}

// the widest tile width that still gives occ tiles per SM
int pick_bn(int m, int n, bool lower, int occ) {
  const long long need = (long long)device_sm_count() * (occ > 0 ? occ : 1);
  if (n > 128 && active_tiles(m, n, lower, 256) >= need) return 256;
  if (n > 64 && active_tiles(m, n, lower, 128) >= need) return 128;
  if (n > 32 && active_tiles(m, n, lower, 64) >= need) return 64;
  return 32;
}

}  // namespace

bool tc_gemm_supported() { return get_encode() != nullptr; }

cudaError_t launch_gemm_f8_tc(double* C, int ldc, const uint8_t* S, int lds, int xr0, int yr0, int k0, int m, int n,
                              int k, bool lower, const int* tile_exp, int ntile_ld, unsigned* dev_err, cudaStream_t s,
                              int occupancy) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  if ((xr0 % TC_BM) || (yr0 % TC_BM) || (k0 % TC_BM) || (lds % 16) || (reinterpret_cast<uintptr_t>(S) & 15))
    return cudaErrorInvalidValue;
  // a column tile must lie within one 128-row scale tile: at most 128 wide
  int bn = pick_bn(m, n, lower, occupancy);
  if (bn > 128) bn = 128;
  const int sms = device_sm_count();
  const long long nt = active_tiles(m, n, lower, bn);
  const bool persistent = bn == 128 && nt > sms;
  if (bn == 128)
    return launch_f8<128>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, tile_exp, ntile_ld, nt, sms, persistent, dev_err, s);
  if (bn == 64)
    return launch_f8<64>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, tile_exp, ntile_ld, nt, sms, false, dev_err, s);
  return launch_f8<32>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, tile_exp, ntile_ld, nt, sms, false, dev_err, s);
}

cudaError_t launch_gemm_tf32x3_tc(double* C, int ldc, const float* H, const float* Lo, int ldh, int xr0, int yr0,
                                  int k0, int m, int n, int k, bool lower, unsigned* dev_err, cudaStream_t s,
                                  int occupancy) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  if ((k0 % 4) != 0 || (ldh % 4) != 0 || (reinterpret_cast<uintptr_t>(H) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(Lo) & 15) != 0)
    return cudaErrorInvalidValue;
  // two accumulators per tile: at most 128 columns, so that a persistent CTA's two tiles
  // (4 x 128 TMEM columns) fit the SM's 512
  int bn = pick_bn(m, n, lower, occupancy);
  if (bn > 128) bn = 128;
  const int sms = device_sm_count();
  const long long nt = active_tiles(m, n, lower, bn);
  const bool persistent = bn == 128 && nt > sms;
  if (bn == 128) return launch_split<128>(C, ldc, H, Lo, ldh, xr0, yr0, k0, m, n, k, lower, nt, sms, persistent, dev_err, s);
  if (bn == 64) return launch_split<64>(C, ldc, H, Lo, ldh, xr0, yr0, k0, m, n, k, lower, nt, sms, false, dev_err, s);
  return launch_split<32>(C, ldc, H, Lo, ldh, xr0, yr0, k0, m, n, k, lower, nt, sms, false, dev_err, s);
}

cudaError_t launch_gemm_f16_tc(double* C, int ldc, const __half* S, int lds, int xr0, int yr0, int k0, int m, int n,
                               int k, bool lower, double scale, unsigned* dev_err, cudaStream_t s, int occupancy) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  if ((k0 % 8) != 0 || (lds % 8) != 0 || (reinterpret_cast<uintptr_t>(S) & 15) != 0) return cudaErrorInvalidValue;
  // The FP64 read-modify-write of the epilogue runs on the SM's FP64 pipe and costs about
  // as much as the tile's MMAs, so small products are cut into narrower tiles until they
  // cover the SMs (tiles of 64 or 32 columns also fit two CTAs per SM, one CTA's epilogue
  // then overlapping the other's MMAs).
  const int bn = pick_bn(m, n, lower, occupancy);
  const int sms = device_sm_count();
  // more tiles than SMs: persistent CTAs with the epilogue of one tile under the MMAs of the next
  if (bn >= 128) {
    const long long nt = active_tiles(m, n, lower, bn);
    if (nt > sms) {
      if (bn == 256)
        return launch_persistent<256>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, nt, sms, dev_err, s);
      return launch_persistent<128>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, nt, sms, dev_err, s);
    }
  }
  if (bn == 256) return launch_bn<256>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, dev_err, s);
  if (bn == 128) return launch_bn<128>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, dev_err, s);
  if (bn == 64) return launch_bn<64>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, dev_err, s);
  return launch_bn<32>(C, ldc, S, lds, xr0, yr0, k0, m, n, k, lower, scale, dev_err, s);
}

}  // namespace hrp
