// Leaf POTRF (Alg. 1 base case) spread over a cluster of 8 CTAs, in FP64 or in
// double-float arithmetic on the FP32 pipe.
//
// FP64 on this GPU: each SM sub-partition issues one FP64 warp instruction per ~64
// cycles (also the dependent latency), the SM as a whole about one per 19 cycles
// (1.7 lane-FMAs per clock, 1.2 TFLOP/s for the device), and a warp instruction costs the
// same however few lanes are active.  The n^3/6 FMAs of a 128 x 128 leaf therefore keep
// one SM busy for ~100 us, and every leaf lies on the recursion's critical path.  Here the
// block is cut into 16 x 16 tiles; tile (I, J), I >= J, lives in the shared memory of CTA
// (I + J) mod 8 for the whole factorization (at most 5 tiles per CTA), and the block is
// factored right-looking by tile columns p = 0, 1, ...:
//   A  the owner D of (p, p) applies the update of panel p-1 to it, factors it
//      (potrf16_chain) and stores L_pp into the shared memory of the CTAs that need it,
//      while the other CTAs apply the update of panel p-1 to their tiles;
//                                                                      cluster barrier
//   B  the owners of (I, p), I > p, solve X L_pp^T = A_Ip (TRSM) and store the result
//      into the shared memory of every CTA that updates a tile with it;
//                                                                      cluster barrier
// D's other tiles get the update of panel p-1 (and D's diagonal tile its FP32 inverse) in
// phase A of panel p + 1, while the next diagonal owner factors.
// Finished panel tiles are written into the consumers' shared memory (distributed shared
// memory stores, double-buffered by panel parity), so no CTA waits on a remote load
// inside the loop.  The only waits are the hardware cluster barriers, which every thread
// of the cluster reaches the same number of times (a failed pivot is seen by all CTAs
// after the same barrier).  The FP32 inverse W = L^{-1} for the FP32 leaf TRSM (when
// requested) is built at the end by column blocks, one CTA per block:
// W_JJ = L_JJ^{-1}, W_IJ = -L_II^{-1} sum_{K=J}^{I-1} L_IK W_KJ.
//
// Double-float mode (df = 1).  The same schedule with every tile held as a pair of binary32
// numbers hi + lo (Dekker 1971; about 48 significant bits): sums by Knuth's error-free TwoSum,
// products by the FMA-based exact product, in the accurate pair forms whose relative errors
// Joldes, Muller and Popescu (2017) bound by a few units of 2^-48, and dot products
// accumulated as in Ogita, Rump and Oishi's Dot2 (2005).  FP32 operations take a few cycles of
// latency where FP64 ones take ~64 (~128 while other sub-partitions issue FP64), and the FP32
// pipe has ~40x the FP64 issue rate, so the pivot chains, the TRSM substitutions and the
// rank-16 updates all run several times faster.
//   - The leaf is scaled by 2^-2s (2s the largest even integer not above the largest
//     diagonal exponent) while it is loaded and converted, exactly in hi and to 2^-48 in lo,
//     by integer operations on the bit fields; L is stored back times 2^s, rounded to FP64.
//     Scaled entries below 2^-60 are read as zero (2^-12 below the pairs' unit roundoff
//     relative to the largest diagonal entry).
//   - A leaf with an entry that is not finite or above 8 times the largest diagonal entry, or
//     with a diagonal entry or pivot that is not positive or falls below 2^-36 times the
//     largest diagonal entry (where the pairs' error terms would leave binary32's normal
//     range), is factored again from the untouched input by the FP64 schedule in the same
//     launch; that also reports the column of a failing pivot exactly as FP64 does.
#include <climits>
#include <cooperative_groups.h>
#include <type_traits>

#include "hrp_internal.cuh"

namespace cg = cooperative_groups;

namespace hrp {
namespace {

constexpr int kCL = 8;                  // CTAs per cluster (portable size)
constexpr int kTS = 16;                 // tile edge
constexpr int kTLD = 17;                // padded row length of a tile (elements)
constexpr int kTileD = kTS * kTLD;      // elements per tile slot
constexpr int kMaxOwn = 5;              // tiles per CTA for 8 x 8 tiles owned by (I + J) mod 8
constexpr int kCThreads = 256;              // threads per CTA: one per entry of a 16 x 16 tile
constexpr int kFT = 128;                    // threads that work in the FP64 tile operations
static_assert(kCThreads == kTS * kTS, "one thread per tile entry");
constexpr int kLowT = kTS * (kTS + 1) / 2;   // entries of a lower 16 x 16 triangle
constexpr int kMaxGather = 36;               // W phase: tiles one CTA reads (28 of L, 8 inverses)
constexpr int kChainWarps = 3;               // worker warps of the 16 x 16 pivot chain
constexpr int kChainSeg = 2;                 // entries of one row per worker thread
constexpr int kFallback = 1;                 // leaf_body's result: factor again in FP64

// a double-float value hi + lo, |lo| <= ulp(hi) / 2 (8-byte aligned: one 64-bit access)
struct __align__(8) dfloat {
  float hi, lo;
};

// E = double (FP64 mode) or dfloat (double-float mode); both are 8 bytes, so the two layouts
// coincide and one dynamic shared-memory size serves both
template <class E>
struct LeafSmem {
  E own[kMaxOwn][kTileD];               // owned tiles, row-major (row i at i * kTLD)
  E pan[2][8][kTileD];                  // pan[p & 1][I] = L_{I,p} (I > p) or L_pp (I = p)
  double cv[kTS][kTS];                  // FP64 pivot chain: cv[k][i] = a_ik after the updates of columns < k
  double dpr[kTS + 2];                  // FP64 pivot chain: a_kk after the updates of columns < k - 1
  double usq[kTS + 2];                  // FP64 pivot chain: a_{k,k-1}^2 after the updates of columns < k - 1
  double dk[kTS];                       // pivots d_k
  double sk[kTS];                       // 1 / d_k
  E rinv[kTS];                          // 1 / L_kk = d_k^{-1/2} of the diagonal tile factored last here
  E rin_copy[kTS];                      // rinv of the diagonal tile the TRSM here uses
  E lt[kTileD];                         // TRSM: unit lower Lt = L diag(rinv) of that tile
  float rinvf[kTS];                     // FP32 rounding of 1 / L_kk (unscaled) for the FP32 inverse
  float ownf[kMaxOwn][kTileD];          // FP32 copies of the finished owned tiles
  float winv[2][kTileD];                // FP32 inverses of the (up to 2) diagonal tiles owned
  float gat[kMaxGather][kTileD];        // W phase: gathered FP32 tiles
  float wcol[8][kTileD];                // W phase: W_KJ of this CTA's column block
  float tmp[kTileD];                    // W phase: sum_K L_IK W_KJ
  const float* gsrc[kMaxGather];        // W phase: where each gathered tile comes from
  dfloat dcol[2][kTS];                  // double-float chain: column k (after the updates of columns < k)
  dfloat drs[kTS];                      // double-float chain: d_k^{-1/2}
  int dred[2][kCThreads / 32];          // double-float load: per-warp largest / smallest diagonal exponent
  int lflag;                            // double-float load: an entry here is out of range
  int fail;                             // written into every CTA by D: 1 a pivot failed (FP64), 2 fall back
  int cfail;                            // pivot chain: column of the failed pivot, or -1
  signed char slot[8][8];               // slot of tile (I, J) in its owner's `own`
};
static_assert(sizeof(LeafSmem<double>) == sizeof(LeafSmem<dfloat>), "one shared-memory size for both modes");

__device__ __forceinline__ int owner_of(int I, int J) { return (I + J) & (kCL - 1); }

// (i, j) of entry e < 136 of a lower 16 x 16 triangle enumerated row by row:
// i = floor((sqrt(8e + 1) - 1) / 2), exact in single precision for these e (checked below)
__device__ __forceinline__ void lower_entry(int e, int& i, int& j) {
  i = (int)((sqrtf((float)(8 * e + 1)) - 1.0f) * 0.5f);
  if ((i + 1) * (i + 2) / 2 <= e) ++i;              // guard against a rounding below an integer
  if (i * (i + 1) / 2 > e) --i;
  j = e - i * (i + 1) / 2;
}

// 0: not positive or not finite; 1: positive finite outside the single-precision seed range;
// 2: positive with |log2 d| < 120.  Integer tests on the bits (no FP64 instruction).
__device__ __forceinline__ int pivot_class(double d) {
  const long long b = __double_as_longlong(d);
  if (b <= 0) return 0;
  const int ex = (int)(b >> 52);
  if (ex == 0x7ff) return 0;
  return (ex > 1023 - 120 && ex < 1023 + 120) ? 2 : 1;
}

// d truncated to single precision and a single-precision value widened to double, both by
// integer operations on the IEEE-754 bit fields (d, f positive and normal with |log2| < 120:
// pivot_class == 2).  On this GPU a conversion instruction costs about as much as a
// dependent DFMA on the FP64 pipe; these take a few integer operations instead.
__device__ __forceinline__ float trunc_to_float(double d) {
  const long long b = __double_as_longlong(d);
  const int hi = (int)(b >> 32);
  const unsigned lo = (unsigned)b;
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;                    // rebias the exponent
  const unsigned m = ((unsigned)(hi & 0xfffff) << 3) | (lo >> 29);    // top 23 mantissa bits
  return __int_as_float((e << 23) | (int)m);
}
__device__ __forceinline__ double widen_float(float f) {
  const unsigned u = __float_as_uint(f);
  const long long e = (long long)(((u >> 23) & 0xff) - 127 + 1023);
  const long long m = (long long)(u & 0x7fffff);
  return __longlong_as_double((e << 52) | (m << 29));
}

// 1/d from the single-precision reciprocal x0 of d truncated to single precision, and one
// third-order step of Householder's iteration for 1/x - d = 0: with e = 1 - d x0,
// 1/d = x0 / (1 - e) = x0 (1 + e + e^2 + O(e^3)).  The seed (truncation of d plus the
// approximation, |e| < 2^-21) leaves a truncation error below 2^-63; three dependent FP64
// operations after the seed.  pivot_class(d) == 2.
__device__ __forceinline__ double recip_third_order(double d) {
  float xf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xf) : "f"(trunc_to_float(d)));
  const double x0 = widen_float(xf);
  const double e = fma(-d, x0, 1.0);
  const double w = fma(e, e, e);
  return fma(x0, w, x0);
}

// 1/sqrt(d) from a single-precision seed r0 and one third-order step: with
// e = 1 - d r0^2, d^{-1/2} = r0 (1 - e)^{-1/2} = r0 (1 + e/2 + 3e^2/8 + O(e^3)); the seed's
// |e| < 2^-20 leaves a truncation error below 2^-60.  Values outside the single-precision
// exponent range take the library sqrt.
__device__ __forceinline__ double rsqrt_third_order(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  const double r = (double)rsqrtf((float)d);
  const double e = fma(-d * r, r, 1.0);
  const double t = fma(0.375, e, 0.5);
  return fma(r * e, t, r);
}

// C -= LI * LJ^T for an off-diagonal 16 x 16 tile, by threads 0..127 (one FP64 warp
// instruction costs the same however many lanes it has, so two entries per thread):
// thread (i, cp) = (tid / 8, tid % 8) owns C[i][2cp], C[i][2cp + 1].
__device__ __forceinline__ void tile_update(double* __restrict__ C, const double* __restrict__ LI,
                                            const double* __restrict__ LJ, int tid) {
  if (tid >= kFT) return;
  const int i = tid >> 3, j0 = 2 * (tid & 7);
  double c0 = C[i * kTLD + j0], c1 = C[i * kTLD + j0 + 1];
#pragma unroll
  for (int k = 0; k < kTS; ++k) {
    const double a = LI[i * kTLD + k];
    c0 = fma(-a, LJ[j0 * kTLD + k], c0);
    c1 = fma(-a, LJ[(j0 + 1) * kTLD + k], c1);
  }
  C[i * kTLD + j0] = c0;
  C[i * kTLD + j0 + 1] = c1;
}

// C -= LI * LI^T on the lower triangle of a diagonal tile (136 entries x 16 terms), spread
// evenly over threads 0..127: entry t (t < 128) is summed by thread t, and each of the last
// 8 entries (row 15, columns 8..15) is split over the 16 threads of a half-warp, one term
// each, and reduced by shuffles; every thread issues 17 FMAs.
__device__ __forceinline__ void tile_update_diag(double* __restrict__ C, const double* __restrict__ LI, int tid) {
  if (tid >= kFT) return;                                  // whole warps
  int i, j;
  lower_entry(tid, i, j);
  double c0 = 0.0, c1 = 0.0;
#pragma unroll
  for (int k = 0; k < kTS; k += 2) {
    c0 = fma(LI[i * kTLD + k], LI[j * kTLD + k], c0);
    c1 = fma(LI[i * kTLD + k + 1], LI[j * kTLD + k + 1], c1);
  }
  const int jx = 8 + (tid >> 4), kx = tid & 15;            // entry (15, jx), term kx
  double x = LI[15 * kTLD + kx] * LI[jx * kTLD + kx];
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  C[i * kTLD + j] -= c0 + c1;
  if (kx == 0) C[15 * kTLD + jx] -= x;
}

// Cholesky of the 16 x 16 tile T (lower part, row-major kTLD) by the 128 threads.  The
// column recurrence runs alone on thread 0 (warp 0, sub-partition 0):
//   d_{k+1} = d'_{k+1} - u_{k+1} s_k,  s_k = 1/d_k,
// with d'_{k+1} = a_{k+1,k+1} and u_{k+1} = a_{k+1,k}^2 after the updates of columns < k.
// NW worker warps (1 .. NW) apply the update of column k, a_ij -= (a_ik s_k) a_jk for
// i >= j > k, one step behind, and publish what the next steps read; each worker thread holds
// up to SEG consecutive entries of one row (one multiply per row and column, then one FMA
// per entry).  One CTA barrier per column; it also carries the recurrence's failure flag
// (__syncthreads_or).  At the end l_jj = d_j r_j and l_ij = a_ij r_j (a_ij after the updates
// of columns < j), r_j = d_j^{-1/2}, also stored in sm.rinv.  Returns the 0-based column of
// the first pivot that is not positive and finite, or -1 (the same in every thread).
template <int NW, int SEG>
__device__ int potrf16_chain_t(double* __restrict__ T, LeafSmem<double>& sm, int tid) {
  const int warp = tid >> 5;
  int wi = -1, wj0 = 0, wcnt = 0;
  double a[SEG];
#pragma unroll
  for (int q = 0; q < SEG; ++q) a[q] = 0.0;
  int fail = 0;                                   // thread 0: the recurrence met a bad pivot
  if (warp >= 1 && warp <= NW) {
    const int w = tid - 32;
    for (int i = 0, idx = 0; i < kTS; ++i) {       // row i has ceil((i + 1) / SEG) segments
      const int ns = (i + SEG) / SEG;
      if (wi < 0 && w < idx + ns) {
        wi = i;
        wj0 = SEG * (w - idx);
        wcnt = min(SEG, i + 1 - wj0);
      }
      idx += ns;
    }
    if (wi >= 0) {
#pragma unroll
      for (int q = 0; q < SEG; ++q)
        if (q < wcnt) a[q] = T[wi * kTLD + wj0 + q];
      if (wj0 == 0) sm.cv[0][wi] = a[0];
      if (wi == 1) {
        sm.dpr[1] = a[1];                          // row 1: one segment holding columns 0, 1
        sm.usq[1] = a[0] * a[0];
      }
    }
  } else if (tid == 0) {
    const double d0 = T[0];
    const int c = pivot_class(d0);
    fail = c ? 0 : 1;
    sm.cfail = c ? -1 : 0;
    sm.dk[0] = d0;
    sm.sk[0] = (c == 2) ? recip_third_order(d0) : 1.0 / d0;
  }
  int bad = __syncthreads_or(fail);
  for (int k = 0; k + 1 < kTS && !bad; ++k) {
    if (tid == 0) {
      const double d = fma(-sm.usq[k + 1], sm.sk[k], sm.dpr[k + 1]);
      const int c = pivot_class(d);
      if (!c) {
        sm.cfail = k + 1;
        fail = 1;
      }
      sm.dk[k + 1] = d;
      sm.sk[k + 1] = (c == 2) ? recip_third_order(d) : 1.0 / d;
    } else if (wi > k && wj0 + wcnt - 1 > k) {
      const double t = sm.cv[k][wi] * sm.sk[k];
#pragma unroll
      for (int q = 0; q < SEG; ++q) {
        const int j = wj0 + q;
        if (q < wcnt && j > k) {
          a[q] = fma(-t, sm.cv[k][j], a[q]);
          if (j == k + 1) sm.cv[k + 1][wi] = a[q];
          if (wi == k + 2) {
            if (j == k + 2) sm.dpr[k + 2] = a[q];
            else if (j == k + 1) sm.usq[k + 2] = a[q] * a[q];
          }
        }
      }
    }
    bad = __syncthreads_or(fail);
  }
  if (bad) return sm.cfail;
  if (tid < kTS) sm.rinv[tid] = rsqrt_third_order(sm.dk[tid]);
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + kCThreads * h;
    if (e >= kLowT) break;
    int i, j;
    lower_entry(e, i, j);
    T[i * kTLD + j] = (i == j ? sm.dk[j] : sm.cv[j][i]) * sm.rinv[j];
  }
  return -1;
}

__device__ __forceinline__ int potrf16_chain(double* __restrict__ T, LeafSmem<double>& sm, int tid) {
  return potrf16_chain_t<kChainWarps, kChainSeg>(T, sm, tid);
}


// ---------------------------------------------------------------------------------------
// Double-float arithmetic (see the file comment)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);                  // x.hi y.hi = p + e exactly
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  const dfloat t = df_two_sum(x.lo, y.lo);
  s = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }
// 1/d for d > 0: single-precision seed x0, e = 1 - d x0 as a pair (1 - fl(d.hi x0) is exact by
// Sterbenz's lemma), then the third-order step x0 (1 + e + e^2); |e| < 2^-21
__device__ __forceinline__ dfloat df_recip(dfloat d) {
  float x0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x0) : "f"(d.hi));
  const float p = d.hi * x0;
  float pe = fmaf(d.hi, x0, -p);
  pe = fmaf(d.lo, x0, pe);
  const dfloat e = df_two_sum(1.0f - p, -pe);
  const float p2 = x0 * e.hi;
  float q = fmaf(x0, e.hi, -p2);
  q = fmaf(x0, e.lo, q);
  q = fmaf(p2, e.hi, q);
  const dfloat r = df_fast_two_sum(x0, p2);
  return df_fast_two_sum(r.hi, r.lo + q);
}
// d^{-1/2} for d > 0: seed r0, e = 1 - d r0^2 as a pair, then r0 (1 + e/2 + 3 e^2 / 8)
__device__ __forceinline__ dfloat df_rsqrt(dfloat d) {
  const float r0 = rsqrtf(d.hi);
  const float y = r0 * r0;
  const dfloat t = df_mul(d, dfloat{y, fmaf(r0, r0, -y)});
  const dfloat e = df_two_sum(1.0f - t.hi, -t.lo);
  const float h = 0.5f * e.hi;
  const float c = fmaf(0.375f * e.hi, e.hi, 0.5f * e.lo);
  const float p2 = r0 * h;
  float q = fmaf(r0, h, -p2);
  q = fmaf(r0, c, q);
  const dfloat r = df_fast_two_sum(r0, p2);
  return df_fast_two_sum(r.hi, r.lo + q);
}
// unbiased binary32 exponent (-127 for zero and subnormals)
__device__ __forceinline__ int f32_exponent(float x) { return (int)((__float_as_uint(x) >> 23) & 0xff) - 127; }

// Dot2 accumulator: the running sum s (binary32, carried on by error-free TwoSum) and c, which
// collects TwoSum's rounding errors and the low-order parts of the products
struct df_acc {
  float s, c;
};
__device__ __forceinline__ df_acc acc_of(dfloat x) { return {x.hi, x.lo}; }
// a -= x y
__device__ __forceinline__ void acc_sub_prod(df_acc& a, dfloat x, dfloat y) {
  const float p = -x.hi * y.hi;
  float e = fmaf(-x.hi, y.hi, -p);                 // -x.hi y.hi = p + e exactly
  e = fmaf(-x.hi, y.lo, e);
  e = fmaf(-x.lo, y.hi, e);
  const float s = a.s + p, bb = s - a.s;
  a.c += ((a.s - (s - bb)) + (p - bb)) + e;
  a.s = s;
}
__device__ __forceinline__ dfloat acc_value(df_acc a) { return df_two_sum(a.s, a.c); }

// x 2^-s2 as a pair, by integer operations: hi = x's sign and leading 24 significand bits
// (truncated) at the scaled exponent e, lo = the remaining 29 bits rounded to binary32 at
// 2^(e - 52), then renormalized.  Returns 0 (converted), 1 (zero, subnormal, or e < -60: out
// = 0) or 2 (not finite or e > 3).
__device__ __forceinline__ int df_split_scaled(double x, int s2, dfloat& out) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0x7ff) return 2;
  const int e = E - 1023 - s2;
  if (E == 0 || e < -60) {
    out = {0.0f, 0.0f};
    return 1;
  }
  if (e > 3) return 2;
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  const float ulo = __uint2float_rn((unsigned)(m & 0x1fffffffu)) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
  out = df_fast_two_sum(hi, __uint_as_float(__float_as_uint(ulo) | sgn));
  return 0;
}
// f 2^off widened to double by integer operations (exact); zero and subnormal f give 0
__device__ __forceinline__ double df_widen_scaled(float f, int off) {
  const unsigned u = __float_as_uint(f);
  const int E = (int)((u >> 23) & 0xff);
  if (E == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(E - 127 + 1023 + off) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double df_to_double_scaled(dfloat x, int off) {
  return df_widen_scaled(x.hi, off) + df_widen_scaled(x.lo, off);
}

// ---------------------------------------------------------------------------------------
// Tile operations in double-float: one entry per thread (the FP32 pipe is not issue-bound here,
// so the more independent chains in flight the better)
// ---------------------------------------------------------------------------------------
// C -= LI * LJ^T for an off-diagonal 16 x 16 tile: thread (i, j) = (tid / 16, tid % 16), its
// 16 terms in two Dot2 sums (even and odd k)
__device__ __forceinline__ void tile_update(dfloat* __restrict__ C, const dfloat* __restrict__ LI,
                                            const dfloat* __restrict__ LJ, int tid) {
  const int i = tid >> 4, j = tid & 15;
  df_acc c0 = acc_of(C[i * kTLD + j]), c1{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kTS; k += 2) {
    acc_sub_prod(c0, LI[i * kTLD + k], LJ[j * kTLD + k]);
    acc_sub_prod(c1, LI[i * kTLD + k + 1], LJ[j * kTLD + k + 1]);
  }
  C[i * kTLD + j] = df_add(acc_value(c0), acc_value(c1));
}

// C -= LI * LI^T on the lower triangle of a diagonal tile: entry t (t < 136) by thread t
__device__ __forceinline__ void tile_update_diag(dfloat* __restrict__ C, const dfloat* __restrict__ LI, int tid) {
  if (tid >= kLowT) return;
  int i, j;
  lower_entry(tid, i, j);
  df_acc c0 = acc_of(C[i * kTLD + j]), c1{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kTS; k += 2) {
    acc_sub_prod(c0, LI[i * kTLD + k], LI[j * kTLD + k]);
    acc_sub_prod(c1, LI[i * kTLD + k + 1], LI[j * kTLD + k + 1]);
  }
  C[i * kTLD + j] = df_add(acc_value(c0), acc_value(c1));
}

// X L^T = A in place, unit-diagonal form as the FP64 trsm16: Lt = L diag(rinv), Y Lt^T = A by
// substitution, X = Y diag(rinv).  Thread (i, j) = (tid / 16, tid % 16) accumulates y_ij as a
// Dot2 sum; y_ik is passed along the row's 16 threads (one half-warp) by shuffles.
__device__ __forceinline__ void trsm16(dfloat* __restrict__ A, const dfloat* __restrict__ L,
                                       const dfloat* __restrict__ rinv, dfloat* __restrict__ Lt, int tid) {
  const int i = tid >> 4, j = tid & 15, lane = tid & 31;
  if (j < i) Lt[i * kTLD + j] = df_mul(L[i * kTLD + j], rinv[j]);
  __syncthreads();
  df_acc c = acc_of(A[i * kTLD + j]);
#pragma unroll
  for (int k = 0; k + 1 < kTS; ++k) {
    const dfloat v = acc_value(c);                       // y_ik in thread (i, k)
    const int src = (lane & 16) | k;
    const dfloat y{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
    if (j > k) acc_sub_prod(c, y, Lt[j * kTLD + k]);
  }
  A[i * kTLD + j] = df_mul(acc_value(c), rinv[j]);
}

// Cholesky of the 16 x 16 tile T (lower part) in double-float, LDL^T form: a_ij -= (a_ik a_jk)
// / d_k for i >= j > k.  Threads 0..119 hold the entries (i, j), i >= j >= 1, in registers;
// column 0 and, after each step, the next column are published in a double-buffered column
// array, one CTA barrier per column.  Every thread forms 1 / d_k itself from the published
// pivot, so every thread sees the same pivot and takes the same exit.  At the end l_ij =
// a_ij r_j, l_jj = d_j r_j, r_j = d_j^{-1/2} (also in sm.rinv).  Returns -1, or -2 when a pivot
// is not positive or falls below 2^-36 (the leaf is then factored again in FP64).
__device__ int potrf16(dfloat* __restrict__ T, LeafSmem<dfloat>& sm, int tid) {
  const bool act = tid < kLowT - kTS;
  int i = 0, j = 0;
  if (act) {
    lower_entry(tid, i, j);
    ++i;
    ++j;
  }
  dfloat a{0.0f, 0.0f}, c0{0.0f, 0.0f};
  if (act) a = T[i * kTLD + j];
  if (tid < kTS) {
    c0 = T[tid * kTLD];
    sm.dcol[0][tid] = c0;
  }
  __syncthreads();
  int res = -1;
  for (int k = 0; k + 1 < kTS; ++k) {
    const dfloat* col = sm.dcol[k & 1];
    const dfloat dk = col[k];
    if (!(dk.hi > 0.0f) || f32_exponent(dk.hi) < -36) {   // the same in every thread
      res = -2;
      break;
    }
    if (act && j > k) {
      a = df_add(a, df_neg(df_mul(df_mul(col[i], col[j]), df_recip(dk))));
      if (j == k + 1) sm.dcol[(k + 1) & 1][i] = a;
    }
    __syncthreads();
  }
  if (res == -1) {
    const dfloat d = sm.dcol[(kTS - 1) & 1][kTS - 1];
    if (!(d.hi > 0.0f) || f32_exponent(d.hi) < -36) res = -2;
  }
  if (res != -1) return res;
  if (act && i == j) sm.drs[j] = df_rsqrt(a);
  if (tid == 0) sm.drs[0] = df_rsqrt(c0);
  __syncthreads();
  if (act) T[i * kTLD + j] = df_mul(a, sm.drs[j]);
  if (tid < kTS) {
    T[tid * kTLD] = df_mul(c0, sm.drs[0]);
    sm.rinv[tid] = sm.drs[tid];
  }
  return -1;
}
__device__ __forceinline__ int potrf16(double* __restrict__ T, LeafSmem<double>& sm, int tid) {
  return potrf16_chain(T, sm, tid);
}

// conversions at the leaf's boundary (s2 = 2s, sc = s: see the file comment)
__device__ __forceinline__ int load_conv(double x, int, double& out) {
  out = x;
  return 0;
}
__device__ __forceinline__ int load_conv(double x, int s2, dfloat& out) { return df_split_scaled(x, s2, out); }
__device__ __forceinline__ void set_small(double& out, int v) { out = (double)v; }
__device__ __forceinline__ void set_small(dfloat& out, int v) { out = {(float)v, 0.0f}; }
__device__ __forceinline__ double store_conv(double x, int) { return x; }
__device__ __forceinline__ double store_conv(dfloat x, int sc) { return df_to_double_scaled(x, sc); }
__device__ __forceinline__ float f32_of(double x, int) { return (float)x; }
__device__ __forceinline__ float f32_of(dfloat x, int sc) { return ldexpf(x.hi, sc); }

// 2s for the double-float leaf (the largest even integer not above the largest diagonal
// exponent), or INT_MIN when a diagonal entry is not positive and finite or lies 2^36 or more
// below the largest; the same in every CTA (each reads the whole diagonal)
__device__ int leaf_scale(const double* __restrict__ A, int ld, int n, LeafSmem<dfloat>& sm, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  int emax = 0, emin = 0x7ff, bad = 0;
  if (tid < n) {
    const int E = (int)(__double_as_longlong(A[(size_t)tid * ld + tid]) >> 52);   // < 0 for x < 0
    if (E <= 0 || E >= 0x7ff) bad = 1;
    else emax = emin = E;
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  emin = __reduce_min_sync(0xffffffffu, emin);
  if (lane == 0) {
    sm.dred[0][warp] = emax;
    sm.dred[1][warp] = emin;
  }
  if (__syncthreads_or(bad)) return INT_MIN;
#pragma unroll
  for (int w = 0; w < kCThreads / 32; ++w) {
    emax = max(emax, sm.dred[0][w]);
    emin = min(emin, sm.dred[1][w]);
  }
  const int s2 = ((emax - 1023) >> 1) * 2;
  return (emin - 1023 - s2 < -36) ? INT_MIN : s2;
}
__device__ __forceinline__ int leaf_scale(const double*, int, int, LeafSmem<double>&, int) { return 0; }


// X L^T = A for the 16 x 16 tile A (in place), L lower with 1/L_kk in rinv, by threads
// 0..127, in unit-diagonal form: with L = Lt diag(L_kk) (Lt_jk = L_jk / L_kk, formed here in
// Lt) and Y = X diag(L_kk), Y Lt^T = A is a substitution without scaling, y_ij = a_ij -
// sum_{k<j} y_ik Lt_jk, and X = Y diag(rinv) at the end; no multiply sits between one
// column's broadcast and the next.  Thread (i, cp) = (tid / 8, tid % 8) holds A[i][2cp],
// A[i][2cp + 1]; y_ik is passed along the row's 8 threads by a shuffle.
__device__ __forceinline__ void trsm16(double* __restrict__ A, const double* __restrict__ L,
                                       const double* __restrict__ rinv, double* __restrict__ Lt, int tid) {
  {
    const int j = tid >> 4, k = tid & 15;
    if (k < j) Lt[j * kTLD + k] = L[j * kTLD + k] * rinv[k];
  }
  __syncthreads();
  if (tid >= kFT) return;                                  // whole warps
  const int i = tid >> 3, cp = tid & 7, lane = tid & 31, j0 = 2 * cp;
  double c0 = A[i * kTLD + j0], c1 = A[i * kTLD + j0 + 1];
#pragma unroll
  for (int k = 0; k < kTS; ++k) {
    const double y = __shfl_sync(0xffffffffu, (k & 1) ? c1 : c0, (lane & ~7) | (k >> 1));
    if (j0 > k) c0 = fma(-y, Lt[j0 * kTLD + k], c0);
    if (j0 + 1 > k) c1 = fma(-y, Lt[(j0 + 1) * kTLD + k], c1);
  }
  A[i * kTLD + j0] = c0 * rinv[j0];
  A[i * kTLD + j0 + 1] = c1 * rinv[j0 + 1];
}

// Store the 16 x 16 tile T into slot `dst` of the shared memory of every CTA in `mask`.
template <class E>
__device__ __forceinline__ void push_tile(cg::cluster_group& cluster, const E* __restrict__ T, E* dst, unsigned mask,
                                          int tid) {
  const int o = (tid >> 4) * kTLD + (tid & 15);
  const E v = T[o];
  for (int r = 0; r < kCL; ++r)
    if (mask & (1u << r)) cluster.map_shared_rank(dst, r)[o] = v;
}

// FP32 copy of the 16 x 16 tile (unscaled: sc is the double-float leaf's scale)
template <class E>
__device__ __forceinline__ void to_f32(const E* __restrict__ T, float* __restrict__ F, int tid, int sc) {
  const int o = (tid >> 4) * kTLD + (tid & 15);
  F[o] = f32_of(T[o], sc);
}

// FP32 inverse of the lower 16 x 16 tile Lf (FP32, row-major kTLD) into Wv, by lanes
// 0..15 of one warp: lane c forms column c by forward substitution, dividing by L_rr as a
// product with rinvf[r], the FP32 rounding of 1/L_rr.
__device__ __forceinline__ void trtri16_f32(const float* __restrict__ Lf, const float* __restrict__ rinvf,
                                            float* __restrict__ Wv, int lane) {
  if (lane >= kTS) return;
  const int c = lane;
  float w[kTS];
#pragma unroll
  for (int r = 0; r < kTS; ++r) {
    float s = (r == c) ? 1.f : 0.f;
#pragma unroll
    for (int q = 0; q < r; ++q) s = fmaf(-Lf[r * kTLD + q], w[q], s);
    w[r] = (r >= c) ? s * rinvf[r] : 0.f;
  }
#pragma unroll
  for (int r = 0; r < kTS; ++r) Wv[r * kTLD + c] = w[r];
}

// CTAs holding a tile that is updated with L_{I,p}: owners of (I, J), p < J <= I, and of (J, I), J >= I
__device__ __forceinline__ unsigned consumers(int I, int p, int NT) {
  unsigned m = 0;
  for (int J = p + 1; J <= I; ++J) m |= 1u << owner_of(I, J);
  for (int J = I; J < NT; ++J) m |= 1u << owner_of(J, I);
  return m;
}


__device__ __forceinline__ float rinv_f32(double r, int) { return (float)r; }
__device__ __forceinline__ float rinv_f32(dfloat r, int sc) { return ldexpf(r.hi, -sc); }

// One factorization of the leaf in arithmetic E (see the file comment).  Returns kFallback
// (the same in every CTA of the cluster, before any write to A, W32 or info) when the
// double-float leaf must be factored again in FP64, else 0.
template <class E>
__device__ int leaf_body(double* __restrict__ A, int ld, int n, int col0, float* __restrict__ W32, int ldw,
                         int* __restrict__ info, unsigned char* smem_raw) {
  constexpr bool kDF = std::is_same<E, dfloat>::value;
  LeafSmem<E>& sm = *reinterpret_cast<LeafSmem<E>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NT = (n + kTS - 1) / kTS;

  // an earlier block failed: stop like LAPACK (every CTA reads the same value: nothing in
  // this kernel writes info before the first cluster barrier)
  const bool skip = *(volatile int*)info != INT_MAX;
  if (tid == 0) {
    int cnt[kCL] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int J = 0; J < 8; ++J)
      for (int I = 0; I < 8; ++I) sm.slot[I][J] = (I >= J && I < NT) ? (signed char)(cnt[owner_of(I, J)]++) : -1;
    sm.fail = 0;
    sm.lflag = 0;
  }
  __syncthreads();
  int s2 = 0;
  if (!skip) {
    // load the owned tiles (all loads issued before the first store, and before the leaf's
    // scale is known: only their conversion needs it); rows / columns past n are the identity
    // NT <= 8, so this CTA owns at most one tile per block column J: row (rank - J) mod 8
    // one entry of each owned tile per thread: (ii, jj) = (tid % 16, tid / 16)
    const int jj = tid >> 4, ii = tid & 15;          // column-major walk: coalesced reads
    double v[kCL];
#pragma unroll
    for (int J = 0; J < kCL; ++J) {
      const int I = (rank - J) & 7;
      double x = 0.0;
      if (J < NT && I >= J && I < NT) {
        const int gi = kTS * I + ii, gj = kTS * J + jj;
        if (gi < n && gj < n) x = (gi >= gj) ? A[(size_t)gj * ld + gi] : 0.0;
        else x = (gi == gj) ? 1.0 : 0.0;
      }
      v[J] = x;
    }
    if (kDF) {
      s2 = leaf_scale(A, ld, n, sm, tid);
      if (s2 == INT_MIN) return kFallback;     // every CTA read the same diagonal
    }
    int lbad = 0;
#pragma unroll
    for (int J = 0; J < kCL; ++J) {
      const int I = (rank - J) & 7;
      if (J < NT && I >= J && I < NT) {
        E x;
        if (kTS * I + ii < n && kTS * J + jj < n) lbad |= load_conv(v[J], s2, x) >> 1;
        else set_small(x, kTS * I + ii == kTS * J + jj ? 1 : 0);
        sm.own[sm.slot[I][J]][ii * kTLD + jj] = x;
      }
    }
    if (kDF) {
      lbad = __syncthreads_or(lbad);
      if (tid == 0) sm.lflag = lbad;
    }
  }
  cluster.sync();
  if (skip) return 0;
  if (kDF) {
    int any = 0;
    for (int r = 0; r < kCL; ++r) any |= *(volatile int*)cluster.map_shared_rank(&sm.lflag, r);
    if (any) return kFallback;
  }
  const int sc = s2 / 2;

  bool failed = false;
  for (int p = 0; p < NT; ++p) {
    const int D = owner_of(p, p);
    const int cur = p & 1, prev = cur ^ 1;
    // ---- A ----
    if (rank == D) {
      E* T = sm.own[sm.slot[p][p]];
      if (p > 0) {
        tile_update_diag(T, sm.pan[prev][p], tid);
        __syncthreads();
      }
      const int bad = potrf16(T, sm, tid);
      if (bad != -1) {
        if (tid == 0) {
          if (bad >= 0) atomicMin(info, col0 + kTS * p + bad + 1);
          for (int r = 0; r < kCL; ++r) *cluster.map_shared_rank(&sm.fail, r) = bad >= 0 ? 1 : 2;
        }
      } else {
        __syncthreads();                                       // L_pp and rinv complete
        unsigned trsm_ctas = 0;
        for (int I = p + 1; I < NT; ++I) trsm_ctas |= 1u << owner_of(I, p);
        push_tile(cluster, T, sm.pan[cur][p], trsm_ctas, tid);
        if (tid < kTS)
          for (int r = 0; r < kCL; ++r)
            if (trsm_ctas & (1u << r)) cluster.map_shared_rank(sm.rin_copy, r)[tid] = sm.rinv[tid];
      }
    } else {
      // the work D(p-1) left for later: its tiles' update with panel p-2 (still in buffer
      // `cur`; panel p's tiles only arrive there in phase B) and the FP32 inverse of its
      // diagonal tile (p-1, p-1)
      if (p >= 2 && rank == owner_of(p - 1, p - 1)) {
        for (int J = p; J < NT; ++J)
          for (int I = J; I < NT; ++I)
            if (owner_of(I, J) == rank) {
              E* C = sm.own[sm.slot[I][J]];
              if (I == J) tile_update_diag(C, sm.pan[cur][I], tid);
              else tile_update(C, sm.pan[cur][I], sm.pan[cur][J], tid);
            }
      }
      if (W32 && p >= 1 && rank == owner_of(p - 1, p - 1)) {
        float* F = sm.ownf[sm.slot[p - 1][p - 1]];
        to_f32(sm.own[sm.slot[p - 1][p - 1]], F, tid, sc);
        if (tid < kTS) sm.rinvf[tid] = rinv_f32(sm.rinv[tid], sc);
        __syncthreads();
        if (warp == 0) trtri16_f32(F, sm.rinvf, sm.winv[p - 1 >= 4 ? 1 : 0], lane);
      }
      if (p > 0)
        for (int J = p; J < NT; ++J)
          for (int I = J; I < NT; ++I)
            if (owner_of(I, J) == rank) {
              E* C = sm.own[sm.slot[I][J]];
              if (I == J) tile_update_diag(C, sm.pan[prev][I], tid);
              else tile_update(C, sm.pan[prev][I], sm.pan[prev][J], tid);
            }
    }
    cluster.sync();                                              // S1
    const int f = *(volatile int*)&sm.fail;
    if (f == 2) return kFallback;
    if (f) {
      failed = true;
      break;
    }
    // ---- B ----
    int mine = -1;
    for (int I = p + 1; I < NT; ++I)
      if (owner_of(I, p) == rank) mine = I;
    if (mine >= 0) {
      E* X = sm.own[sm.slot[mine][p]];
      trsm16(X, sm.pan[cur][p], sm.rin_copy, sm.lt, tid);
      __syncthreads();
      push_tile(cluster, X, sm.pan[cur][mine], consumers(mine, p, NT), tid);
      if (W32) to_f32(X, sm.ownf[sm.slot[mine][p]], tid, sc);
    }
    // D's other tiles and the FP32 inverse of (p, p) wait for phase A of panel p + 1 (done
    // there while D(p+1) factors), except after the last panel
    if (rank == D && W32 && p + 1 == NT) {
      float* F = sm.ownf[sm.slot[p][p]];
      to_f32(sm.own[sm.slot[p][p]], F, tid, sc);
      if (tid < kTS) sm.rinvf[tid] = rinv_f32(sm.rinv[tid], sc);
      __syncthreads();
      if (warp == 0) trtri16_f32(F, sm.rinvf, sm.winv[p >= 4 ? 1 : 0], lane);
    }
    cluster.sync();                                              // S2
  }
  if (!failed) {
    // store the owned tiles (lower part inside the block)
    for (int J = 0; J < NT; ++J)
      for (int I = J; I < NT; ++I) {
        if (owner_of(I, J) != rank) continue;
        const E* T = sm.own[sm.slot[I][J]];
        for (int e = tid; e < kTS * kTS; e += kCThreads) {
          const int jj = e >> 4, ii = e & 15;
          const int gi = kTS * I + ii, gj = kTS * J + jj;
          if (gi < n && gj < n && gi >= gj) A[(size_t)gj * ld + gi] = store_conv(T[ii * kTLD + jj], sc);
        }
      }
    // FP32 inverse, column block J = rank: gather L_IK (J <= K < I) and W_II (I >= J)
    const int J = rank;
    if (W32 && J < NT) {
      const int m = NT - J;
      const int nl = m * (m - 1) / 2, ng = nl + m;
      if (tid < ng) {
        const float* src;
        if (tid < nl) {
          int I = J + 1, t = tid;                 // enumerate (I, K), K = J .. I-1, row by row
          while (t >= I - J) {
            t -= I - J;
            ++I;
          }
          const int K = J + t;
          src = cluster.map_shared_rank(sm.ownf[sm.slot[I][K]], owner_of(I, K));
        } else {
          const int I = J + (tid - nl);
          src = cluster.map_shared_rank(sm.winv[I >= 4 ? 1 : 0], owner_of(I, I));
        }
        sm.gsrc[tid] = src;
      }
      __syncthreads();
      // kTileD = 272 floats = 68 float4 per tile; 8 loads in flight per thread
      constexpr int kV4 = kTileD / 4;
      const int nchunk = ng * kV4;
      for (int c0 = tid; c0 < nchunk; c0 += 8 * kCThreads) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + u * kCThreads;
          if (c < nchunk) v[u] = reinterpret_cast<const float4*>(sm.gsrc[c / kV4])[c % kV4];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + u * kCThreads;
          if (c < nchunk) reinterpret_cast<float4*>(sm.gat[c / kV4])[c % kV4] = v[u];
        }
      }
      __syncthreads();
      // gathered index of L_IK: row I starts at (I-J-1)(I-J)/2; W_II follows the nl L tiles
      for (int e = tid; e < kTileD; e += kCThreads) sm.wcol[J][e] = sm.gat[nl][e];
      __syncthreads();
      // right-looking: once W_KJ is final, every later row block I adds L_IK W_KJ to its sum
      // tmp_I (slot I - J - 1 of acc; the terms arrive in the order K = J, J + 1, .., as a
      // left-looking sum would take them), and W_{K+1,J} = -W_{K+1,K+1} tmp_{K+1}: a step
      // costs one tile product on the chain instead of I - J of them
      const int r = tid >> 4, q = tid & 15;
      float acc[kCL - 1];
#pragma unroll
      for (int t = 0; t < kCL - 1; ++t) acc[t] = 0.f;
      for (int K = J; K + 1 < NT; ++K) {
        float wk[kTS];                                   // column q of W_KJ, read once per step
#pragma unroll
        for (int k = 0; k < kTS; ++k) wk[k] = sm.wcol[K][k * kTLD + q];
#pragma unroll
        for (int t = 0; t < kCL - 1; ++t) {
          const int I = J + 1 + t;
          if (I > K && I < NT) {
            const float* L = sm.gat[(I - J - 1) * (I - J) / 2 + (K - J)];
#pragma unroll
            for (int k = 0; k < kTS; ++k) acc[t] = fmaf(L[r * kTLD + k], wk[k], acc[t]);
            if (I == K + 1) sm.tmp[r * kTLD + q] = acc[t];
          }
        }
        __syncthreads();
        const float* Wi = sm.gat[nl + (K + 1 - J)];
        float wi[kTS], tq[kTS];
#pragma unroll
        for (int mm = 0; mm < kTS; ++mm) {
          wi[mm] = Wi[r * kTLD + mm];
          tq[mm] = sm.tmp[mm * kTLD + q];
        }
        float o0 = 0.f;
#pragma unroll
        for (int mm = 0; mm < kTS; ++mm) o0 = fmaf(-wi[mm], tq[mm], o0);
        sm.wcol[K + 1][r * kTLD + q] = o0;
        __syncthreads();
      }
      // write column block J of W (column-major, zeros above the diagonal)
      for (int jj = warp; jj < kTS; jj += kCThreads / 32) {
        const int gj = kTS * J + jj;
        if (gj >= n) break;
        for (int gi = lane; gi < n; gi += 32) {
          const int I = gi >> 4, ii = gi & 15;
          float v = 0.f;
          if (I > J || (I == J && ii >= jj)) v = sm.wcol[I][ii * kTLD + jj];
          W32[(size_t)gj * ldw + gi] = v;
        }
      }
    }
  }
  cluster.sync();                       // no CTA leaves while others may read its tiles
  return 0;
}

__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kCThreads, 1)
potrf_leaf_cluster_kernel(double* __restrict__ A, int ld, int n, int col0, float* __restrict__ W32, int ldw,
                          int* __restrict__ info, int df) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (df) {
    if (leaf_body<dfloat>(A, ld, n, col0, W32, ldw, info, smem_raw) != kFallback) return;
    cg::this_cluster().sync();          // every CTA has left the double-float attempt
  }
  (void)leaf_body<double>(A, ld, n, col0, W32, ldw, info, smem_raw);
}

}  // namespace

cudaError_t launch_potrf_leaf_cluster(double* A, int ld, int n, int col0, float* W32, int ldw, int* info,
                                      cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 128) return cudaErrorInvalidValue;
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(potrf_leaf_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(LeafSmem<double>));
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  (void)launch_pdl(potrf_leaf_cluster_kernel, dim3(kCL), dim3(kCThreads), sizeof(LeafSmem<double>), s, A, ld, n, col0,
                   W32, ldw, info, launch_ctx().leaf_df ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace hrp
