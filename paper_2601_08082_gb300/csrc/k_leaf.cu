// Leaf kernels of the recursion (Alg. 1 and Alg. 2 base cases): POTRF of a diagonal
// block staged in shared memory, and TRSM_{R,L,T} of a row panel against it.
#include <climits>
#include <cstdio>

#include <cooperative_groups.h>

#include "hrp_internal.cuh"

namespace cg = cooperative_groups;

namespace hrp {
namespace {

__device__ __forceinline__ double round_to_f16(double x) { return (double)__half2float(__double2half(x)); }

// ---------------------------------------------------------------------------------------
// Reciprocal square root by Newton's method (r <- r + r (1 - d r^2) / 2, quadratic
// convergence) from a single-precision seed: two steps take the seed's ~22 correct bits
// past double precision.  On this GPU a dependent FP64 operation costs ~64 cycles, so
// the 6 dependent operations here are far cheaper than sqrt followed by a division.
// Values outside the single-precision exponent range take the library sqrt.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double hr = 0.5 * r;
    const double e = fma(-d * r, r, 1.0);
    r = fma(hr, e, r);
  }
  return r;
}
__device__ __forceinline__ float rsqrt_newton(float d) {
  float r = rsqrtf(d);
  const float e = fmaf(-d * r, r, 1.0f);
  return fmaf(0.5f * r, e, r);
}

constexpr int kInvLD = 132;   // leading dimension of the FP32 factor / inverse staging (16B rows)

// FP32 inverse W = L^{-1} of the n x n lower-triangular Lf (column-major, ld kInvLD, rows
// >= n zero), n <= 128, written column-major into Wt (ld kInvLD).  Blocked by 32:
// W_II = L_II^{-1} per diagonal block (one warp each, lane c = column c, registers), then
// W_IJ = -W_II * sum_{K=J}^{I-1} L_IK W_KJ for I - J = 1, 2, 3 (one warp per block).
__device__ void trtri32_blocked(const float* __restrict__ Lf, float* __restrict__ Wt, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = (n + 31) / 32;
  if (warp < nb) {
    const int I0 = warp * 32;
    float w[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      float sacc = (r == lane) ? 1.f : 0.f;
#pragma unroll
      for (int q = 0; q < r; ++q) sacc = fmaf(-Lf[(I0 + q) * kInvLD + I0 + r], w[q], sacc);
      const float dg = Lf[(I0 + r) * kInvLD + I0 + r];
      w[r] = (I0 + r < n && r >= lane) ? sacc / dg : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) Wt[(I0 + lane) * kInvLD + I0 + r] = w[r];
  }
  __syncthreads();
  for (int dlt = 1; dlt < nb; ++dlt) {
    const int J = warp, I = warp + dlt;
    if (I < nb) {
      const int I0 = I * 32, J0 = J * 32;
      float t[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) t[r] = 0.f;
      for (int K = J; K < I; ++K) {
        const int K0 = K * 32;
        for (int q = 0; q < 32; ++q) {
          const float wv = Wt[(J0 + lane) * kInvLD + K0 + q];
          const float4* lc = reinterpret_cast<const float4*>(Lf + (K0 + q) * kInvLD + I0);
#pragma unroll
          for (int r4 = 0; r4 < 8; ++r4) {
            const float4 l = lc[r4];
            t[4 * r4 + 0] = fmaf(l.x, wv, t[4 * r4 + 0]);
            t[4 * r4 + 1] = fmaf(l.y, wv, t[4 * r4 + 1]);
            t[4 * r4 + 2] = fmaf(l.z, wv, t[4 * r4 + 2]);
            t[4 * r4 + 3] = fmaf(l.w, wv, t[4 * r4 + 3]);
          }
        }
      }
      float o[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) o[r] = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < 32; ++s2) {
        const float4* wc = reinterpret_cast<const float4*>(Wt + (I0 + s2) * kInvLD + I0);
#pragma unroll
        for (int r4 = 0; r4 < 8; ++r4) {
          const float4 v = wc[r4];
          o[4 * r4 + 0] = fmaf(-v.x, t[s2], o[4 * r4 + 0]);
          o[4 * r4 + 1] = fmaf(-v.y, t[s2], o[4 * r4 + 1]);
          o[4 * r4 + 2] = fmaf(-v.z, t[s2], o[4 * r4 + 2]);
          o[4 * r4 + 3] = fmaf(-v.w, t[s2], o[4 * r4 + 3]);
        }
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) Wt[(J0 + lane) * kInvLD + I0 + r] = (I0 + r < n) ? o[r] : 0.f;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Leaf POTRF (Alg. 1 base case "A <- POTRF_L(A)") of an n x n block, n <= 128, one CTA of
// 256 threads, right-looking with the block held in registers.
//
// Thread (ti, tj) = (t % 16, t / 16) owns the 64 entries (ti + 16a, tj + 16b), a, b < 8,
// for the whole factorization.  Step k: the 16 threads owning column k (one half-warp)
// read the pivot a_kk by a shuffle, check it is positive and finite (first failure:
// atomicMin of the global column into info, and the CTA stops), form r = 1/sqrt(a_kk) by
// Newton's method, scale their column entries and publish the column in shared memory;
// after one barrier every thread applies the rank-1 update to the entries it owns.  The
// step loop is split as k = 16 KB + kt with KB unrolled, so register indices are static
// and the blocks a < b or b < KB, which hold no work, are skipped at compile time.
// Optionally the FP32 inverse of the stored factor is formed for the FP32 leaf TRSM.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, 1)
potrf_leaf_kernel(double* __restrict__ A, int ld, int n, int col0, int round16,
                  float* __restrict__ W32, int ldw, int* __restrict__ info, unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T col[2][128];
  __shared__ int s_fail;
  if (*(volatile int*)info != INT_MAX) return;   // an earlier block failed: stop like LAPACK
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = tid & 15, tj = tid >> 4;
  T reg[8][8];
  bool over16 = false;                               // an F16 value beyond kF16Max
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ti + 16 * a, j = tj + 16 * b;
      double v = (i < n && j < n && i >= j) ? A[(size_t)j * ld + i] : 0.0;
      if (round16) {
        over16 |= fabs(v) > (double)kF16Max;
        v = round_to_f16(v);
      }
      reg[a][b] = (T)v;
    }
  if (round16 && __any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
  if (tid == 0) s_fail = 0;
  __syncthreads();

#pragma unroll
  for (int KB = 0; KB < 8; ++KB) {
    if (16 * KB >= n) break;
    for (int kt = 0; kt < 16; ++kt) {
      const int k = 16 * KB + kt;
      if (k >= n) break;
      const int buf = k & 1;
      // (a) the half-warp owning column k: pivot, 1/sqrt by Newton, scale, publish
      if (warp == (kt >> 1)) {
        const int src = ((kt & 1) << 4) + kt;       // lane of thread (ti, tj) = (kt, kt)
        const T d = __shfl_sync(0xffffffffu, reg[KB][KB], src);
        const bool mine = (tj == kt);
        if (!((d > (T)0) && isfinite((double)d))) {
          if (lane == src) {
            atomicMin(info, col0 + k + 1);
            s_fail = 1;
          }
        } else if (mine) {
          const T r = rsqrt_newton(d);
#pragma unroll
          for (int a = KB; a < 8; ++a) {
            const int i = ti + 16 * a;
            if (i == k) {
              reg[a][KB] = d * r;
              col[buf][i] = d * r;
            } else if (i > k && i < n) {
              reg[a][KB] *= r;
              col[buf][i] = reg[a][KB];
            }
          }
        }
      }
      __syncthreads();
      if (s_fail) return;
      // (b) rank-1 update of the owned entries (i >= j > k)
      T ci[8], cj[8];
#pragma unroll
      for (int a = KB; a < 8; ++a) ci[a] = col[buf][ti + 16 * a];
#pragma unroll
      for (int b = KB; b < 8; ++b) cj[b] = col[buf][tj + 16 * b];
#pragma unroll
      for (int b = KB; b < 8; ++b) {
        if (b == KB && tj <= kt) continue;             // j <= k
#pragma unroll
        for (int a = b; a < 8; ++a) {
          if (a == b && ti < tj) continue;             // i < j
          reg[a][b] -= ci[a] * cj[b];
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ti + 16 * a, j = tj + 16 * b;
      if (i < n && j < n && i >= j) {
        double v = (double)reg[a][b];
        if (round16) {                                 // F16 leaf: the stored factor is FP16
          over16 |= fabs(v) > (double)kF16Max;
          v = round_to_f16(v);
        }
        A[(size_t)j * ld + i] = v;
      }
    }
  if (round16 && __any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
  if (W32 == nullptr) return;
  __syncthreads();

  // ---- FP32 inverse of the stored factor (read back from global, as float) ----
  float* Lf = reinterpret_cast<float*>(smem_raw);
  float* Wt = Lf + 128 * kInvLD;
  const int nb32 = ((n + 31) / 32) * 32;
  for (int j = warp; j < nb32; j += 8) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      v[q] = (i < n && j < n && i >= j) ? __ldcg(A + (size_t)j * ld + i) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (lane + 32 * q < nb32) Lf[j * kInvLD + lane + 32 * q] = (float)v[q];
  }
  __syncthreads();
  trtri32_blocked(Lf, Wt, n);
  for (int j = warp; j < n; j += 8)
    for (int i = lane; i < n; i += 32) W32[(size_t)j * ldw + i] = (i >= j) ? Wt[j * kInvLD + i] : 0.f;
}

// ---------------------------------------------------------------------------------------
// Leaf TRSM by substitution (Alg. 2 base case "B <- TRSM(...; L, B)", right side, lower,
// transposed), with T the arithmetic type (FP32 here; the FP64 leaf TRSM is the right-looking
// kernel below): each thread owns one row of B and substitutes column by column,
// x_j = (b_j - sum_{k<j} x_k l_jk) / l_jj.  B = A[r0.., c0..] and L = Lm[c0.., c0..]
// (Lm = A inside the factorization, a separate factor for a standalone TRSM).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(64)
trsm_subst_kernel(double* __restrict__ A, int ld, int r0, int m, int c0, int nc, const double* __restrict__ Lm,
                  int ldl, __half* __restrict__ S, int lds, float* __restrict__ S32, int ld32,
                  const int* __restrict__ info, unsigned* __restrict__ err, int rows_per_cta) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (*(volatile const int*)info != INT_MAX) return;
  T* Ls = reinterpret_cast<T*>(smem_raw);              // row-major nc x nc: Ls[j * nc + k]
  T* Xs = Ls + nc * nc;                                 // Xs[k * RT + t]
  const int RT = rows_per_cta;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RT;
  for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
    int k = idx % nc, j = idx / nc;
    Ls[j * nc + k] = (k <= j) ? (T)Lm[(size_t)(c0 + k) * ldl + (c0 + j)] : (T)0;
  }
  for (int idx = tid; idx < RT * nc; idx += blockDim.x) {
    int t = idx % RT, k = idx / RT;
    int r = row0 + t;
    Xs[k * RT + t] = (r < m) ? (T)A[(size_t)(c0 + k) * ld + (r0 + r)] : (T)0;
  }
  __syncthreads();
  for (int t = tid; t < RT; t += blockDim.x) {
    for (int j = 0; j < nc; ++j) {
      T s0 = Xs[j * RT + t], s1 = 0, s2 = 0, s3 = 0;
      const T* Lj = Ls + j * nc;
      int k = 0;
      for (; k + 3 < j; k += 4) {
        s0 -= Xs[k * RT + t] * Lj[k];
        s1 -= Xs[(k + 1) * RT + t] * Lj[k + 1];
        s2 -= Xs[(k + 2) * RT + t] * Lj[k + 2];
        s3 -= Xs[(k + 3) * RT + t] * Lj[k + 3];
      }
      for (; k < j; ++k) s0 -= Xs[k * RT + t] * Lj[k];
      Xs[j * RT + t] = ((s0 + s1) + (s2 + s3)) / Lj[j];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < RT * nc; idx += blockDim.x) {
    int t = idx % RT, k = idx / RT;
    int r = row0 + t;
    if (r < m) {
      A[(size_t)(c0 + k) * ld + (r0 + r)] = (double)Xs[k * RT + t];
      if (S32 != nullptr) S32[(size_t)(c0 + k) * ld32 + (r0 + r)] = (float)Xs[k * RT + t];
    }
  }
  if (S != nullptr) {
    bool over16 = false;
    for (int idx = tid; idx < RT * nc; idx += blockDim.x) {
      int k = idx % nc, t = idx / nc;
      int r = row0 + t;
      if (r < m) {
        const double v = (double)Xs[k * RT + t];
        over16 |= fabs(v) > (double)kF16Max;
        S[(size_t)(r0 + r) * lds + (c0 + k)] = __double2half(v);
      }
    }
    if (__any_sync(0xffffffffu, over16) && (tid & 31) == 0) atomicOr(err, DEV_ERR_RANGE16);
  }
}

// ---------------------------------------------------------------------------------------
// Leaf TRSM in FP64, right-looking in unit-diagonal form (the FP64 base case of Alg. 2):
// with Lt = L diag(1/l_kk) and Y = X diag(l_kk), Y Lt^T = B is a substitution without
// divisions, y_ij = b_ij - sum_{k<j} y_ik Lt_jk, and X = Y diag(1/l_kk) at the end.  A row of
// B is one half-warp's: lane q holds the row's columns q, q + 16, q + 32, ... (CPT of them);
// at step k the holder of y_ik passes it along the half-warp by a shuffle and every lane
// subtracts it from its columns j > k.  One dependent FMA per step sits on the row's chain
// (the substitution above divides and sums a column's whole row in each step), and 8 rows
// per CTA spread the FP64 work over many SMs.
// ---------------------------------------------------------------------------------------
constexpr int kR64Rows = 8;                        // rows of B per CTA (16 lanes each)
template <int CPT>
__global__ void __launch_bounds__(kR64Rows * 16)
trsm_rl64_kernel(double* __restrict__ A, int ld, int r0, int m, int c0, int nc, const double* __restrict__ Lm,
                 int ldl, __half* __restrict__ S, int lds, float* __restrict__ S32, int ld32,
                 const int* __restrict__ info, unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (*(volatile const int*)info != INT_MAX) return;
  double* Lt = reinterpret_cast<double*>(smem_raw);     // Lt[j * nc + k] = l_jk / l_kk, k < j
  double* rinv = Lt + (size_t)nc * nc;                   // 1 / l_kk
  const int tid = threadIdx.x, lane = tid & 31;
  const int q = tid & 15, rr = tid >> 4;
  const int row = blockIdx.x * kR64Rows + rr;
  const bool live = row < m;
  if (tid < nc) rinv[tid] = 1.0 / Lm[(size_t)(c0 + tid) * ldl + (c0 + tid)];
  // this lane's entries of B (all loads in flight before the staging of Lt is used)
  double y[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int j = q + 16 * c;
    y[c] = (live && j < nc) ? A[(size_t)(c0 + j) * ld + (r0 + row)] : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
    const int j = idx / nc, k = idx % nc;
    if (k < j) Lt[idx] = Lm[(size_t)(c0 + k) * ldl + (c0 + j)] * rinv[k];
  }
  __syncthreads();
  const int base = lane & 16;                            // the half-warp of this row
  // column panels of 16: while k runs through panel p only slots c >= p change, and the
  // panel loop is unrolled so that no FP64 instruction is issued for the others (on this
  // GPU the SM retires under two FP64 lane-FMAs per clock, predicated-off lanes included)
#pragma unroll
  for (int p = 0; p < CPT; ++p) {
    if (16 * p + 1 >= nc) break;
    const int kend = min(16 * p + 16, nc - 1);
    for (int k = 16 * p; k < kend; ++k) {
      const double v = __shfl_sync(0xffffffffu, y[p], base | (k & 15));   // y_ik from the lane holding column k
      const double* Lk = Lt + k;
      if (q > k - 16 * p && q + 16 * p < nc) y[p] = fma(-v, Lk[(size_t)(q + 16 * p) * nc], y[p]);
#pragma unroll
      for (int c = p + 1; c < CPT; ++c) {
        const int j = q + 16 * c;
        if (j < nc) y[c] = fma(-v, Lk[(size_t)j * nc], y[c]);
      }
    }
  }
  bool over16 = false;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int j = q + 16 * c;
    if (live && j < nc) {
      const double x = y[c] * rinv[j];
      A[(size_t)(c0 + j) * ld + (r0 + row)] = x;
      if (S32 != nullptr) S32[(size_t)(c0 + j) * ld32 + (r0 + row)] = (float)x;
      if (S != nullptr) {
        over16 |= fabs(x) > (double)kF16Max;
        S[(size_t)(r0 + row) * lds + (c0 + j)] = __double2half(x);
      }
    }
  }
  if (S != nullptr && __any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
}

// ---------------------------------------------------------------------------------------
// Leaf TRSM in FP32 through the inverse of the diagonal block: X = fl32(B) W^T with
// W = fl32(L)^{-1} precomputed by the leaf POTRF.  A tile of 16 rows is computed by 256
// threads: warp w the rows 2w and 2w + 1, each lane CPL consecutive columns; per k one load
// of W (16 bytes for CPL = 4) and one broadcast of B(row, k) per row feed 2 CPL FMAs.  With
// CPL = 4 one CTA owns the tile's 128 columns (about 76 KB of shared memory, two CTAs per
// SM); panels with fewer tiles than SMs use CPL = 2 or 1 and split the columns over a cluster
// of 2 or 4 CTAs.  The kernel is bound by the latency of its dependent FMA chains and of
// staging W, not by bandwidth.
// ---------------------------------------------------------------------------------------
constexpr int kT32Rows = 16;
constexpr int kT32Threads = 256;
constexpr int kT32WLD = 132;   // row stride (floats) of W and of the staged rows (16-byte rows)

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// CPL = output columns per lane: the CTA computes the 16 rows x C = 32 CPL columns
// jc0 .. jc0 + C - 1 of X (jc0 = blockIdx.y C), so small panels spread over more SMs.
// When a row tile is split over several CTAs (gridDim.y > 1) they form one cluster
// (1 x gridDim.y) and meet at a cluster barrier after all of them have staged B and before
// any writes X in place.  Every CTA reaches it: the only early exit reads `info`, which no
// kernel writes while this one runs, so all CTAs see the same value.
// w_done: W was written by a kernel that completed before the previous launch on this stream
// started (the host knows), so it is staged before the wait for that launch, under its tail.
template <int CPL>
__global__ void __launch_bounds__(kT32Threads)
trsm_inv32_kernel(double* __restrict__ A, int ld, int r0, int m, int c0, int nc,
                  const float* __restrict__ W, int ldw, __half* __restrict__ S, int lds,
                  float* __restrict__ S32, int ld32, const int* __restrict__ info, unsigned* __restrict__ err,
                  int w_done) {
  constexpr int C = 32 * CPL;
  constexpr int WLD = C + 4;                               // 16-byte rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int jc0 = blockIdx.y * C;                          // < nc: gridDim.y = ceil(nc / C)
  float* Ws = reinterpret_cast<float*>(smem_raw);          // Ws[k * WLD + jj] = W(jc0 + jj, k)
  float* Bs = Ws + 128 * WLD;                              // Bs[r * 132 + k] = B(row0 + r, k); later X
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kT32Rows;
  const bool vecw = (nc == 128) && ((ldw & 3) == 0) && ((reinterpret_cast<uintptr_t>(W) & 15) == 0);
  auto stage_w = [&]() {
    if (vecw) {
      for (int e = tid; e < 128 * (C / 4); e += kT32Threads) {
        const int k = e / (C / 4), q = e % (C / 4);
        cp_async16(Ws + k * WLD + 4 * q, W + (size_t)k * ldw + jc0 + 4 * q);
      }
    } else {
      for (int e = tid; e < 128 * C; e += kT32Threads) {
        const int k = e / C, jj = e % C, j = jc0 + jj;
        Ws[k * WLD + jj] = (j < nc && k < nc) ? W[(size_t)k * ldw + j] : 0.f;
      }
    }
  };
  if (w_done) stage_w();
  pdl_wait();
  pdl_trigger();
  if (*(volatile const int*)info != INT_MAX) {
    cp_async_wait_all();
    return;
  }
  if (!w_done) stage_w();
  // B: 8 values per thread, all loads in flight before the conversions
  double bv[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = tid + kT32Threads * u;                   // e = k * 16 + r: 16 rows of column k
    const int k = e >> 4, r = e & 15;
    const int gr = row0 + r;
    bv[u] = (k < nc && gr < m) ? __ldcg(A + (size_t)(c0 + k) * ld + (r0 + gr)) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = tid + kT32Threads * u;
    Bs[(e & 15) * kT32WLD + (e >> 4)] = (float)bv[u];
  }
  cp_async_wait_all();
  __syncthreads();
  if (gridDim.y > 1) cg::this_cluster().sync();             // every slice has read B
  // warp w: rows 2w, 2w + 1; lane: columns CPL lane .. CPL lane + CPL - 1
  const int ra = 2 * warp, rb = 2 * warp + 1;
  float xa[CPL], xb[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) xa[c] = xb[c] = 0.f;
  const float* Ba = Bs + ra * kT32WLD;
  const float* Bb = Bs + rb * kT32WLD;
#pragma unroll 8
  for (int k = 0; k < nc; ++k) {
    float w[CPL];
    if constexpr (CPL == 4) {
      const float4 v = *reinterpret_cast<const float4*>(Ws + k * WLD + 4 * lane);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (CPL == 2) {
      const float2 v = *reinterpret_cast<const float2*>(Ws + k * WLD + 2 * lane);
      w[0] = v.x; w[1] = v.y;
    } else {
      w[0] = Ws[k * WLD + lane];
    }
    const float a = Ba[k], b = Bb[k];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      xa[c] = fmaf(a, w[c], xa[c]);
      xb[c] = fmaf(b, w[c], xb[c]);
    }
  }
  __syncthreads();                                         // all reads of B done: reuse Bs for X
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    Bs[ra * kT32WLD + CPL * lane + c] = xa[c];
    Bs[rb * kT32WLD + CPL * lane + c] = xb[c];
  }
  __syncthreads();
  const int ncol = min(C, nc - jc0);
  // master (column-major): 16 consecutive rows of one column per half-warp
  for (int e = tid; e < ncol * kT32Rows; e += kT32Threads) {
    const int jj = e >> 4, r = e & 15;
    const int gr = row0 + r;
    if (gr < m) {
      A[(size_t)(c0 + jc0 + jj) * ld + (r0 + gr)] = (double)Bs[r * kT32WLD + jj];
      if (S32 != nullptr) S32[(size_t)(c0 + jc0 + jj) * ld32 + (r0 + gr)] = Bs[r * kT32WLD + jj];
    }
  }
  // FP16 shadow (row-major): consecutive columns of one row
  if (S != nullptr) {
    bool over16 = false;
    for (int e = tid; e < ncol * kT32Rows; e += kT32Threads) {
      const int r = e / ncol, jj = e - r * ncol;
      const int gr = row0 + r;
      if (gr < m) {
        const float v = Bs[r * kT32WLD + jj];
        over16 |= fabsf(v) > kF16Max;
        S[(size_t)(r0 + gr) * lds + (c0 + jc0 + jj)] = __float2half_rn(v);
      }
    }
    if (__any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
  }
}

}  // namespace

cudaError_t launch_potrf_leaf(double* A, int ld, int n, int col0, bool compute64, bool round16,
                              float* W32, int ldw, int* info, unsigned* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 128) return cudaErrorInvalidValue;
  if (compute64 && !round16 && n > 32) return launch_potrf_leaf_cluster(A, ld, n, col0, W32, ldw, info, s);
  const size_t smem = W32 ? (size_t)2 * 128 * kInvLD * 4 : 0;
  static unsigned long long attr_mask = 0;     // one opt-in to the largest footprint (n = 128, with W)
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    const int maxb = (int)((size_t)2 * 128 * kInvLD * 4);
    cudaError_t e = cudaFuncSetAttribute(potrf_leaf_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(potrf_leaf_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  if (compute64)
    (void)launch_pdl(potrf_leaf_kernel<double>, dim3(1), dim3(256), smem, s, A, ld, n, col0, round16 ? 1 : 0, W32, ldw, info, err);
  else
    (void)launch_pdl(potrf_leaf_kernel<float>, dim3(1), dim3(256), smem, s, A, ld, n, col0, round16 ? 1 : 0, W32, ldw, info, err);
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf64(double* A, int ld, int r0, int m, int c0, int nc,
                               __half* shadow16, int lds, float* shadow32, int ld32, const int* info, unsigned* err,
                               cudaStream_t s, const double* Lm, int ldl) {
  if (!Lm) {
    Lm = A;
    ldl = ld;
  }
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 144) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)nc * nc + (size_t)nc) * sizeof(double);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    const int mx = (int)(((size_t)144 * 144 + 144) * sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(trsm_rl64_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(trsm_rl64_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(trsm_rl64_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  const dim3 grid((m + kR64Rows - 1) / kR64Rows), block(kR64Rows * 16);
  if (nc <= 64)
    (void)launch_pdl(trsm_rl64_kernel<4>, grid, block, smem, s, A, ld, r0, m, c0, nc, Lm, ldl, shadow16, lds, shadow32,
                     ld32, info, err);
  else if (nc <= 128)
    (void)launch_pdl(trsm_rl64_kernel<8>, grid, block, smem, s, A, ld, r0, m, c0, nc, Lm, ldl, shadow16, lds, shadow32,
                     ld32, info, err);
  else
    (void)launch_pdl(trsm_rl64_kernel<9>, grid, block, smem, s, A, ld, r0, m, c0, nc, Lm, ldl, shadow16, lds, shadow32,
                     ld32, info, err);
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf32_subst(double* A, int ld, int r0, int m, int c0, int nc,
                                     __half* shadow16, int lds, float* shadow32, int ld32, const int* info,
                                     unsigned* err, cudaStream_t s, const double* Lm, int ldl) {
  if (!Lm) {
    Lm = A;
    ldl = ld;
  }
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 144) return cudaErrorInvalidValue;
  int RT = 64;
  size_t smem = ((size_t)nc * nc + (size_t)RT * nc) * sizeof(float);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(trsm_subst_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(((size_t)144 * 144 + (size_t)64 * 144) * sizeof(float)));
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  int grid = (m + RT - 1) / RT;
  (void)launch_pdl(trsm_subst_kernel<float>, dim3(grid), dim3(64), smem, s, A, ld, r0, m, c0, nc, Lm, ldl, shadow16, lds,
                   shadow32, ld32, info, err, RT);
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf32(double* A, int ld, int r0, int m, int c0, int nc,
                               const float* W, int ldw, __half* shadow16, int lds, float* shadow32, int ld32,
                               const int* info, unsigned* err, cudaStream_t s, bool w_done) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 128) return cudaErrorInvalidValue;
  const int sms = device_sm_count();
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(trsm_inv32_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((128 * 132 + kT32Rows * kT32WLD) * 4));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(trsm_inv32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((128 * 68 + kT32Rows * kT32WLD) * 4));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(trsm_inv32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((128 * 36 + kT32Rows * kT32WLD) * 4));
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  // row tiles of 16; panels with fewer row tiles than SMs split their columns over 2 or 4
  // CTAs (each then stages only its slice of W)
  const int gx = (m + kT32Rows - 1) / kT32Rows;
  const int cpl = gx >= sms ? 4 : (2 * gx >= sms ? 2 : 1);
  const int C = 32 * cpl;
  const dim3 grid(gx, (nc + C - 1) / C);
  const size_t smem = (size_t)(128 * (C + 4) + kT32Rows * kT32WLD) * 4;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kT32Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (launch_ctx().pdl) {                                  // see launch_pdl
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (grid.y > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = 1;
    at[na].val.clusterDim.y = grid.y;                      // the slices of one row tile
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  cudaError_t e;
  if (cpl == 4)
    e = cudaLaunchKernelEx(&cfg, trsm_inv32_kernel<4>, A, ld, r0, m, c0, nc, W, ldw, shadow16, lds, shadow32, ld32,
                           info, err, w_done ? 1 : 0);
  else if (cpl == 2)
    e = cudaLaunchKernelEx(&cfg, trsm_inv32_kernel<2>, A, ld, r0, m, c0, nc, W, ldw, shadow16, lds, shadow32, ld32,
                           info, err, w_done ? 1 : 0);
  else
    e = cudaLaunchKernelEx(&cfg, trsm_inv32_kernel<1>, A, ld, r0, m, c0, nc, W, ldw, shadow16, lds, shadow32, ld32,
                           info, err, w_done ? 1 : 0);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace hrp
