// Persistent batched factorization: one launch factors every system of a batch.
//
// The host walks Alg. 1-3 for each system exactly as for a single factorization, but
// records the base cases and GEMMs it would launch (with the precision the tree gives each)
// as a list of operations.  This kernel runs one CTA per SM; a CTA takes the next system
// from an atomic ticket (the host orders the systems longest first, so the tickets hand
// them out in LPT order) and executes that system's operations in order, a CTA barrier
// between two of them, then takes the next system.  No CTA ever waits on another CTA: the
// operations of a system depend only on their predecessors in the same list.
//
// Operations (single-CTA versions of the stream path's kernels, same arithmetic classes):
//   POTRF  leaf Cholesky of a diagonal block, FP64, or FP32 (on FP16-rounded input for an
//          F16 leaf, result rounded to FP16), in registers, right-looking;
//   TRSM   leaf X L^T = B by substitution in FP64 or FP32 (one row per thread); it also
//          writes the FP32 and FP16 roundings of X into the system's shadows;
//   GEMM   C -= X Y^T, operands from the FP64 master (F64 levels) or the FP32 / FP16 shadow
//          (rounded once, when the leaf TRSM finished them: conversions from FP64 run on this
//          GPU's FP64 pipe), accumulated in FP64 or FP32, 64 x 64 tiles.
// A system whose leaf POTRF fails stops at once (its info holds the failing column).
#include <climits>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int BT = 256;          // threads per CTA

__device__ __forceinline__ double round_f16(double x) { return (double)__half2float(__double2half(x)); }

// Newton reciprocal square root from a single-precision seed (two steps in FP64, one in
// FP32); values outside the single-precision range take the library sqrt.
__device__ __forceinline__ double rsqrt_nt(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
#pragma unroll
  for (int it = 0; it < 2; ++it) r = fma(0.5 * r, fma(-d * r, r, 1.0), r);
  return r;
}
__device__ __forceinline__ float rsqrt_nt(float d) {
  const float r = rsqrtf(d);
  return fmaf(0.5f * r, fmaf(-d * r, r, 1.0f), r);
}

// ---- leaf POTRF of the n x n block at A (n <= 128): thread (ti, tj) = (t % 16, t / 16)
// holds entries (ti + 16 a, tj + 16 b); step k publishes the scaled column k in col ----
template <typename T>
__device__ void dev_potrf(double* __restrict__ A, int ld, int n, int col0, bool round16, int* __restrict__ info,
                          unsigned* __restrict__ err, T (*col)[128], int* s_fail) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = tid & 15, tj = tid >> 4;
  T reg[8][8];
  bool over16 = false;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ti + 16 * a, j = tj + 16 * b;
      double v = (i < n && j < n && i >= j) ? A[(size_t)j * ld + i] : 0.0;
      if (round16) {
        over16 |= fabs(v) > (double)kF16Max;
        v = round_f16(v);
      }
      reg[a][b] = (T)v;
    }
  if (round16 && __any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
  if (tid == 0) *s_fail = 0;
  __syncthreads();
#pragma unroll
  for (int KB = 0; KB < 8; ++KB) {
    if (16 * KB >= n) break;
    for (int kt = 0; kt < 16; ++kt) {
      const int k = 16 * KB + kt;
      if (k >= n) break;
      const int buf = k & 1;
      if (warp == (kt >> 1)) {
        const int src = ((kt & 1) << 4) + kt;
        const T d = __shfl_sync(0xffffffffu, reg[KB][KB], src);
        const bool mine = (tj == kt);
        if (!((d > (T)0) && isfinite((double)d))) {
          if (lane == src) {
            atomicMin(info, col0 + k + 1);
            *s_fail = 1;
          }
        } else if (mine) {
          const T r = rsqrt_nt(d);
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
      if (*s_fail) return;
      T ci[8], cj[8];
#pragma unroll
      for (int a = KB; a < 8; ++a) ci[a] = col[buf][ti + 16 * a];
#pragma unroll
      for (int b = KB; b < 8; ++b) cj[b] = col[buf][tj + 16 * b];
#pragma unroll
      for (int b = KB; b < 8; ++b) {
        if (b == KB && tj <= kt) continue;
#pragma unroll
        for (int a = b; a < 8; ++a) {
          if (a == b && ti < tj) continue;
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
        if (round16) {
          over16 |= fabs(v) > (double)kF16Max;
          v = round_f16(v);
        }
        A[(size_t)j * ld + i] = v;
      }
    }
  if (round16 && __any_sync(0xffffffffu, over16) && lane == 0) atomicOr(err, DEV_ERR_RANGE16);
}

// ---- leaf TRSM X L^T = B for B = A[r0:r0+m, c0:c0+nc], L = A[c0.., c0..] (nc <= 144), by
// substitution in T; rows in groups of RT, one row per thread (RT keeps L and the group
// within batched_interp_smem()) ----
template <typename T>
__device__ void dev_trsm(double* __restrict__ A, int ld, int r0, int m, int c0, int nc, float* __restrict__ s32,
                         __half* __restrict__ s16, int lds, unsigned* __restrict__ err, unsigned char* smem) {
  const int RT = sizeof(T) == 8 ? (nc > 128 ? 32 : 64) : 128;
  T* Ls = reinterpret_cast<T*>(smem);                 // row-major nc x nc
  T* Xs = Ls + nc * nc;                               // Xs[k * RT + t]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nc * nc; idx += BT) {
    const int k = idx % nc, j = idx / nc;
    Ls[j * nc + k] = (k <= j) ? (T)A[(size_t)(c0 + k) * ld + (c0 + j)] : (T)0;
  }
  for (int g0 = 0; g0 < m; g0 += RT) {
    __syncthreads();                                  // Ls ready / previous group stored
    for (int idx = tid; idx < RT * nc; idx += BT) {
      const int t = idx % RT, k = idx / RT;
      Xs[k * RT + t] = (g0 + t < m) ? (T)A[(size_t)(c0 + k) * ld + r0 + g0 + t] : (T)0;
    }
    __syncthreads();
    if (tid < RT) {
      for (int j = 0; j < nc; ++j) {
        T s0 = Xs[j * RT + tid], s1 = 0, s2 = 0, s3 = 0;
        const T* Lj = Ls + j * nc;
        int k = 0;
        for (; k + 3 < j; k += 4) {
          s0 -= Xs[k * RT + tid] * Lj[k];
          s1 -= Xs[(k + 1) * RT + tid] * Lj[k + 1];
          s2 -= Xs[(k + 2) * RT + tid] * Lj[k + 2];
          s3 -= Xs[(k + 3) * RT + tid] * Lj[k + 3];
        }
        for (; k < j; ++k) s0 -= Xs[k * RT + tid] * Lj[k];
        Xs[j * RT + tid] = ((s0 + s1) + (s2 + s3)) / Lj[j];
      }
    }
    __syncthreads();
    bool over16 = false;
    for (int idx = tid; idx < RT * nc; idx += BT) {
      const int t = idx % RT, k = idx / RT;
      if (g0 + t < m) {
        const double v = (double)Xs[k * RT + t];
        A[(size_t)(c0 + k) * ld + r0 + g0 + t] = v;
        if (s32) {
          const size_t o = (size_t)(c0 + k) * lds + r0 + g0 + t;
          s32[o] = (float)Xs[k * RT + t];
          // FP32 results round to FP16 from FP32 (the same value, off the FP64 pipe)
          if constexpr (sizeof(T) == 4) s16[o] = __float2half_rn(Xs[k * RT + t]);
          else s16[o] = __double2half(v);
          over16 |= fabs(v) > (double)kF16Max;
        }
      }
    }
    if (s32 && __any_sync(0xffffffffu, over16) && (tid & 31) == 0) atomicOr(err, DEV_ERR_RANGE16);
  }
}

// ---- C[m x n] -= X Y^T (column-major views of the master), operands rounded per RND
// (0 FP64, 1 FP32, 2 FP16) and accumulated in FP64 (RND 0) or FP32; lower: only entries
// with row >= column.  64 x 64 tiles, thread (tx, ty) = (t % 16, t / 16) owns 4 x 4 ----
template <int RND> struct BAcc { using T = float; };
template <> struct BAcc<0> { using T = double; };

__device__ __forceinline__ double bload(double x) { return x; }
__device__ __forceinline__ float bload(float x) { return x; }
__device__ __forceinline__ float bload(__half x) { return __half2float(x); }

// TIN: operand storage (double master, float or __half shadow); RND 0 accumulates in FP64
template <int RND, typename TIN>
__device__ void dev_gemm(double* __restrict__ C, int ldc, const TIN* __restrict__ X, int ldx,
                         const TIN* __restrict__ Y, int ldy, int m, int n, int k, bool lower,
                         unsigned char* smem) {
  using T = typename BAcc<RND>::T;
  constexpr int TL = 64, BK = 16, R = TL / 16;
  T (*Xs)[TL + 1] = reinterpret_cast<T (*)[TL + 1]>(smem);
  T (*Ys)[TL + 1] = reinterpret_cast<T (*)[TL + 1]>(smem + sizeof(T) * BK * (TL + 1));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int gm = (m + TL - 1) / TL, gn = (n + TL - 1) / TL;
  for (int tile = 0; tile < gm * gn; ++tile) {
    const int m0 = (tile % gm) * TL, n0 = (tile / gm) * TL;
    if (lower && m0 + TL - 1 < n0) continue;          // uniform over the CTA
    T acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] = (T)0;
    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
      for (int q = 0; q < (TL * BK) / BT; ++q) {
        const int e = tid + BT * q;
        const int r = e % TL, kk = e / TL;
        const int gk = k0 + kk;
        Xs[kk][r] = (m0 + r < m && gk < k) ? (T)bload(X[(size_t)gk * ldx + m0 + r]) : (T)0;
        Ys[kk][r] = (n0 + r < n && gk < k) ? (T)bload(Y[(size_t)gk * ldy + n0 + r]) : (T)0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = Xs[kk][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Ys[kk][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int gc = n0 + ty + 16 * j, gr = m0 + tx + 16 * i;
        if (gc < n && gr < m && !(lower && gr < gc)) C[(size_t)gc * ldc + gr] -= (double)acc[i][j];
      }
  }
}

__global__ void __launch_bounds__(BT, 1)
batched_interp_kernel(const BatchOp* __restrict__ ops, const BatchSys* __restrict__ sys, int nsys,
                      int* __restrict__ ticket, unsigned* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double col64[2][128];
  __shared__ float col32[2][128];
  __shared__ int s_fail, s_sys;
  while (true) {
    if (threadIdx.x == 0) s_sys = atomicAdd(ticket, 1);
    __syncthreads();
    const int si = s_sys;
    __syncthreads();                                  // s_sys is rewritten next round
    if (si >= nsys) break;
    const BatchSys S = sys[si];
    if (threadIdx.x == 0) *S.info = INT_MAX;
    if (S.src)                                         // factor a copy: the lower triangle of src
      for (long long e = threadIdx.x; e < (long long)S.n * S.n; e += BT) {
        const int i = (int)(e % S.n), j = (int)(e / S.n);
        if (i >= j) S.A[(size_t)j * S.lda + i] = S.src[(size_t)j * S.ldsrc + i];
      }
    __syncthreads();
    for (int o = S.op0; o < S.op1; ++o) {
      if (*(volatile int*)S.info != INT_MAX) break;  // a leaf failed: every thread read it after the barrier
      const BatchOp op = ops[o];
      double* A = S.A;
      const int ld = S.lda;
      switch (op.type) {
        case BOP_POTRF: {
          double* blk = A + (size_t)op.a * ld + op.a;
          if (op.p == HRP_F64) dev_potrf<double>(blk, ld, op.b, op.a, false, S.info, err, col64, &s_fail);
          else dev_potrf<float>(blk, ld, op.b, op.a, op.p == HRP_F16, S.info, err, col32, &s_fail);
          break;
        }
        case BOP_TRSM:
          if (op.e) dev_trsm<double>(A, ld, op.a, op.b, op.c, op.d, S.s32, S.s16, S.n, err, smem);
          else dev_trsm<float>(A, ld, op.a, op.b, op.c, op.d, S.s32, S.s16, S.n, err, smem);
          break;
        case BOP_GEMM: {
          double* C = A + (size_t)op.c * ld + op.a;
          const size_t xo = (size_t)op.e * S.n + op.a, yo = (size_t)op.e * S.n + op.c;
          if (op.p == HRP_F64)
            dev_gemm<0>(C, ld, A + (size_t)op.e * ld + op.a, ld, A + (size_t)op.e * ld + op.c, ld, op.b, op.d, op.f,
                        op.g != 0, smem);
          else if (op.p == HRP_F32)
            dev_gemm<1>(C, ld, S.s32 + xo, S.n, S.s32 + yo, S.n, op.b, op.d, op.f, op.g != 0, smem);
          else
            dev_gemm<2>(C, ld, S.s16 + xo, S.n, S.s16 + yo, S.n, op.b, op.d, op.f, op.g != 0, smem);
          break;
        }
        default:
          break;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && *(volatile int*)S.info == INT_MAX) *S.info = 0;
    __syncthreads();
  }
}

}  // namespace

// Dynamic shared memory of the interpreter: the FP64 TRSM staging is the largest, nc = 144
// with 32-row groups (144^2 + 32 * 144 doubles) or nc = 128 with 64-row groups.
size_t batched_interp_smem() { return ((size_t)144 * 144 + (size_t)32 * 144) * sizeof(double); }

cudaError_t launch_batched_interp(const BatchOp* ops, const BatchSys* sys, int nsys, int* ticket, unsigned* err,
                                  cudaStream_t s) {
  if (nsys <= 0) return cudaSuccess;
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(batched_interp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_interp_smem());
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = nsys < device_sm_count() ? nsys : device_sm_count();
  batched_interp_kernel<<<grid, BT, batched_interp_smem(), s>>>(ops, sys, nsys, ticket, err);
  return cudaGetLastError();
}

}  // namespace hrp
