// SIMT GEMM for the FP64 and FP32 levels of the tree (and the FP16-operand fallback):
// C -= X Y^T on column-major views of the FP64 master.  This is the update
// "B2 <- B2 - B1 L21^T" of Alg. 2 and "C21 <- C21 - A2 A1^T" of Alg. 3 (alpha = -1,
// beta = 1 in Alg. 1); with `lower` it is the leaf SYRK of Alg. 3 on a diagonal block.
#include <cstdint>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

// inner-dimension slice per stage: 16 for FP64, 64 for FP32 accumulation (fewer
// latency-bound stages for the small GEMMs of the FP32 levels)
template <int RND> struct Slice { static constexpr int BK = 64; };
template <> struct Slice<0> { static constexpr int BK = 16; };

template <int RND> struct Acc { using T = float; };
template <> struct Acc<0> { using T = double; };

template <int RND>
__device__ __forceinline__ typename Acc<RND>::T cvt_op(double x) {
  if constexpr (RND == 0) return x;
  else if constexpr (RND == 1) return __double2float_rn(x);
  else return __half2float(__double2half(x));
}
// operands already in FP32 (the FP32 shadow of L): no rounding on load
template <int RND>
__device__ __forceinline__ float cvt_op(float x) { return x; }

// TL x TL tile (TL = 64 or 32), 256 threads; thread (tx, ty) = (tid % 16, tid / 16) owns
// rows tx + 16 i and columns ty + 16 j, i, j < TL / 16.
template <int RND, int TL, typename TIN = double>
__global__ void __launch_bounds__(256)
gemm_simt_kernel(double* __restrict__ C, int ldc, const TIN* __restrict__ X, int ldx,
                 const TIN* __restrict__ Y, int ldy, int m, int n, int k, int lower) {
  pdl_wait();
  pdl_trigger();
  using T = typename Acc<RND>::T;
  constexpr int BK = Slice<RND>::BK;
  constexpr int BM = TL, BN = TL, R = TL / 16;
  __shared__ T Xs[BK][BM + 1];
  __shared__ T Ys[BK][BN + 1];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (lower && m0 + BM - 1 < n0) return;          // tile strictly above the diagonal
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = (T)0;

  // register prefetch of the next BK slice while the current one is multiplied
  T px[(BM * BK) / 256], py[(BN * BK) / 256];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + 256 * q;
      const int r = e % BM, kk = e / BM;
      const int gr = m0 + r, gk = k0 + kk, gc = n0 + r;
      px[q] = (gr < m && gk < k) ? cvt_op<RND>(X[(size_t)gk * ldx + gr]) : (T)0;
      py[q] = (gc < n && gk < k) ? cvt_op<RND>(Y[(size_t)gk * ldy + gc]) : (T)0;
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + 256 * q;
      Xs[e / BM][e % BM] = px[q];
      Ys[e / BM][e % BM] = py[q];
    }
    __syncthreads();
    if (k0 + BK < k) fetch(k0 + BK);
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
  double cv[R][R];
#pragma unroll
  for (int j = 0; j < R; ++j)
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int gc = n0 + ty + 16 * j, gr = m0 + tx + 16 * i;
      const bool ok = gc < n && gr < m && !(lower && gr < gc);
      cv[i][j] = ok ? C[(size_t)gc * ldc + gr] : 0.0;
    }
#pragma unroll
  for (int j = 0; j < R; ++j)
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int gc = n0 + ty + 16 * j, gr = m0 + tx + 16 * i;
      const bool ok = gc < n && gr < m && !(lower && gr < gc);
      if (ok) C[(size_t)gc * ldc + gr] = cv[i][j] - (double)acc[i][j];
    }
}

// FP32 products of the FP32 levels with operands from the FP32 shadow, for large tiles:
// 128 x 128 outputs per CTA, 256 threads, 8 x 8 per thread (rows 4 tx + i and 64 + 4 tx + i,
// columns 4 ty + j and 64 + 4 ty + j), K in slices of 16 staged in shared memory (k-major,
// 16-byte loads and reads) with the next slice prefetched into registers.  The FP64 master
// update C -= acc is the epilogue; `lower` skips tiles above the diagonal and masks entries
// above it.
constexpr int SG_T = 128, SG_BK = 16;

__global__ void __launch_bounds__(256)
sgemm128_kernel(double* __restrict__ C, int ldc, const float* __restrict__ X, int ldx,
                const float* __restrict__ Y, int ldy, int m, int n, int k, int lower) {
  pdl_wait();
  pdl_trigger();
  __shared__ __align__(16) float Xs[SG_BK][SG_T];
  __shared__ __align__(16) float Ys[SG_BK][SG_T];
  const int m0 = blockIdx.x * SG_T, n0 = blockIdx.y * SG_T;
  if (lower && m0 + SG_T - 1 < n0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loader: thread t covers rows 4 (t % 32) .. +3 of slice rows kk = t / 32 and kk + 8
  const int lr = 4 * (tid & 31), lk = tid >> 5;
  const bool fullm = m0 + SG_T <= m, fulln = n0 + SG_T <= n;
  float4 px[2], py[2];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gk = k0 + lk + 8 * h;
      if (gk < k && fullm) {
        px[h] = *reinterpret_cast<const float4*>(X + (size_t)gk * ldx + m0 + lr);
      } else {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (gk < k && m0 + lr + q < m) ? X[(size_t)gk * ldx + m0 + lr + q] : 0.f;
        px[h] = make_float4(v[0], v[1], v[2], v[3]);
      }
      if (gk < k && fulln) {
        py[h] = *reinterpret_cast<const float4*>(Y + (size_t)gk * ldy + n0 + lr);
      } else {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (gk < k && n0 + lr + q < n) ? Y[(size_t)gk * ldy + n0 + lr + q] : 0.f;
        py[h] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  fetch(0);
  for (int k0 = 0; k0 < k; k0 += SG_BK) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      *reinterpret_cast<float4*>(&Xs[lk + 8 * h][lr]) = px[h];
      *reinterpret_cast<float4*>(&Ys[lk + 8 * h][lr]) = py[h];
    }
    __syncthreads();
    if (k0 + SG_BK < k) fetch(k0 + SG_BK);
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[kk][4 * tx]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[kk][64 + 4 * tx]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Ys[kk][4 * ty]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ys[kk][64 + 4 * ty]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int gc = n0 + (j < 4 ? 4 * ty + j : 64 + 4 * ty + (j - 4));
    if (gc >= n) continue;
    double cv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gr = m0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + (i - 4));
      cv[i] = (gr < m && !(lower && gr < gc)) ? C[(size_t)gc * ldc + gr] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gr = m0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + (i - 4));
      if (gr < m && !(lower && gr < gc)) C[(size_t)gc * ldc + gr] = cv[i] - (double)acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_gemm_simt(double* C, int ldc, const double* X, int ldx, const double* Y, int ldy,
                             int m, int n, int k, OpRound rnd, bool lower, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  // 64 x 64 tiles unless that leaves most SMs idle: the operand rounding and the FP64
  // read-modify-write of C run on the FP64 pipe, so the small products of the FP32 levels
  // are spread over 32 x 32 tiles
  const int sms = device_sm_count();
  const bool small = (long long)((m + 63) / 64) * ((n + 63) / 64) < sms;
  const int tl = small ? 32 : 64;
  dim3 grid((m + tl - 1) / tl, (n + tl - 1) / tl);
  if (grid.y > 65535) return cudaErrorInvalidValue;
#define HRP_SIMT(R_, T_) (void)launch_pdl(gemm_simt_kernel<R_, T_>, dim3(grid), dim3(256), 0, s, C, ldc, X, ldx, Y, ldy, m, n, k, lower)
  switch (rnd) {
    case OpRound::F64: if (small) HRP_SIMT(0, 32); else HRP_SIMT(0, 64); break;
    case OpRound::F32: if (small) HRP_SIMT(1, 32); else HRP_SIMT(1, 64); break;
    case OpRound::F16: if (small) HRP_SIMT(2, 32); else HRP_SIMT(2, 64); break;
  }
#undef HRP_SIMT
  return cudaGetLastError();
}

cudaError_t launch_gemm_simt_f32(double* C, int ldc, const float* X, int ldx, const float* Y, int ldy,
                                 int m, int n, int k, bool lower, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  const int sms = device_sm_count();
  // large products: 128 x 128 tiles once they cover the SMs (16-byte operand loads need
  // 16-byte aligned operand columns)
  const bool vec = (ldx % 4) == 0 && (ldy % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  if (vec && k >= 64 && (long long)((m + 127) / 128) * ((n + 127) / 128) >= sms / 2) {
    dim3 g128((m + 127) / 128, (n + 127) / 128);
    if (g128.y > 65535) return cudaErrorInvalidValue;
    (void)launch_pdl(sgemm128_kernel, dim3(g128), dim3(256), 0, s, C, ldc, X, ldx, Y, ldy, m, n, k, lower);
    return cudaGetLastError();
  }
  const bool small = (long long)((m + 63) / 64) * ((n + 63) / 64) < sms;
  const int tl = small ? 32 : 64;
  dim3 grid((m + tl - 1) / tl, (n + tl - 1) / tl);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (small)
    (void)launch_pdl(gemm_simt_kernel<1, 32, float>, dim3(grid), dim3(256), 0, s, C, ldc, X, ldx, Y, ldy, m, n, k, lower);
  else
    (void)launch_pdl(gemm_simt_kernel<1, 64, float>, dim3(grid), dim3(256), 0, s, C, ldc, X, ldx, Y, ldy, m, n, k, lower);
  return cudaGetLastError();
}

}  // namespace hrp
