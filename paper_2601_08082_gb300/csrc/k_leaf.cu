// Leaf kernels of the recursion (Alg. 1 and Alg. 2 base cases): POTRF of a diagonal
// block staged in shared memory, and TRSM_{R,L,T} of a row panel against it.
#include <climits>
#include <cstdio>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

__device__ __forceinline__ double round_to_f16(double x) { return (double)__half2float(__double2half(x)); }

// ---------------------------------------------------------------------------------------
// Leaf POTRF (Alg. 1 base case "A <- POTRF_L(A)") of an n x n block, n <= 128, one CTA.
// Right-looking column Cholesky in shared memory: for each column k the pivot
// l_kk = sqrt(a_kk) is checked (positive and finite), the column below is divided by it
// and the trailing lower triangle receives the rank-1 update.  Optionally the FP32
// inverse W = fl32(L)^{-1} is formed afterwards (column j of W by forward substitution
// against e_j) for the FP32 leaf TRSM kernel.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
potrf_leaf_kernel(double* __restrict__ A, int ld, int n, int col0, int round16,
                  float* __restrict__ W32, int ldw, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_fail;
  if (*(volatile int*)info != INT_MAX) return;   // an earlier block failed: stop like LAPACK
  T* a = reinterpret_cast<T*>(smem_raw);
  const int lda_s = n + 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;

  for (int idx = tid; idx < n * n; idx += nthr) {
    int i = idx % n, j = idx / n;
    if (i >= j) {
      double v = A[(size_t)j * ld + i];
      if (round16) v = round_to_f16(v);
      a[j * lda_s + i] = (T)v;
    }
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      T d = a[k * lda_s + k];
      if (!(d > (T)0) || !isfinite((double)d)) {
        s_fail = 1;
        atomicMin(info, col0 + k + 1);
      } else {
        a[k * lda_s + k] = dsqrt<T>(d);
      }
    }
    __syncthreads();
    if (s_fail) return;
    const T piv = a[k * lda_s + k];
    for (int i = k + 1 + tid; i < n; i += nthr) a[k * lda_s + i] = a[k * lda_s + i] / piv;
    __syncthreads();
    // trailing update: warp w owns columns j = k+1+w, k+1+w+nwarps, ...; lanes own rows i >= j
    for (int j = k + 1 + warp; j < n; j += nwarps) {
      const T ljk = a[k * lda_s + j];
      for (int i = j + lane; i < n; i += 32) a[j * lda_s + i] -= a[k * lda_s + i] * ljk;
    }
    __syncthreads();
  }

  for (int idx = tid; idx < n * n; idx += nthr) {
    int i = idx % n, j = idx / n;
    if (i >= j) {
      double v = (double)a[j * lda_s + i];
      if (round16) {               // F16 leaf: the stored factor is rounded to FP16
        v = round_to_f16(v);
        a[j * lda_s + i] = (T)v;
      }
      A[(size_t)j * ld + i] = v;
    }
  }
  if (W32 == nullptr) return;
  __syncthreads();

  // ---- FP32 inverse W = fl32(L)^{-1} (lower triangular) ----
  float* Lf = reinterpret_cast<float*>(smem_raw);          // n x (n+1), column-major
  float* Wt = Lf + n * lda_s;                               // Wt[i * lda_s + j] = W(i, j)
  // Lf may overlap a when T == double: read everything into registers first, column by column
  if (sizeof(T) == sizeof(double)) {
    for (int j = 0; j < n; ++j) {
      // gather column j of a (double) then store as float; process in chunks to avoid overlap
      float v0 = 0.f;
      int i = tid;
      if (i < n) v0 = (i >= j) ? (float)a[j * lda_s + i] : 0.f;
      __syncthreads();
      // the float column j occupies bytes [4*j*lda_s, 4*(j+1)*lda_s) which lie inside double
      // columns < j/2+1 <= j, already consumed
      if (i < n) Lf[j * lda_s + i] = v0;
      __syncthreads();
    }
  } else {
    for (int idx = tid; idx < n * n; idx += nthr) {
      int i = idx % n, j = idx / n;
      if (i < j) Lf[j * lda_s + i] = 0.f;
      else Lf[j * lda_s + i] = (float)a[j * lda_s + i];
    }
    __syncthreads();
  }
  // thread j computes column j of W: w_i = (delta_ij - sum_{kk<i} L_i,kk w_kk) / L_ii
  if (tid < n) {
    const int j = tid;
    const int kstart = (j / 32) * 32;      // w_kk = 0 for kk < j, skip whole warps' worth
    for (int i = 0; i < kstart && i < n; ++i) Wt[i * lda_s + j] = 0.f;
    for (int i = kstart; i < n; ++i) {
      float s0 = (i == j) ? 1.f : 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int kk = kstart;
      for (; kk + 3 < i; kk += 4) {
        s0 -= Lf[kk * lda_s + i] * Wt[kk * lda_s + j];
        s1 -= Lf[(kk + 1) * lda_s + i] * Wt[(kk + 1) * lda_s + j];
        s2 -= Lf[(kk + 2) * lda_s + i] * Wt[(kk + 2) * lda_s + j];
        s3 -= Lf[(kk + 3) * lda_s + i] * Wt[(kk + 3) * lda_s + j];
      }
      for (; kk < i; ++kk) s0 -= Lf[kk * lda_s + i] * Wt[kk * lda_s + j];
      float w = ((s0 + s1) + (s2 + s3)) / Lf[i * lda_s + i];
      Wt[i * lda_s + j] = (i < j) ? 0.f : w;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nthr) {
    int i = idx % n, j = idx / n;
    W32[(size_t)j * ldw + i] = (i >= j) ? Wt[i * lda_s + j] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// Leaf TRSM in FP64 (Alg. 2 base case "B <- TRSM(...; L, B)", right side, lower,
// transposed): each thread owns one row of B and substitutes column by column,
// x_j = (b_j - sum_{k<j} x_k l_jk) / l_jj.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(64)
trsm_subst_kernel(double* __restrict__ A, int ld, int r0, int m, int c0, int nc,
                  __half* __restrict__ S, int lds, const int* __restrict__ info, int rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (*(volatile const int*)info != INT_MAX) return;
  T* Ls = reinterpret_cast<T*>(smem_raw);              // row-major nc x nc: Ls[j * nc + k]
  T* Xs = Ls + nc * nc;                                 // Xs[k * RT + t]
  const int RT = rows_per_cta;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RT;
  for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
    int k = idx % nc, j = idx / nc;
    Ls[j * nc + k] = (k <= j) ? (T)A[(size_t)(c0 + k) * ld + (c0 + j)] : (T)0;
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
    if (r < m) A[(size_t)(c0 + k) * ld + (r0 + r)] = (double)Xs[k * RT + t];
  }
  if (S != nullptr) {
    for (int idx = tid; idx < RT * nc; idx += blockDim.x) {
      int k = idx % nc, t = idx / nc;
      int r = row0 + t;
      if (r < m) S[(size_t)(r0 + r) * lds + (c0 + k)] = __double2half((double)Xs[k * RT + t]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Leaf TRSM in FP32 through the inverse of the diagonal block: X = fl32(B) W^T with
// W = fl32(L)^{-1} precomputed by the leaf POTRF.  One CTA owns 64 full rows of the
// panel (so reading B and writing X in place never race), 256 threads, each thread a
// 4-row x (nc/16)-column register tile.
// ---------------------------------------------------------------------------------------
constexpr int kT32Rows = 64;

__global__ void __launch_bounds__(256)
trsm_inv32_kernel(double* __restrict__ A, int ld, int r0, int m, int c0, int nc,
                  const float* __restrict__ W, int ldw, __half* __restrict__ S, int lds,
                  const int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (*(volatile const int*)info != INT_MAX) return;
  float* Bs = reinterpret_cast<float*>(smem_raw);       // Bs[k * 64 + r]
  float* Ws = Bs + nc * kT32Rows;                       // Ws[k * ncp + j] = W(j, k)
  const int ncp = nc + 1;
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * kT32Rows;
  for (int idx = tid; idx < kT32Rows * nc; idx += 256) {
    int r = idx % kT32Rows, k = idx / kT32Rows;
    int gr = row0 + r;
    Bs[k * kT32Rows + r] = (gr < m) ? (float)A[(size_t)(c0 + k) * ld + (r0 + gr)] : 0.f;
  }
  for (int idx = tid; idx < nc * nc; idx += 256) {
    int j = idx % nc, k = idx / nc;                     // W stored column-major: W[k*ldw + j] = W(j,k)
    Ws[k * ncp + j] = W[(size_t)k * ldw + j];
  }
  __syncthreads();
  const int rq = (tid & 15) * 4;                        // rows rq..rq+3
  const int cg = tid >> 4;                              // columns cg, cg+16, ...
  constexpr int MAXC = 9;                               // nc <= 144
  float acc[4][MAXC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < MAXC; ++c) acc[a][c] = 0.f;
  const int ncol = (nc - cg + 15) / 16;
  for (int k = 0; k < nc; ++k) {
    float4 b = *reinterpret_cast<const float4*>(&Bs[k * kT32Rows + rq]);
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      if (c < ncol) {
        float w = Ws[k * ncp + cg + 16 * c];
        acc[0][c] += b.x * w;
        acc[1][c] += b.y * w;
        acc[2][c] += b.z * w;
        acc[3][c] += b.w * w;
      }
    }
  }
  __syncthreads();
  // stage X (float) back into Bs, then write master and shadow coalesced
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    if (c < ncol) {
      int j = cg + 16 * c;
#pragma unroll
      for (int a = 0; a < 4; ++a) Bs[j * kT32Rows + rq + a] = acc[a][c];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kT32Rows * nc; idx += 256) {
    int r = idx % kT32Rows, k = idx / kT32Rows;
    int gr = row0 + r;
    if (gr < m) A[(size_t)(c0 + k) * ld + (r0 + gr)] = (double)Bs[k * kT32Rows + r];
  }
  if (S != nullptr) {
    for (int idx = tid; idx < kT32Rows * nc; idx += 256) {
      int k = idx % nc, r = idx / nc;
      int gr = row0 + r;
      if (gr < m) S[(size_t)(r0 + gr) * lds + (c0 + k)] = __double2half((double)Bs[k * kT32Rows + r]);
    }
  }
}

}  // namespace

cudaError_t launch_potrf_leaf(double* A, int ld, int n, int col0, bool compute64, bool round16,
                              float* W32, int ldw, int* info, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 128) return cudaErrorInvalidValue;
  size_t bytes_a = (size_t)n * (n + 1) * (compute64 ? 8 : 4);
  size_t bytes_w = W32 ? (size_t)2 * n * (n + 1) * 4 : 0;
  size_t smem = bytes_a > bytes_w ? bytes_a : bytes_w;
  if (!compute64 && W32) smem = bytes_a + (size_t)n * (n + 1) * 4;
  cudaError_t e;
  if (compute64) {
    e = cudaFuncSetAttribute(potrf_leaf_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    potrf_leaf_kernel<double><<<1, 256, smem, s>>>(A, ld, n, col0, round16 ? 1 : 0, W32, ldw, info);
  } else {
    e = cudaFuncSetAttribute(potrf_leaf_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    potrf_leaf_kernel<float><<<1, 256, smem, s>>>(A, ld, n, col0, round16 ? 1 : 0, W32, ldw, info);
  }
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf64(double* A, int ld, int r0, int m, int c0, int nc,
                               __half* shadow16, int lds, const int* info, cudaStream_t s) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 144) return cudaErrorInvalidValue;
  int RT = nc <= 128 ? 64 : 32;
  size_t smem = ((size_t)nc * nc + (size_t)RT * nc) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(trsm_subst_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (m + RT - 1) / RT;
  trsm_subst_kernel<double><<<grid, 64, smem, s>>>(A, ld, r0, m, c0, nc, shadow16, lds, info, RT);
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf32_subst(double* A, int ld, int r0, int m, int c0, int nc,
                                     __half* shadow16, int lds, const int* info, cudaStream_t s) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 144) return cudaErrorInvalidValue;
  int RT = 64;
  size_t smem = ((size_t)nc * nc + (size_t)RT * nc) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(trsm_subst_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (m + RT - 1) / RT;
  trsm_subst_kernel<float><<<grid, 64, smem, s>>>(A, ld, r0, m, c0, nc, shadow16, lds, info, RT);
  return cudaGetLastError();
}

cudaError_t launch_trsm_leaf32(double* A, int ld, int r0, int m, int c0, int nc,
                               const float* W, int ldw, __half* shadow16, int lds,
                               const int* info, cudaStream_t s) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if (nc > 144) return cudaErrorInvalidValue;
  size_t smem = ((size_t)nc * kT32Rows + (size_t)nc * (nc + 1)) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(trsm_inv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (m + kT32Rows - 1) / kT32Rows;
  trsm_inv32_kernel<<<grid, 256, smem, s>>>(A, ld, r0, m, c0, nc, W, ldw, shadow16, lds, info);
  return cudaGetLastError();
}

}  // namespace hrp
