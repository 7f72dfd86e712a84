// POTRS: solve A X = B with the Cholesky factor, L Y = B then L^T X = Y.
//
// One launch per sweep.  The n rows are cut into 64-row blocks; each CTA takes the next
// block in the sweep order from an atomic ticket (so every block it waits for belongs to
// a CTA that started earlier and is resident: no deadlock), accumulates the off-diagonal
// products of already-solved blocks as soon as their ready flags are published
// (release/acquire at GPU scope), then substitutes through its 64 x 64 diagonal block with
// one warp per right-hand side (rows held two per lane, pivots broadcast by shuffles).
// Waits are bounded by %globaltimer; on expiry the CTA records DEV_ERR_TIMEOUT and stops.
#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int PB = 64;
constexpr int PT = 256;
constexpr int MAX_RHS = 16;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// thread 0 waits for flags[j] == epoch; returns false on timeout
__device__ bool wait_flag(const int* flags, int j, int epoch) {
  if (ld_acquire(flags + j) == epoch) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (ld_acquire(flags + j) == epoch) return true;
    if (gtimer() - t0 > kWaitTimeoutNs) return false;
  }
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(PT)
potrs_sweep_kernel(const double* __restrict__ L, int ldl, double* __restrict__ B, int ldb, int n, int nrhs,
                   int* __restrict__ ticket, int* __restrict__ flags, int epoch, unsigned* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ld = reinterpret_cast<T*>(smem_raw);   // diagonal block, Ld[k * 65 + i] = L(R0 + i, R0 + k)
  T* yS = Ld + PB * (PB + 1);               // solved block of another CTA
  T* accS = yS + MAX_RHS * PB;
  T* Ls = accS + MAX_RHS * PB;              // off-diagonal block (backward sweep staging)
  __shared__ int s_r, s_abort;
  const int tid = threadIdx.x;
  const int nb = (n + PB - 1) / PB;
  if (tid == 0) {
    int t = atomicAdd(ticket, 1);
    s_r = FWD ? t : nb - 1 - t;
    s_abort = 0;
  }
  __syncthreads();
  const int r = s_r;
  const int R0 = r * PB;
  const int rows = min(PB, n - R0);
  for (int idx = tid; idx < PB * PB; idx += PT) {
    int i = idx % PB, k = idx / PB;
    Ld[k * (PB + 1) + i] = (i < rows && k < rows && i >= k) ? (T)L[(size_t)(R0 + k) * ldl + R0 + i] : (T)0;
  }
  const int i = tid % PB, g = tid / PB;    // row i, rhs group g: columns g, g+4, g+8, g+12
  T acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int c = g + 4 * q;
    acc[q] = (c < nrhs && i < rows) ? (T)B[(size_t)c * ldb + R0 + i] : (T)0;
  }
  const int jbeg = FWD ? 0 : r + 1;
  const int jend = FWD ? r : nb;
  for (int j = jbeg; j < jend; ++j) {
    if (tid == 0 && !wait_flag(flags, j, epoch)) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();
    if (s_abort) return;
    const int J0 = j * PB;
    const int jrows = min(PB, n - J0);
    for (int idx = tid; idx < nrhs * PB; idx += PT) {
      int kk = idx % PB, c = idx / PB;
      yS[c * PB + kk] = (kk < jrows) ? (T)__ldcg(B + (size_t)c * ldb + J0 + kk) : (T)0;
    }
    if (!FWD) {
      // stage L(J0 + kk, R0 + i) as Ls[i * 65 + kk] (coalesced along kk)
      for (int idx = tid; idx < PB * PB; idx += PT) {
        int kk = idx % PB, ii = idx / PB;
        Ls[ii * (PB + 1) + kk] = (kk < jrows && ii < rows) ? (T)L[(size_t)(R0 + ii) * ldl + J0 + kk] : (T)0;
      }
    }
    __syncthreads();
    if (i < rows) {
      if (FWD) {
        for (int kk = 0; kk < jrows; ++kk) {
          const T l = (T)L[(size_t)(J0 + kk) * ldl + R0 + i];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (g + 4 * q < nrhs) acc[q] -= l * yS[(g + 4 * q) * PB + kk];
        }
      } else {
        for (int kk = 0; kk < jrows; ++kk) {
          const T l = Ls[i * (PB + 1) + kk];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (g + 4 * q < nrhs) acc[q] -= l * yS[(g + 4 * q) * PB + kk];
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int c = g + 4 * q;
    if (c < nrhs) accS[c * PB + i] = acc[q];
  }
  __syncthreads();
  // diagonal block: one warp per right-hand side, lane owns rows lane and lane + 32
  const int warp = tid >> 5, lane = tid & 31;
  for (int c = warp; c < nrhs; c += PT / 32) {
    T a0 = accS[c * PB + lane], a1 = accS[c * PB + lane + 32];
    if (FWD) {
      for (int k = 0; k < rows; ++k) {
        T v = __shfl_sync(0xffffffffu, (k < 32) ? a0 : a1, k & 31);
        T yk = v / Ld[k * (PB + 1) + k];
        if (k < 32) { if (lane == k) a0 = yk; } else { if (lane == k - 32) a1 = yk; }
        if (lane > k) a0 -= Ld[k * (PB + 1) + lane] * yk;
        if (lane + 32 > k) a1 -= Ld[k * (PB + 1) + lane + 32] * yk;
      }
    } else {
      for (int k = rows - 1; k >= 0; --k) {
        T v = __shfl_sync(0xffffffffu, (k < 32) ? a0 : a1, k & 31);
        T xk = v / Ld[k * (PB + 1) + k];
        if (k < 32) { if (lane == k) a0 = xk; } else { if (lane == k - 32) a1 = xk; }
        // rows i < k: a_i -= L(k, i) x_k
        if (lane < k) a0 -= Ld[lane * (PB + 1) + k] * xk;
        if (lane + 32 < k) a1 -= Ld[(lane + 32) * (PB + 1) + k] * xk;
      }
    }
    if (lane < rows) B[(size_t)c * ldb + R0 + lane] = (double)a0;
    if (lane + 32 < rows) B[(size_t)c * ldb + R0 + lane + 32] = (double)a1;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(flags + r, epoch);
}

template <typename T, bool FWD>
size_t potrs_smem() {
  return sizeof(T) * ((size_t)PB * (PB + 1) * (FWD ? 1 : 2) + 2 * (size_t)MAX_RHS * PB);
}

template <typename T, bool FWD>
cudaError_t potrs_launch_one(const double* L, int ldl, double* B, int ldb, int n, int nrhs, int* ticket, int* flags,
                             int epoch, unsigned* err, cudaStream_t s) {
  const size_t smem = potrs_smem<T, FWD>();
  cudaError_t e = cudaFuncSetAttribute(potrs_sweep_kernel<T, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nb = (n + PB - 1) / PB;
  potrs_sweep_kernel<T, FWD><<<nb, PT, smem, s>>>(L, ldl, B, ldb, n, nrhs, ticket, flags, epoch, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_potrs(const double* L, int ldl, double* B, int ldb, int n, int nrhs, bool fp32,
                         int* ticket, int* flags, int epoch, unsigned* dev_err, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  for (int c0 = 0; c0 < nrhs; c0 += MAX_RHS) {
    const int nc = nrhs - c0 < MAX_RHS ? nrhs - c0 : MAX_RHS;
    double* Bc = B + (size_t)c0 * ldb;
    for (int pass = 0; pass < 2; ++pass) {
      const int ep = epoch + 2 * (c0 / MAX_RHS) + pass;
      cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(int), s);
      if (e != cudaSuccess) return e;
      if (pass == 0)
        e = fp32 ? potrs_launch_one<float, true>(L, ldl, Bc, ldb, n, nc, ticket, flags, ep, dev_err, s)
                 : potrs_launch_one<double, true>(L, ldl, Bc, ldb, n, nc, ticket, flags, ep, dev_err, s);
      else
        e = fp32 ? potrs_launch_one<float, false>(L, ldl, Bc, ldb, n, nc, ticket, flags, ep, dev_err, s)
                 : potrs_launch_one<double, false>(L, ldl, Bc, ldb, n, nc, ticket, flags, ep, dev_err, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// number of epochs consumed by one launch_potrs call
int potrs_epochs(int nrhs) { return 2 * ((nrhs + MAX_RHS - 1) / MAX_RHS); }

}  // namespace hrp
