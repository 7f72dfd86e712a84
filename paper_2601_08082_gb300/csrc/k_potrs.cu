// POTRS: solve A X = B with the Cholesky factor, L Y = B then L^T X = Y.
//
// Two launches per sweep pair plus one pre-pass:
//   1. inverse pre-pass: every 64 x 64 diagonal block L_rr is inverted in parallel (one
//      CTA per block, right-looking, all columns at once), W_r = L_rr^{-1}.
//   2. forward sweep: the rows are cut into 64-row blocks; each CTA takes the next block
//      in sweep order from an atomic ticket (every block it waits for belongs to a CTA
//      that started earlier and is resident: no deadlock).  As soon as a solved block's
//      ready flag is published (release/acquire at GPU scope) the CTA accumulates its
//      off-diagonal product, 4 threads per row each over 16 columns with all 16 loads in
//      flight; at the end y_r = W_r (b_r - sum_j L_rj y_j) is a small matrix product, so
//      no division sits on the dependency chain between blocks.
//   3. backward sweep, the same with L^T: x_r = W_r^T (y_r - sum_{j>r} L_jr^T x_j).
// Epochs: a block's ready flag holds the epoch of the sweep that solved it, so flags never
// need clearing between sweeps.  The epochs come from a device counter that the first
// kernel of every solve advances in stream order (and that clears the flags before the
// counter would overflow), so a solve captured in a CUDA graph takes fresh epochs on every
// replay.
// All waits are bounded by %globaltimer: on expiry the CTA records DEV_ERR_TIMEOUT, writes
// NaN into its own block of the solution and still publishes it, so blocks downstream turn
// NaN as well instead of waiting in turn; no flag is left unpublished.
#include <climits>

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
// true once flags[j] == epoch; false when limit_ns of %globaltimer have passed first
__device__ bool wait_flag(const int* flags, int j, int epoch, unsigned long long limit_ns) {
  if (ld_acquire(flags + j) == epoch) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    for (int i = 0; i < 16; ++i) {
      if (ld_acquire(flags + j) == epoch) return true;
      __nanosleep(64);
    }
    if (gtimer() - t0 > limit_ns) return false;
  }
}

// One thread waits through wait_flag on *flag reaching 1, which nothing writes: the wait
// must expire after limit_ns, record DEV_ERR_TIMEOUT and return.  out[0] = the time waited.
__global__ void wait_probe_kernel(const int* flag, unsigned long long limit_ns, unsigned* err,
                                  unsigned long long* out) {
  if (threadIdx.x != 0) return;
  const unsigned long long t0 = gtimer();
  if (!wait_flag(flag, 0, 1, limit_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
  out[0] = gtimer() - t0;
}

// ---- 0. epochs of this solve: epochs ctr + 1 .. ctr + ne, flags cleared on wrap-around ----
__global__ void __launch_bounds__(256) potrs_epoch_kernel(int* __restrict__ ctr, int* __restrict__ flags, int nflags,
                                                          int ne) {
  __shared__ int s_base;
  if (threadIdx.x == 0) {
    int base = ctr[0] + 1;
    if (base < 1 || base > INT_MAX - ne) base = -1;        // wrap: clear the flags first
    s_base = base;
  }
  __syncthreads();
  if (s_base < 0)
    for (int i = threadIdx.x; i < nflags; i += blockDim.x) flags[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) ctr[0] = (s_base < 0 ? 1 : s_base) + ne - 1;
}

// epoch q (0-based) of the solve whose epochs end at ctr[0]
__device__ __forceinline__ int solve_epoch(const int* ctr, int ne, int q) { return *(volatile const int*)ctr - ne + 1 + q; }

// ---- 1. W_r = L_rr^{-1} for every 64-row diagonal block (one CTA each) ----
template <typename T>
__global__ void __launch_bounds__(PT)
potrs_diag_inverse_kernel(const double* __restrict__ L, int ldl, int n, T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*Ls)[PB + 1] = reinterpret_cast<T (*)[PB + 1]>(smem_raw);               // Ls[i][k] = L(R0+i, R0+k)
  T (*Ws)[PB + 1] = reinterpret_cast<T (*)[PB + 1]>(smem_raw + sizeof(T) * PB * (PB + 1));  // W(i, c)
  __shared__ T rinv[PB];
  const int r = blockIdx.x, R0 = r * PB, rows = min(PB, n - R0);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < PB * PB; idx += PT) {
    const int i = idx % PB, k = idx / PB;
    const T v = (i < rows && k < rows && i >= k) ? (T)L[(size_t)(R0 + k) * ldl + R0 + i] : (T)0;
    Ls[i][k] = v;
    Ws[i][k] = (i == k) ? (T)1 : (T)0;      // right-hand side: the identity
  }
  __syncthreads();
  if (tid < PB) rinv[tid] = (tid < rows) ? (T)1 / Ls[tid][tid] : (T)1;
  __syncthreads();
  // right-looking forward substitution on all 64 columns of the identity at once:
  // step k finalizes row k (w_kc = acc_kc / l_kk) and removes it from rows i > k
  for (int k = 0; k < rows; ++k) {
    if (tid <= k) Ws[k][tid] *= rinv[k];
    __syncthreads();
    const int cnt = (rows - 1 - k) * (k + 1);   // (i > k) x (c <= k)
    for (int e = tid; e < cnt; e += PT) {
      const int i = k + 1 + e / (k + 1), c = e % (k + 1);
      Ws[i][c] -= Ls[i][k] * Ws[k][c];
    }
    __syncthreads();
  }
  // store W_r column-major (ld 64) at W + r * 64 * 64
  T* Wr = W + (size_t)r * PB * PB;
  for (int idx = tid; idx < PB * PB; idx += PT) {
    const int i = idx % PB, c = idx / PB;
    Wr[c * PB + i] = (i >= c && i < rows) ? Ws[i][c] : (T)0;
  }
}

// ---- 2/3. sweeps ----
template <typename T, bool FWD>
__global__ void __launch_bounds__(PT, 1)
potrs_sweep_kernel(const double* __restrict__ L, int ldl, const T* __restrict__ W, double* __restrict__ B, int ldb,
                   int n, int nrhs, int* __restrict__ ticket, int* __restrict__ flags, const int* __restrict__ ctr,
                   int ne, int q, unsigned* __restrict__ err, unsigned long long limit_ns) {
  __shared__ T yS[MAX_RHS][PB];          // solved block of another CTA; later the reduced rhs
  __shared__ T part[4][MAX_RHS][PB];     // per-chunk partial sums
  __shared__ int s_r, s_abort;
  T (*accS)[PB] = yS;
  const int tid = threadIdx.x;
  const int nb = (n + PB - 1) / PB;
  const int epoch = solve_epoch(ctr, ne, q);
  if (tid == 0) {
    const int t = atomicAdd(ticket, 1);
    s_r = FWD ? t : nb - 1 - t;
    s_abort = 0;
  }
  __syncthreads();
  const int r = s_r, R0 = r * PB, rows = min(PB, n - R0);
  const int i = tid % PB, ch = tid / PB;           // row i, k-chunk ch (16 columns each)
  T acc[MAX_RHS];
#pragma unroll
  for (int c = 0; c < MAX_RHS; ++c) acc[c] = (T)0;

  // this block's right-hand side does not depend on other blocks either: its DRAM latency
  // stays off the block-to-block chain (thread tid holds entries tid + PT u)
  constexpr int kBU = MAX_RHS * PB / PT;
  T bpre[kBU];
#pragma unroll
  for (int u = 0; u < kBU; ++u) {
    const int idx = tid + PT * u, ii = idx % PB, c = idx / PB;
    bpre[u] = (c < nrhs && ii < rows) ? (T)B[(size_t)c * ldb + R0 + ii] : (T)0;
  }
  // W_r does not depend on other blocks: fetch this thread's 16 entries now
  const T* Wr = W + (size_t)r * PB * PB;      // column-major, ld 64
  T wv[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int kk = ch * 16 + q;
    wv[q] = FWD ? Wr[kk * PB + i] : Wr[i * PB + kk];
  }
  // dependencies in the order they complete: j = 0, 1, .. (forward), nb-1, nb-2, .. (backward)
  const int ndep = FWD ? r : nb - 1 - r;
  for (int jj = 0; jj < ndep; ++jj) {
    const int j = FWD ? jj : nb - 1 - jj;
    const int J0 = j * PB, jrows = min(PB, n - J0);
    // this thread's 16 factor entries do not depend on the flag: load them first
    T lv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int kk = ch * 16 + q;
      if (FWD) lv[q] = (kk < jrows && i < rows) ? (T)L[(size_t)(J0 + kk) * ldl + R0 + i] : (T)0;
      else lv[q] = (kk < jrows && i < rows) ? (T)L[(size_t)(R0 + i) * ldl + J0 + kk] : (T)0;
    }
    if (tid == 0 && !wait_flag(flags, j, epoch, limit_ns)) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();
    if (s_abort) {
      // this block cannot be solved: NaN marks it (and, through the products, every block
      // that depends on it); publishing it spares those blocks a wait of their own
      for (int idx = tid; idx < nrhs * PB; idx += PT) {
        const int ii = idx % PB, c = idx / PB;
        if (ii < rows) B[(size_t)c * ldb + R0 + ii] = __longlong_as_double(0x7ff8000000000000ll);
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release(flags + r, epoch);
      return;
    }
    for (int idx = tid; idx < nrhs * PB; idx += PT) {
      const int kk = idx % PB, c = idx / PB;
      yS[c][kk] = (kk < jrows) ? (T)__ldcg(B + (size_t)c * ldb + J0 + kk) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MAX_RHS; ++c) {
      if (c < nrhs) {
        T s = (T)0;
#pragma unroll
        for (int q = 0; q < 16; ++q) s = fma(lv[q], yS[c][ch * 16 + q], s);
        acc[c] += s;
      }
    }
    __syncthreads();
  }
  // reduce the four chunks, subtract from the right-hand side
#pragma unroll
  for (int c = 0; c < MAX_RHS; ++c)
    if (c < nrhs) part[ch][c][i] = acc[c];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kBU; ++u) {
    const int idx = tid + PT * u, ii = idx % PB, c = idx / PB;
    if (c < nrhs) accS[c][ii] = bpre[u] - ((part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii]));
  }
  __syncthreads();
  // y_r = W_r acc (forward) or x_r = W_r^T acc (backward): row i, chunk ch of 16 columns
#pragma unroll
  for (int c = 0; c < MAX_RHS; ++c) {
    if (c < nrhs) {
      T s = (T)0;
#pragma unroll
      for (int q = 0; q < 16; ++q) s = fma(wv[q], accS[c][ch * 16 + q], s);
      part[ch][c][i] = s;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < nrhs * PB; idx += PT) {
    const int ii = idx % PB, c = idx / PB;
    if (ii < rows)
      B[(size_t)c * ldb + R0 + ii] =
          (double)((part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii]));
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release(flags + r, epoch);
}

template <typename T>
cudaError_t potrs_t(const double* L, int ldl, double* B, int ldb, int n, int nrhs, T* W, int* ticket, int* flags,
                    int* ctr, unsigned* err, unsigned long long limit_ns, cudaStream_t s) {
  const int nb = (n + PB - 1) / PB;
  const int ne = potrs_epochs(nrhs);
  const size_t smem = 2 * sizeof(T) * PB * (PB + 1);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  cudaError_t e;
  if (!(attr_mask & attr_bit)) {
    if ((e = cudaFuncSetAttribute(potrs_diag_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    attr_mask |= attr_bit;
  }
  potrs_epoch_kernel<<<1, 256, 0, s>>>(ctr, flags, nb, ne);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  potrs_diag_inverse_kernel<T><<<nb, PT, smem, s>>>(L, ldl, n, W);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int c0 = 0; c0 < nrhs; c0 += MAX_RHS) {
    const int nc = nrhs - c0 < MAX_RHS ? nrhs - c0 : MAX_RHS;
    double* Bc = B + (size_t)c0 * ldb;
    for (int pass = 0; pass < 2; ++pass) {
      const int q = 2 * (c0 / MAX_RHS) + pass;
      if ((e = cudaMemsetAsync(ticket, 0, sizeof(int), s)) != cudaSuccess) return e;
      if (pass == 0)
        potrs_sweep_kernel<T, true><<<nb, PT, 0, s>>>(L, ldl, W, Bc, ldb, n, nc, ticket, flags, ctr, ne, q, err, limit_ns);
      else
        potrs_sweep_kernel<T, false><<<nb, PT, 0, s>>>(L, ldl, W, Bc, ldb, n, nc, ticket, flags, ctr, ne, q, err, limit_ns);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

size_t potrs_workspace_bytes(int n) { return (size_t)((n + PB - 1) / PB) * PB * PB * sizeof(double); }

cudaError_t launch_potrs(const double* L, int ldl, double* B, int ldb, int n, int nrhs, bool fp32, void* work,
                         int* ticket, int* flags, int* epoch_ctr, unsigned* dev_err, cudaStream_t s,
                         unsigned long long wait_limit_ns) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (fp32)
    return potrs_t<float>(L, ldl, B, ldb, n, nrhs, static_cast<float*>(work), ticket, flags, epoch_ctr, dev_err,
                          wait_limit_ns, s);
  return potrs_t<double>(L, ldl, B, ldb, n, nrhs, static_cast<double*>(work), ticket, flags, epoch_ctr, dev_err,
                         wait_limit_ns, s);
}

cudaError_t launch_wait_probe(const int* flag, unsigned long long limit_ns, unsigned* dev_err,
                              unsigned long long* waited_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(flag, limit_ns, dev_err, waited_ns);
  return cudaGetLastError();
}

// two sweeps per chunk of MAX_RHS columns (written without forming nrhs + MAX_RHS - 1)
int potrs_epochs(int nrhs) { return 2 * (nrhs / MAX_RHS + (nrhs % MAX_RHS != 0)); }

size_t potrs_flag_count(int n) { return (size_t)((n + PB - 1) / PB); }

}  // namespace hrp
