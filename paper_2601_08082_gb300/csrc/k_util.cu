// Small device utilities of the solver: info handling, copies, the FP64 residual of the
// refinement loop (R = B - A X with A read once from its lower triangle), column norms,
// and the FP64 backward error ||A - L L^T||_F / ||A||_F (Sec. 4.2 accuracy metric).
#include <climits>

#include <algorithm>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

__global__ void fill_int_kernel(int* p, int v, int count) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}
__global__ void finalize_info_kernel(int* info) {
  pdl_wait();
  pdl_trigger();
  if (*info == INT_MAX) *info = 0;
}
__global__ void copy_lower_kernel(double* dst, int ldd, const double* src, int lds, int n) {
  pdl_wait();
  pdl_trigger();
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * n;
  for (; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    if (i >= j) dst[(size_t)j * ldd + i] = src[(size_t)j * lds + i];
  }
}
__global__ void copy_matrix_kernel(double* dst, int ldd, const double* src, int lds, int m, int n) {
  pdl_wait();
  pdl_trigger();
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)m * n;
  for (; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % m), j = (int)(idx / m);
    dst[(size_t)j * ldd + i] = src[(size_t)j * lds + i];
  }
}
__global__ void axpy_matrix_kernel(double* X, int ldx, const double* D, int ldd, int n, int nrhs) {
  pdl_wait();
  pdl_trigger();
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * nrhs;
  for (; idx < tot; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    X[(size_t)j * ldx + i] += D[(size_t)j * ldd + i];
  }
}

// ---- residual R -= A X over lower-triangle tiles (R preset to B) ----
constexpr int RT = 64;
constexpr int RNRHS = 16;

__device__ __forceinline__ void tri_index(long long t, int& I, int& J) {
  long long i = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = (int)i;
  J = (int)(t - i * (i + 1) / 2);
}

__global__ void __launch_bounds__(256)
residual_tile_kernel(const double* __restrict__ A, int lda, const double* __restrict__ X, int ldx,
                     double* __restrict__ R, int ldr, int n, int nrhs) {
  pdl_wait();
  pdl_trigger();
  __shared__ double As[RT][RT + 1];
  __shared__ double xI[RNRHS][RT];
  __shared__ double xJ[RNRHS][RT];
  int I, J;
  tri_index(blockIdx.x, I, J);
  const int I0 = I * RT, J0 = J * RT;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < RT * RT; idx += 256) {
    int i = idx % RT, j = idx / RT;
    int gi = I0 + i, gj = J0 + j;
    As[i][j] = (gi < n && gj < n && gi >= gj) ? A[(size_t)gj * lda + gi] : 0.0;
  }
  for (int idx = tid; idx < RT * nrhs; idx += 256) {
    int i = idx % RT, c = idx / RT;
    xI[c][i] = (I0 + i < n) ? X[(size_t)c * ldx + I0 + i] : 0.0;
    xJ[c][i] = (J0 + i < n) ? X[(size_t)c * ldx + J0 + i] : 0.0;
  }
  __syncthreads();
  const int i = tid % RT, g = tid / RT;          // 4 groups of right-hand sides
  for (int c = g; c < nrhs; c += 4) {
    // row i of block I: sum_j A(I0+i, J0+j) x(J0+j), using symmetry inside a diagonal tile
    double y = 0.0;
    if (I == J) {
      for (int j = 0; j < RT; ++j) y += (j <= i ? As[i][j] : As[j][i]) * xJ[c][j];
    } else {
      for (int j = 0; j < RT; ++j) y += As[i][j] * xJ[c][j];
    }
    if (I0 + i < n) atomicAdd(R + (size_t)c * ldr + I0 + i, -y);
    if (I != J) {
      double z = 0.0;                          // row i of block J: sum_r A(I0+r, J0+i) x(I0+r)
      for (int r = 0; r < RT; ++r) z += As[r][i] * xI[c][r];
      if (J0 + i < n) atomicAdd(R + (size_t)c * ldr + J0 + i, -z);
    }
  }
}

__global__ void col_norms2_kernel(const double* R, int ldr, const double* B, int ldb, int n, int nrhs, double* out) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  double sr = 0.0, sb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double r = R[(size_t)c * ldr + i], b = B[(size_t)c * ldb + i];
    sr += r * r;
    sb += b * b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out + c, sr);
    atomicAdd(out + nrhs + c, sb);
  }
}

// ---- backward error: tiles (I >= J) of L L^T in FP64, 64 x 64, BK = 16 ----
__global__ void __launch_bounds__(256)
backward_error_kernel(const double* __restrict__ A, int lda, const double* __restrict__ L, int ldl, int n,
                      double* __restrict__ out) {
  __shared__ double Xs[16][65];
  __shared__ double Ys[16][65];
  __shared__ double red[2][8];
  int I, J;
  tri_index(blockIdx.x, I, J);
  const int m0 = I * 64, n0 = J * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4] = {};
  const int kend = min(n, n0 + 64);             // L(j, k) = 0 for k > j
  for (int k0 = 0; k0 < kend; k0 += 16) {
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int r = e % 64, kk = e / 64;
      int gk = k0 + kk;
      int gr = m0 + r, gc = n0 + r;
      Xs[kk][r] = (gr < n && gk <= gr) ? L[(size_t)gk * ldl + gr] : 0.0;
      Ys[kk][r] = (gc < n && gk <= gc) ? L[(size_t)gk * ldl + gc] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
      for (int i = 0; i < 4; ++i) a[i] = Xs[kk][tx + 16 * i];
      for (int j = 0; j < 4; ++j) b[j] = Ys[kk][ty + 16 * j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double se = 0.0, sa = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int gr = m0 + tx + 16 * i, gc = n0 + ty + 16 * j;
      if (gr < n && gc < n && gr >= gc) {
        double a = A[(size_t)gc * lda + gr];
        double d = a - acc[i][j];
        double w = (gr == gc) ? 1.0 : 2.0;
        se += w * d * d;
        sa += w * a * a;
      }
    }
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if ((tid & 31) == 0) { red[0][tid >> 5] = se; red[1][tid >> 5] = sa; }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) { a += red[0][w]; b += red[1][w]; }
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
  }
}

__global__ void diag_check_kernel(const double* A, int lda, int n, double limit, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = A[(size_t)i * lda + i];
    if (!(d <= limit)) atomicExch(flag, 1);
  }
}

int grid_for(size_t work, int threads) {
  size_t g = (work + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

namespace {
// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014):
// the finalizer of the state x + (key + 1) * 0x9e3779b97f4a7c15.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// A_ij = A_ji uniform in [-1, 1) from the counter (seed, min(i,j), max(i,j)); A_ii = n.
__global__ void fill_spd_uniform_kernel(double* __restrict__ A, int lda, int n, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  double v;
  if (i == j) {
    v = (double)n;
  } else {
    const unsigned long long lo = (unsigned long long)min(i, j), hi = (unsigned long long)max(i, j);
    const unsigned long long r = splitmix64(seed ^ splitmix64(hi * 0x100000000ull + lo));
    v = 2.0 * ((double)(r >> 11) * 0x1.0p-53) - 1.0;
  }
  A[(size_t)j * lda + i] = v;
}

}  // namespace

cudaError_t launch_fill_spd_uniform(double* A, int lda, int n, unsigned long long seed, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 65535) return cudaErrorInvalidValue;
  fill_spd_uniform_kernel<<<dim3((n + 255) / 256, n), 256, 0, s>>>(A, lda, n, seed);
  return cudaGetLastError();
}

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

cudaError_t launch_fill_int(int* p, int v, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  (void)launch_pdl(fill_int_kernel, dim3((count + 255) / 256), dim3(256), 0, s, p, v, count);
  return cudaGetLastError();
}
cudaError_t launch_finalize_info(int* info, cudaStream_t s) {
  (void)launch_pdl(finalize_info_kernel, dim3(1), dim3(1), 0, s, info);
  return cudaGetLastError();
}
cudaError_t launch_copy_lower(double* dst, int ldd, const double* src, int lds, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  (void)launch_pdl(copy_lower_kernel, dim3(grid_for((size_t)n * n, 256)), dim3(256), 0, s, dst, ldd, src, lds, n);
  return cudaGetLastError();
}
cudaError_t launch_copy_matrix(double* dst, int ldd, const double* src, int lds, int m, int n, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  (void)launch_pdl(copy_matrix_kernel, dim3(grid_for((size_t)m * n, 256)), dim3(256), 0, s, dst, ldd, src, lds, m, n);
  return cudaGetLastError();
}
cudaError_t launch_axpy_matrix(double* X, int ldx, const double* D, int ldd, int n, int nrhs, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  (void)launch_pdl(axpy_matrix_kernel, dim3(grid_for((size_t)n * nrhs, 256)), dim3(256), 0, s, X, ldx, D, ldd, n, nrhs);
  return cudaGetLastError();
}
cudaError_t launch_residual(const double* A, int lda, const double* X, int ldx, const double* B, int ldb,
                            double* R, int ldr, int n, int nrhs, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  cudaError_t e = launch_copy_matrix(R, ldr, B, ldb, n, nrhs, s);
  if (e != cudaSuccess) return e;
  const long long nt = (n + RT - 1) / RT;
  const long long tiles = nt * (nt + 1) / 2;
  for (int c0 = 0; c0 < nrhs; c0 += RNRHS) {
    int nc = nrhs - c0 < RNRHS ? nrhs - c0 : RNRHS;
    (void)launch_pdl(residual_tile_kernel, dim3((unsigned)tiles), dim3(256), 0, s, A, lda, X + (size_t)c0 * ldx, ldx, R + (size_t)c0 * ldr,
                                                         ldr, n, nc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t launch_col_norms2(const double* R, int ldr, const double* B, int ldb, int n, int nrhs, double* out,
                              cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 2 * nrhs, s);
  if (e != cudaSuccess) return e;
  dim3 grid(grid_for((size_t)n, 256) > 64 ? 64 : grid_for((size_t)n, 256), nrhs);
  (void)launch_pdl(col_norms2_kernel, dim3(grid), dim3(256), 0, s, R, ldr, B, ldb, n, nrhs, out);
  return cudaGetLastError();
}
cudaError_t launch_backward_error(const double* A, int lda, const double* L, int ldl, int n, double* out,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long nt = (n + 63) / 64;
  backward_error_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, lda, L, ldl, n, out);
  return cudaGetLastError();
}
// 32 x 32 tiles through shared memory: coalesced reads of the column-major block and
// coalesced writes of the row-major copy
__global__ void __launch_bounds__(256) cast_f16_rows_kernel(const double* __restrict__ X, int ldx, int m, int k,
                                                            __half* __restrict__ S, int lds, unsigned* err) {
  pdl_wait();
  pdl_trigger();
  __shared__ double t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;     // 8 rows of threads
  for (int c = ty; c < 32; c += 8) {
    const int gr = r0 + tx, gc = c0 + c;
    t[c][tx] = (gr < m && gc < k) ? X[(size_t)gc * ldx + gr] : 0.0;
  }
  __syncthreads();
  bool over = false;
  for (int r = ty; r < 32; r += 8) {
    const int gr = r0 + r, gc = c0 + tx;
    if (gr < m && gc < k) {
      const double v = t[tx][r];
      over |= fabs(v) > (double)kF16Max;
      S[(size_t)gr * lds + gc] = __double2half(v);
    }
  }
  if (__any_sync(0xffffffffu, over) && tx == 0) atomicOr(err, DEV_ERR_RANGE16);
}

__global__ void __launch_bounds__(256) cast_f32_kernel(const double* __restrict__ X, int ldx, int m, int k,
                                                       float* __restrict__ S, int ld32) {
  pdl_wait();
  pdl_trigger();
  const long long total = (long long)m * k;
  for (long long e = blockIdx.x * 256ll + threadIdx.x; e < total; e += (long long)gridDim.x * 256) {
    const int r = (int)(e % m), c = (int)(e / m);
    S[(size_t)c * ld32 + r] = (float)X[(size_t)c * ldx + r];
  }
}

cudaError_t launch_cast_f16_rows(const double* X, int ldx, int m, int k, __half* S16, int lds, unsigned* err,
                                 cudaStream_t s) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  const dim3 grid((m + 31) / 32, (k + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  (void)launch_pdl(cast_f16_rows_kernel, grid, dim3(256), 0, s, X, ldx, m, k, S16, lds, err);
  return cudaGetLastError();
}

cudaError_t launch_cast_f32(const double* X, int ldx, int m, int k, float* S32, int ld32, cudaStream_t s) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  const long long total = (long long)m * k;
  const int grid = (int)std::min<long long>((total + 255) / 256, 8LL * device_sm_count());
  (void)launch_pdl(cast_f32_kernel, dim3(grid), dim3(256), 0, s, X, ldx, m, k, S32, ld32);
  return cudaGetLastError();
}

// ---- TF32 split of FP32 operands (error-corrected FP32 GEMM on tensor cores) ----
// round to nearest even at 10 explicit mantissa bits, on the binary32 bit pattern
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7F800000u) != 0x7F800000u) {
    b += 0x0FFFu + ((b >> 13) & 1u);
    b &= 0xFFFFE000u;
  }
  return __uint_as_float(b);
}
// A: column-major FP64 block (rows r0 .. r0 + m, columns c0 .. c0 + nc); writes the row-major
// hi = tf32(x) and lo = tf32(x - hi) of x = fp32(a) at [(r0 + i) ldh + c0 + j], through a
// 32 x 32 shared-memory transpose (reads and writes both coalesced)
__global__ void split_tf32_kernel(const double* __restrict__ A, int lda, int r0, int m, int c0, int nc,
                                  float* __restrict__ H, float* __restrict__ Lo, int ldh) {
  pdl_wait();
  pdl_trigger();
  __shared__ float t[32][33];
  const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int i = i0 + threadIdx.x, j = j0 + jj;
    t[jj][threadIdx.x] = (i < m && j < nc) ? (float)A[(size_t)(c0 + j) * lda + r0 + i] : 0.f;
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + threadIdx.x;
    if (i < m && j < nc) {
      const float x = t[threadIdx.x][ii];
      const float hi = round_tf32(x);
      const size_t o = (size_t)(r0 + i) * ldh + c0 + j;
      H[o] = hi;
      Lo[o] = round_tf32(x - hi);                 // x - hi is exact in binary32
    }
  }
}

cudaError_t launch_split_tf32(const double* A, int lda, int r0, int m, int c0, int nc, float* H, float* Lo, int ldh,
                              cudaStream_t s) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  const dim3 grid((nc + 31) / 32, (m + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  (void)launch_pdl(split_tf32_kernel, grid, dim3(32, 8), 0, s, A, lda, r0, m, c0, nc, H, Lo, ldh);
  return cudaGetLastError();
}

// ---- dynamic quantization: two-sided power-of-two diagonal scaling ----
// e[i] = floor(ex / 2) for a_ii = m 2^ex, m in [0.5, 1) (0 when a_ii <= 0 or not finite)
__global__ void diag_exponents_kernel(const double* __restrict__ A, int lda, int n, int* __restrict__ e) {
  pdl_wait();
  pdl_trigger();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = A[(size_t)i * lda + i];
    int ex = 0;
    if (a > 0.0 && isfinite(a)) frexp(a, &ex);
    e[i] = (a > 0.0 && isfinite(a)) ? (ex >= 0 ? ex / 2 : -((1 - ex) / 2)) : 0;   // floor(ex / 2)
  }
}
// lower triangle: a_ij <- a_ij 2^(sign (e_i + e_j)) with sign = -1 (scale) or the rows only,
// a_ij <- a_ij 2^(e_i) (unscale the factor); exact in FP64 away from the subnormal range
__global__ void diag_scale_kernel(double* __restrict__ A, int lda, int n, const int* __restrict__ e, int unscale) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.y;
  for (int j0 = j; j0 < n; j0 += gridDim.y) {
    const int ej = e[j0];
    for (int i = j0 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double* p = A + (size_t)j0 * lda + i;
      *p = unscale ? ldexp(*p, e[i]) : ldexp(*p, -(e[i] + ej));
    }
  }
}

cudaError_t launch_diag_scale(double* A, int lda, int n, int* e, bool unscale, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  if (!unscale) {
    (void)launch_pdl(diag_exponents_kernel, dim3((n + 255) / 256), dim3(256), 0, s, A, lda, n, e);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const dim3 grid((n + 255) / 256 < 8 ? (n + 255) / 256 : 8, n < 4096 ? n : 4096);
  (void)launch_pdl(diag_scale_kernel, grid, dim3(256), 0, s, A, lda, n, (const int*)e, unscale ? 1 : 0);
  return cudaGetLastError();
}

// ---- Krylov helpers of the GMRES refinement (FP64) ----
// out[j] += sum_i V[j ldv + i] w[i] for j < nv: blocks of 1024 rows per column, reduced in
// shared memory, one FP64 atomic per block and column (out is zeroed by the caller)
__global__ void __launch_bounds__(256) multi_dot_kernel(const double* __restrict__ V, int ldv, int nv,
                                                         const double* __restrict__ w, int n, double* out) {
  __shared__ double red[8];
  const int j = blockIdx.y;
  const int i0 = blockIdx.x * 1024;
  double acc = 0.0;
  for (int i = i0 + threadIdx.x; i < min(n, i0 + 1024); i += 256) acc = fma(V[(size_t)j * ldv + i], w[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    atomicAdd(out + j, t);
  }
}
// w[i] -= sum_{j<nv} V[j ldv + i] c[j] (c on the device)
__global__ void gemv_sub_kernel(double* __restrict__ w, const double* __restrict__ V, int ldv, int nv,
                                const double* __restrict__ c, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < nv; ++j) acc = fma(-V[(size_t)j * ldv + i], c[j], acc);
    w[i] = acc;
  }
}
// y = a x (+ y when accumulate)
__global__ void scale_kernel(double* __restrict__ y, const double* __restrict__ x, double a, int n, int accumulate) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = accumulate ? fma(a, x[i], y[i]) : a * x[i];
}

cudaError_t launch_multi_dot(const double* V, int ldv, int nv, const double* w, int n, double* out, cudaStream_t s) {
  if (n <= 0 || nv <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nv, s);
  if (e != cudaSuccess) return e;
  multi_dot_kernel<<<dim3((n + 1023) / 1024, nv), 256, 0, s>>>(V, ldv, nv, w, n, out);
  return cudaGetLastError();
}
cudaError_t launch_gemv_sub(double* w, const double* V, int ldv, int nv, const double* c, int n, cudaStream_t s) {
  if (n <= 0 || nv <= 0) return cudaSuccess;
  gemv_sub_kernel<<<std::min((n + 255) / 256, 4 * device_sm_count()), 256, 0, s>>>(w, V, ldv, nv, c, n);
  return cudaGetLastError();
}
cudaError_t launch_scale(double* y, const double* x, double a, int n, bool accumulate, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  scale_kernel<<<std::min((n + 255) / 256, 4 * device_sm_count()), 256, 0, s>>>(y, x, a, n, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_diag_check(const double* A, int lda, int n, double limit, int* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  diag_check_kernel<<<grid_for((size_t)n, 256), 256, 0, s>>>(A, lda, n, limit, flag);
  return cudaGetLastError();
}

}  // namespace hrp

// ---------------------------------------------------------------------------------------
// E4M3 quantization of finished L tiles (FP8 levels of the tree).
//
// One CTA per 128 x 128 tile of the global grid: amax over the tile, scale
// s = 2^ceil(log2(amax / 448)) (exact power of two; 1 for an all-zero tile), each entry
// rounded to E4M3FN (round to nearest even, saturating; written here from the OCP format
// definition: 4 exponent bits with bias 7, 3 mantissa bits, subnormals k * 2^-9, largest
// finite 448), then stored as the FP16 number 2^G * s * e4m3(x / s).  That number is
// exact in FP16 whenever 2^G * amax <= 65504 and 2^(G-24) <= s * 2^-9 (checked; a tile
// outside that window sets DEV_ERR_RANGE), so a kind::f16 tensor-core product of two such
// operands, scaled by 2^-2G, equals the block-scaled E4M3 product.
// ---------------------------------------------------------------------------------------
namespace hrp {
namespace {

// FP16 bit pattern of 2^(sig + G) e4m3(x 2^-sig), e4m3 = round to nearest even onto the E4M3
// grid (3 mantissa bits, normal exponents -6 .. 8, subnormal spacing 2^-9, saturating at
// 448), by 32-bit integer operations on the bits of x (this GPU runs FP64 arithmetic and FP64
// conversions on its slow FP64 pipe).  |x 2^-sig| <= 448 and the product's representability
// in FP16 are guaranteed by the caller's choice of sig and range check.
__device__ __forceinline__ unsigned short quant_e4m3_h(double x, int sig, int G) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = (hi >> 31) << 15;
  const int E = (int)((hi >> 20) & 0x7ff);
  if (E == 0) return (unsigned short)sign;                   // zero or FP64 subnormal: rounds to 0
  if (E == 0x7ff) {                                          // NaN stays NaN; infinity saturates
    if ((hi & 0xfffffu) | lo) return (unsigned short)(sign | 0x7e00u);
    const int ef = 5 + sig + G + 15;                         // 448 = 1.75 * 2^8 -> 14 * 2^5
    return (unsigned short)(sign | ((unsigned)(ef + 3) << 10) | (3u << 8));
  }
  const unsigned S = (hi & 0xfffffu) | 0x100000u;            // top 21 bits of the 53-bit significand
  const int ey = E - 1023 - sig;                             // binade of y = x 2^-sig
  // y / spacing = significand >> sh, spacing 2^(ey-3) (normal) or 2^-9 (subnormal); sh in [49, 54]
  int qe = ey >= -6 ? ey - 3 : -9;
  const int sh = 52 - (ey - qe);
  if (sh > 54) return (unsigned short)sign;                  // below half the smallest E4M3 step
  const int s32 = sh - 32;                                   // 17 .. 22: shift within S
  unsigned r = S >> s32;
  const unsigned halfbit = (S >> (s32 - 1)) & 1u;
  const unsigned sticky = (S & ((1u << (s32 - 1)) - 1u)) | lo;
  r += halfbit & ((sticky != 0u) | (r & 1u));
  if (r == 0) return (unsigned short)sign;
  if (ey > 8 || (ey == 8 && r > 14u)) {                      // saturate at 448 = 14 * 2^5
    r = 14u;
    qe = 5;
  }
  // value = r 2^e2 with 1 <= r <= 16, exact in FP16 (normal or subnormal)
  const int e2 = qe + sig + G;
  const int pw = 31 - __clz((int)r);                         // r = 1.f 2^pw
  const int be = pw + e2 + 15;                               // FP16 biased exponent
  unsigned h;
  if (be >= 1) h = ((unsigned)be << 10) | ((r - (1u << pw)) << (10 - pw));
  else h = r << (e2 + 24);                                   // subnormal: units of 2^-24
  return (unsigned short)(h | sign);
}

// E4M3FN code (sign, 4 exponent bits with bias 7, 3 mantissa bits; 0x7F = NaN) of
// e4m3(x 2^-sig), rounded exactly as quant_e4m3_h rounds (nearest even, saturating at 448).
__device__ __forceinline__ unsigned char quant_e4m3_code(double x, int sig) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = (hi >> 31) << 7;
  const int E = (int)((hi >> 20) & 0x7ff);
  if (E == 0) return (unsigned char)sign;
  if (E == 0x7ff) {
    if ((hi & 0xfffffu) | lo) return (unsigned char)(sign | 0x7fu);
    return (unsigned char)(sign | 0x7eu);                    // infinity saturates to 448
  }
  const unsigned S = (hi & 0xfffffu) | 0x100000u;
  const int ey = E - 1023 - sig;
  int qe = ey >= -6 ? ey - 3 : -9;
  const int sh = 52 - (ey - qe);
  if (sh > 54) return (unsigned char)sign;
  const int s32 = sh - 32;
  unsigned r = S >> s32;
  const unsigned halfbit = (S >> (s32 - 1)) & 1u;
  const unsigned sticky = (S & ((1u << (s32 - 1)) - 1u)) | lo;
  r += halfbit & ((sticky != 0u) | (r & 1u));
  if (r == 0) return (unsigned char)sign;
  if (ey > 8 || (ey == 8 && r > 14u)) {
    r = 14u;
    qe = 5;
  }
  // value = r 2^qe, 1 <= r <= 16: subnormal code r (qe = -9, r < 8), else 1.m 2^(pw + qe)
  if (qe == -9 && r < 8u) return (unsigned char)(sign | r);
  const int pw = 31 - __clz((int)r);
  const unsigned mant = (r - (1u << pw)) << (3 - pw);           // pw <= 3, or r = 16 (mant 0)
  return (unsigned char)(sign | ((unsigned)(pw + qe + 7) << 3) | (pw == 4 ? 0u : mant));
}

constexpr int kQT = 128;     // tile edge (rows and columns)
constexpr int kQLD = 129;    // row stride (doubles) of the staged tile
constexpr int kQThreads = 1024;

// One 128 x 128 tile (rows R0 .. R0 + rows - 1, columns c0 .. c0 + 127) by one CTA: the tile
// is read once from the master (coalesced along rows, all 16 loads per thread in flight) into
// shared memory, its amax gives the power-of-two scale s = 2^sig = 2^ceil(log2(amax / 448)),
// and the FP16 shadow is written row by row (coalesced along columns).
__device__ __forceinline__ void quant_tile(const double* __restrict__ A, int ld, int R0, int rows, int c0,
                                           __half* __restrict__ S8, unsigned char* __restrict__ B8, int lds,
                                           int* __restrict__ tile_exp, int ntile_ld, int G,
                                           unsigned* __restrict__ err, double* tileq) {
  __shared__ unsigned long long red[kQThreads / 32];
  __shared__ int s_sig;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kPer = kQT * kQT / kQThreads;
  double v[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int idx = tid + u * kQThreads;
    const int i = idx & (kQT - 1), j = idx >> 7;
    v[u] = i < rows ? A[(size_t)(c0 + j) * ld + R0 + i] : 0.0;
  }
  // amax over finite entries, as the largest |x| bit pattern (non-negative doubles order like
  // their bits)
  unsigned long long abits = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int idx = tid + u * kQThreads;
    tileq[(idx & (kQT - 1)) * kQLD + (idx >> 7)] = v[u];
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[u]) & 0x7fffffffffffffffull;
    if (b < 0x7ff0000000000000ull && b > abits) abits = b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, abits, o);
    if (w > abits) abits = w;
  }
  if (lane == 0) red[warp] = abits;
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0;
    for (int w = 0; w < kQThreads / 32; ++w) a = red[w] > a ? red[w] : a;
    const double amax = __longlong_as_double((long long)a);
    int sig = 0;                                   // s = 2^sig
    if (amax > 0.0) {
      int ex;
      const double f = frexp(amax / 448.0, &ex);   // amax / 448 = f * 2^ex
      sig = (f == 0.5) ? ex - 1 : ex;              // ceil(log2(amax / 448))
    }
    tile_exp[(size_t)(R0 / kQT) * ntile_ld + c0 / kQT] = sig;
    // FP16 storage: 2^G amax and the smallest E4M3 step 2^(sig - 9 + G) inside FP16's range;
    // E4M3 codes: the scale 2^sig a UE8M0 code (127 + sig in 0 .. 254)
    const bool fits16 = !(amax > 0.0) || (ldexp(amax, G) <= 65504.0 && sig - 9 + G >= -24);
    const bool fits8 = sig >= -127 && sig <= 127;
    if ((S8 != nullptr && !fits16) || (B8 != nullptr && !fits8)) atomicOr(err, DEV_ERR_RANGE);
    s_sig = sig;
  }
  __syncthreads();
  const int sig = s_sig;
  if (S8 != nullptr) {
#pragma unroll 4
    for (int idx = tid; idx < kQT * kQT; idx += kQThreads) {
      const int j = idx & (kQT - 1), i = idx >> 7;   // consecutive threads: consecutive columns
      if (i < rows) S8[(size_t)(R0 + i) * lds + c0 + j] = __ushort_as_half(quant_e4m3_h(tileq[i * kQLD + j], sig, G));
    }
  }
  if (B8 != nullptr) {
    // four codes per thread, one 32-bit store: 128 rows x 32 words
    for (int idx = tid; idx < kQT * (kQT / 4); idx += kQThreads) {
      const int w = idx & (kQT / 4 - 1), i = idx >> 5;
      if (i < rows) {
        const double* q = tileq + i * kQLD + 4 * w;
        const unsigned word = (unsigned)quant_e4m3_code(q[0], sig) | ((unsigned)quant_e4m3_code(q[1], sig) << 8) |
                              ((unsigned)quant_e4m3_code(q[2], sig) << 16) |
                              ((unsigned)quant_e4m3_code(q[3], sig) << 24);
        *reinterpret_cast<unsigned*>(B8 + (size_t)(R0 + i) * lds + c0 + 4 * w) = word;
      }
    }
  }
}

// The panel rows r0 .. r0 + m - 1, columns c0 .. c0 + 127: one CTA per row tile.
__global__ void __launch_bounds__(kQThreads)
quant_e4m3_kernel(const double* __restrict__ A, int ld, int r0, int m, int c0, __half* __restrict__ S8,
                  unsigned char* __restrict__ B8, int lds, int* __restrict__ tile_exp, int ntile_ld, int G,
                  unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double tileq[];                  // [128][kQLD]
  const int R0 = r0 + blockIdx.x * kQT;
  quant_tile(A, ld, R0, min(kQT, r0 + m - R0), c0, S8, B8, lds, tile_exp, ntile_ld, G, err, tileq);
}

// Every tile strictly below the diagonal tiles of the block A[off:off+nb, off:off+nb]: CTA e
// takes tile (I, J), e = I (I - 1) / 2 + J, 0 <= J < I.
__global__ void __launch_bounds__(kQThreads)
quant_e4m3_lower_kernel(const double* __restrict__ A, int ld, int off, int nb, __half* __restrict__ S8,
                        unsigned char* __restrict__ B8, int lds, int* __restrict__ tile_exp, int ntile_ld, int G,
                        unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double tileq[];                  // [128][kQLD]
  const int e = blockIdx.x;
  int I = (int)((1.0f + sqrtf(8.0f * (float)e + 1.0f)) * 0.5f);
  while (I * (I - 1) / 2 > e) --I;                   // guards against the float rounding
  while ((I + 1) * I / 2 <= e) ++I;
  const int J = e - I * (I - 1) / 2;
  const int R0 = off + I * kQT;
  quant_tile(A, ld, R0, min(kQT, off + nb - R0), off + J * kQT, S8, B8, lds, tile_exp, ntile_ld, G, err, tileq);
}

}  // namespace

cudaError_t launch_quant_e4m3(const double* A, int ld, int r0, int m, int c0, int nc, __half* S8, unsigned char* B8,
                              int lds, int* tile_exp, int ntile_ld, int G, unsigned* err, cudaStream_t s) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  if ((r0 % 128) || (c0 % 128) || nc != 128) return cudaErrorInvalidValue;
  const size_t smem = (size_t)128 * kQLD * sizeof(double);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e = cudaFuncSetAttribute(quant_e4m3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  (void)launch_pdl(quant_e4m3_kernel, dim3((m + 127) / 128), dim3(kQThreads), smem, s, A, ld, r0, m, c0, S8, B8, lds,
                   tile_exp, ntile_ld, G, err);
  return cudaGetLastError();
}

cudaError_t launch_quant_e4m3_lower(const double* A, int ld, int off, int nb, __half* S8, unsigned char* B8, int lds,
                                    int* tile_exp, int ntile_ld, int G, unsigned* err, cudaStream_t s) {
  const int nt = (nb + kQT - 1) / kQT;
  if (nt < 2) return cudaSuccess;
  if (off % kQT) return cudaErrorInvalidValue;
  const size_t smem = (size_t)128 * kQLD * sizeof(double);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  if (!(attr_mask & attr_bit)) {
    cudaError_t e =
        cudaFuncSetAttribute(quant_e4m3_lower_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_mask |= attr_bit;
  }
  (void)launch_pdl(quant_e4m3_lower_kernel, dim3(nt * (nt - 1) / 2), dim3(kQThreads), smem, s, A, ld, off, nb, S8, B8,
                   lds, tile_exp, ntile_ld, G, err);
  return cudaGetLastError();
}

}  // namespace hrp
