// Learned precision policy: matrix features, Lanczos, and the MLP 12 -> 64 -> 64 -> 8
// (forward, softmax cross-entropy gradient, Adam step), all in FP32 except the FP64
// matrix passes.  Not in the paper: an extension that predicts the precision tree.
//
// Features (same order and definitions as the oracle): log2 n; min / mean / fraction > 1
// of the row dominance ratios r_i = a_ii / sum_{j!=i} |a_ij|; log10 ||A||_F; log10 of
// diagonal max, min and their ratio; log10 of the extreme Ritz values of k Lanczos steps
// from the start vector v_i ~ 1 + (i mod 7)/7, their ratio, and log10(n lambda_min/||A||_F).
#include <cfloat>
#include <cmath>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int FT = 64;

__device__ __forceinline__ void tri_index64(long long t, int& I, int& J) {
  long long i = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = (int)i;
  J = (int)(t - i * (i + 1) / 2);
}

// rowsum[i] += sum_{j != i} |a_ij| (lower tiles, both triangles by symmetry);
// stats[0] += ||A||_F^2 contribution
__global__ void __launch_bounds__(256)
rowsum_kernel(const double* __restrict__ A, int lda, int n, double* __restrict__ rowsum, double* __restrict__ stats) {
  __shared__ double As[FT][FT + 1];
  __shared__ double red[8];
  int I, J;
  tri_index64(blockIdx.x, I, J);
  const int I0 = I * FT, J0 = J * FT, tid = threadIdx.x;
  double fro = 0.0;
  for (int idx = tid; idx < FT * FT; idx += 256) {
    const int i = idx % FT, j = idx / FT, gi = I0 + i, gj = J0 + j;
    double v = (gi < n && gj < n && gi >= gj) ? A[(size_t)gj * lda + gi] : 0.0;
    As[i][j] = (gi == gj) ? 0.0 : fabs(v);
    fro += (gi == gj ? 1.0 : 2.0) * v * v;
  }
  __syncthreads();
  if (tid < FT) {
    double r = 0.0, c = 0.0;
    for (int j = 0; j < FT; ++j) r += As[tid][j];
    // row I0+tid: its entries left of the diagonal; row J0+tid: by symmetry the entries of
    // column J0+tid below (inside a diagonal tile, the entries right of its diagonal)
    if (I0 + tid < n) atomicAdd(rowsum + I0 + tid, r);
    for (int i = 0; i < FT; ++i) c += As[i][tid];
    if (J0 + tid < n) atomicAdd(rowsum + J0 + tid, c);
  }
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(stats, s);
  }
}

__device__ __forceinline__ void atomic_min_d(double* p, double v) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(p);
  unsigned long long old = *a, assumed;
  do {
    assumed = old;
    if (__longlong_as_double(assumed) <= v) return;
    old = atomicCAS(a, assumed, __double_as_longlong(v));
  } while (old != assumed);
}
__device__ __forceinline__ void atomic_max_d(double* p, double v) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(p);
  unsigned long long old = *a, assumed;
  do {
    assumed = old;
    if (__longlong_as_double(assumed) >= v) return;
    old = atomicCAS(a, assumed, __double_as_longlong(v));
  } while (old != assumed);
}

// stats: [1] min r, [2] sum min(r, 1e6), [3] count r > 1, [4] diag min, [5] max |diag|
__global__ void dominance_kernel(const double* __restrict__ A, int lda, int n, const double* __restrict__ rowsum,
                                 double* __restrict__ stats) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = A[(size_t)i * lda + i];
    const double off = rowsum[i];
    const double r = off > 0.0 ? d / off : 1e30;
    atomic_min_d(stats + 1, r);
    atomicAdd(stats + 2, fmin(r, 1e6));
    if (r > 1.0) atomicAdd(stats + 3, 1.0);
    atomic_min_d(stats + 4, d);
    atomic_max_d(stats + 5, fabs(d));
  }
}

// R -= A v over lower tiles (A read once in FP64, products and tile sums in FP32: the
// features need the extreme Ritz values only to a few digits)
__global__ void __launch_bounds__(256)
symv32_tile_kernel(const double* __restrict__ A, int lda, const double* __restrict__ v, double* __restrict__ R, int n) {
  __shared__ float As[FT][FT + 1];
  __shared__ float vI[FT], vJ[FT];
  int I, J;
  tri_index64(blockIdx.x, I, J);
  const int I0 = I * FT, J0 = J * FT, tid = threadIdx.x;
  for (int idx = tid; idx < FT * FT; idx += 256) {
    const int i = idx % FT, j = idx / FT, gi = I0 + i, gj = J0 + j;
    As[i][j] = (gi < n && gj < n && gi >= gj) ? (float)A[(size_t)gj * lda + gi] : 0.f;
  }
  if (tid < FT) {
    vI[tid] = (I0 + tid < n) ? (float)v[I0 + tid] : 0.f;
    vJ[tid] = (J0 + tid < n) ? (float)v[J0 + tid] : 0.f;
  }
  __syncthreads();
  if (tid < FT) {
    float y = 0.f;
    if (I == J) {
      for (int j = 0; j < FT; ++j) y = fmaf(j <= tid ? As[tid][j] : As[j][tid], vJ[j], y);
    } else {
      for (int j = 0; j < FT; ++j) y = fmaf(As[tid][j], vJ[j], y);
    }
    if (I0 + tid < n) atomicAdd(R + I0 + tid, -(double)y);
  } else if (tid < 2 * FT && I != J) {
    const int c = tid - FT;
    float z = 0.f;
    for (int r = 0; r < FT; ++r) z = fmaf(As[r][c], vI[r], z);
    if (J0 + c < n) atomicAdd(R + J0 + c, -(double)z);
  }
}

__global__ void lanczos_start_kernel(double* v, int n, double inv_norm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = (1.0 + (double)(i % 7) / 7.0) * inv_norm;
}
// w = -R (R = 0 - A v from the residual kernel); out[0] += w . v
__global__ void lanczos_dot_kernel(const double* R, const double* v, int n, double* out) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += -R[i] * v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}
// w = -R - alpha v - beta v_prev (stored into R); out[0] += ||w||^2; beta read from the device
__global__ void lanczos_axpy_kernel(double* R, const double* v, const double* vp, int n, const double* alpha,
                                    const double* beta_p, double* out) {
  const double a = *alpha;
  const double beta = beta_p ? *beta_p : 0.0;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = -R[i] - a * v[i] - beta * vp[i];
    R[i] = w;
    s += w * w;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}
// beta = ||w|| (from the accumulated square); v_prev = v; v = w / beta (0 if beta is 0)
__global__ void lanczos_next_kernel(const double* w, double* vp, double* v, int n, const double* norm2,
                                    double* beta_out) {
  const double beta = sqrt(*norm2);
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *beta_out = beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    vp[i] = v[i];
    v[i] = w[i] * inv;
  }
}

// ---- MLP ----
constexpr int NI = 12, NH = 64, NO = 8;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;

// one CTA of 64 threads per sample: h1, h2, z in shared memory
__device__ void mlp_forward_one(const float* __restrict__ p, const float* __restrict__ x, float* h1, float* h2,
                                float* z) {
  const int t = threadIdx.x;
  float s = p[OFF_B1 + t];
  for (int k = 0; k < NI; ++k) s = fmaf(p[OFF_W1 + t * NI + k], x[k], s);
  h1[t] = fmaxf(s, 0.f);
  __syncthreads();
  s = p[OFF_B2 + t];
  for (int k = 0; k < NH; ++k) s = fmaf(p[OFF_W2 + t * NH + k], h1[k], s);
  h2[t] = fmaxf(s, 0.f);
  __syncthreads();
  if (t < NO) {
    s = p[OFF_B3 + t];
    for (int k = 0; k < NH; ++k) s = fmaf(p[OFF_W3 + t * NH + k], h2[k], s);
    z[t] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(64) mlp_forward_kernel(const float* __restrict__ p, const float* __restrict__ X,
                                                         float* __restrict__ Z) {
  __shared__ float h1[NH], h2[NH], z[NO];
  const int b = blockIdx.x;
  mlp_forward_one(p, X + (size_t)b * NI, h1, h2, z);
  if (threadIdx.x < NO) Z[(size_t)b * NO + threadIdx.x] = z[threadIdx.x];
}

// gradient of the mean softmax cross-entropy, accumulated with atomics over the batch
__global__ void __launch_bounds__(64) mlp_grad_kernel(const float* __restrict__ p, const float* __restrict__ X,
                                                      const int* __restrict__ y, int batch, float* __restrict__ g,
                                                      float* __restrict__ loss) {
  __shared__ float h1[NH], h2[NH], z[NO], dz[NO], dh2[NH], dh1[NH];
  const int b = blockIdx.x, t = threadIdx.x;
  const float* x = X + (size_t)b * NI;
  mlp_forward_one(p, x, h1, h2, z);
  const float inv_b = 1.f / (float)batch;
  if (t == 0) {
    float m = z[0];
    for (int o = 1; o < NO; ++o) m = fmaxf(m, z[o]);
    float se = 0.f;
    for (int o = 0; o < NO; ++o) se += expf(z[o] - m);
    const int lab = y[b];
    for (int o = 0; o < NO; ++o) dz[o] = (expf(z[o] - m) / se - (o == lab ? 1.f : 0.f)) * inv_b;
    atomicAdd(loss, (logf(se) + m - z[lab]) * inv_b);
  }
  __syncthreads();
  // layer 3
  for (int o = 0; o < NO; ++o) atomicAdd(g + OFF_W3 + o * NH + t, dz[o] * h2[t]);
  if (t < NO) atomicAdd(g + OFF_B3 + t, dz[t]);
  float s = 0.f;
  for (int o = 0; o < NO; ++o) s = fmaf(p[OFF_W3 + o * NH + t], dz[o], s);
  dh2[t] = h2[t] > 0.f ? s : 0.f;
  __syncthreads();
  // layer 2
  for (int k = 0; k < NH; ++k) atomicAdd(g + OFF_W2 + t * NH + k, dh2[t] * h1[k]);
  atomicAdd(g + OFF_B2 + t, dh2[t]);
  s = 0.f;
  for (int o = 0; o < NH; ++o) s = fmaf(p[OFF_W2 + o * NH + t], dh2[o], s);
  dh1[t] = h1[t] > 0.f ? s : 0.f;
  __syncthreads();
  // layer 1
  for (int k = 0; k < NI; ++k) atomicAdd(g + OFF_W1 + t * NI + k, dh1[t] * x[k]);
  atomicAdd(g + OFF_B1 + t, dh1[t]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int count, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

int policy_nparam() { return NPARAM; }

cudaError_t launch_rowsum(const double* A, int lda, int n, double* rowsum, double* stats, cudaStream_t s) {
  const long long nt = (n + FT - 1) / FT;
  rowsum_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, lda, n, rowsum, stats);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dominance_kernel<<<64, 256, 0, s>>>(A, lda, n, rowsum, stats);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_start(double* v, int n, cudaStream_t s) {
  double ss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double t = 1.0 + (double)(i % 7) / 7.0;
    ss += t * t;
  }
  lanczos_start_kernel<<<64, 256, 0, s>>>(v, n, 1.0 / sqrt(ss));
  return cudaGetLastError();
}
cudaError_t launch_symv32(const double* A, int lda, const double* v, double* R, int n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(R, 0, sizeof(double) * n, s);
  if (e != cudaSuccess) return e;
  const long long nt = (n + FT - 1) / FT;
  symv32_tile_kernel<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, lda, v, R, n);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_dot(const double* R, const double* v, int n, double* out, cudaStream_t s) {
  lanczos_dot_kernel<<<64, 256, 0, s>>>(R, v, n, out);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_axpy(double* R, const double* v, const double* vp, int n, const double* alpha,
                                const double* beta, double* out, cudaStream_t s) {
  lanczos_axpy_kernel<<<64, 256, 0, s>>>(R, v, vp, n, alpha, beta, out);
  return cudaGetLastError();
}
cudaError_t launch_lanczos_next(const double* w, double* vp, double* v, int n, const double* norm2, double* beta,
                                cudaStream_t s) {
  lanczos_next_kernel<<<64, 256, 0, s>>>(w, vp, v, n, norm2, beta);
  return cudaGetLastError();
}
cudaError_t launch_mlp_forward(const float* p, int batch, const float* X, float* Z, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  mlp_forward_kernel<<<batch, 64, 0, s>>>(p, X, Z);
  return cudaGetLastError();
}
cudaError_t launch_mlp_grad(const float* p, int batch, const float* X, const int* y, float* g, float* loss,
                            cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(g, 0, sizeof(float) * NPARAM, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess || batch <= 0) return e;
  mlp_grad_kernel<<<batch, 64, 0, s>>>(p, X, y, batch, g, loss);
  return cudaGetLastError();
}
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int t, float lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(p, g, m, v, NPARAM, lr, b1, b2, 1e-8f,
                                                   1.f - powf(b1, (float)t), 1.f - powf(b2, (float)t));
  return cudaGetLastError();
}

}  // namespace hrp
