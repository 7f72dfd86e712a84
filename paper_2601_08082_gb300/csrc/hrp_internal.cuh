// Internal declarations shared by the HRP CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/hrp.h"

namespace hrp {

// Error flags written by kernels into the handle's device status word.
enum : unsigned {
  DEV_ERR_TIMEOUT = 1u,     // a bounded wait expired
  DEV_ERR_BOUNDS = 2u,      // a checked index fell outside its buffer
  DEV_ERR_RANGE = 4u,       // an E4M3 tile fell outside the exact FP16 storage window
  DEV_ERR_RANGE16 = 8u,     // an FP16 operand exceeded 65504 (Sec. 3.4 would need alpha > 1)
};

// Largest finite FP16 value, R_max of the Sec. 3.4 scaling rule alpha = max(1, amax / R_max)
constexpr float kF16Max = 65504.0f;

// Bounded device waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitTimeoutNs = 2000ull * 1000ull * 1000ull;

// Rounding applied to GEMM operands read from the FP64 master.
enum class OpRound : int { F64 = 0, F32 = 1, F16 = 2 };

// Programmatic dependent launch.  The factorization is a long chain of dependent launches
// on one stream; a kernel launched by launch_pdl may be scheduled while the previous kernel
// of the stream still runs.  Every such kernel calls pdl_wait() before its first access to
// global memory (the wait returns once the previous grid has completed and its writes are
// visible; it returns at once for a kernel launched without the attribute), then
// pdl_trigger() to let the next kernel be scheduled in turn.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch settings the scheduler sets for the next launches of the calling host thread:
//   pdl: launch with programmatic stream serialization.  Cleared for the first kernel after
//        the stream waited on another stream's event, so that no kernel overlaps the
//        predecessor it may depend on across streams.
//   max_ctas: upper bound on the CTAs of a persistent kernel (0 = one per SM), so that work
//        on a side stream leaves SMs to the critical path.
struct LaunchCtx {
  bool pdl = true;
  int max_ctas = 0;
  bool leaf_df = false;   // FP64 leaves: 16 x 16 pivot chains in double-float (k_leaf_cluster.cu)
};
inline LaunchCtx& launch_ctx() {
  thread_local LaunchCtx c;
  return c;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = launch_ctx().pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------- leaf kernels (k_leaf.cu) ----------------
// Leaf POTRF of the n x n diagonal block at A (ld), n <= 128, computed in FP64
// (compute64 = true) or FP32; round16: round input and output to FP16 (F16 leaf).
// If W32 != nullptr also writes the FP32 inverse of the (FP32-rounded) factor,
// column-major n x n with leading dimension ldw.  info: device int, atomicMin of the
// 1-based global column (col0 + k + 1) of the first failing pivot (INT_MAX = none).
// err: device status word; an F16 leaf whose input or factor exceeds kF16Max sets
// DEV_ERR_RANGE16.
cudaError_t launch_potrf_leaf(double* A, int ld, int n, int col0, bool compute64, bool round16,
                              float* W32, int ldw, int* info, unsigned* err, cudaStream_t s);

// The same FP64 leaf POTRF (no FP16 rounding) on a cluster of 8 CTAs holding 16 x 16
// tiles in shared memory (k_leaf_cluster.cu); launch_potrf_leaf uses it for n > 32.
cudaError_t launch_potrf_leaf_cluster(double* A, int ld, int n, int col0, float* W32, int ldw, int* info,
                                      cudaStream_t s);

// Leaf TRSM B <- B L^{-T} with B = A[r0.., c0..] (m x nc) and L = A[c0.., c0..] (nc x nc),
// in FP64 by substitution.  shadow16 (row-major, lds) receives FP16(X) and shadow32
// (column-major, ld32, the master's indexing) FP32(X), each if non-null.  An entry of X
// beyond kF16Max written to shadow16 sets DEV_ERR_RANGE16 in err (the FP16 operand would
// need the Sec. 3.4 scale alpha > 1).
// Lm, ldl: the matrix holding L when it is not A (a standalone TRSM); nullptr = A.
cudaError_t launch_trsm_leaf64(double* A, int ld, int r0, int m, int c0, int nc,
                               __half* shadow16, int lds, float* shadow32, int ld32, const int* info, unsigned* err,
                               cudaStream_t s, const double* Lm = nullptr, int ldl = 0);
// Same in FP32 using the precomputed FP32 inverse W (nc x nc lower, ldw) of the block:
// X = fl32(B) * W^T, result stored in FP64.
// w_done: W was written by a kernel that completed before the previous launch on s started
// (the kernel may then read it before waiting for that launch)
cudaError_t launch_trsm_leaf32(double* A, int ld, int r0, int m, int c0, int nc,
                               const float* W, int ldw, __half* shadow16, int lds, float* shadow32, int ld32,
                               const int* info, unsigned* err, cudaStream_t s, bool w_done = false);
// FP32 substitution variant (no inverse), for blocks whose inverse is not available.
cudaError_t launch_trsm_leaf32_subst(double* A, int ld, int r0, int m, int c0, int nc,
                                     __half* shadow16, int lds, float* shadow32, int ld32, const int* info,
                                     unsigned* err, cudaStream_t s, const double* Lm = nullptr, int ldl = 0);

// ---------------- SIMT GEMM (k_gemm_simt.cu) ----------------
// C[m x n] -= X[m x k] * Y[n x k]^T, all FP64 column-major views of the master, with
// operands rounded per `rnd` and accumulated in FP64 (rnd == F64) or FP32.  lower: C is a
// diagonal block, only entries with row >= col (in C's coordinates) are updated.
cudaError_t launch_gemm_simt(double* C, int ldc, const double* X, int ldx, const double* Y, int ldy,
                             int m, int n, int k, OpRound rnd, bool lower, cudaStream_t s);
// FP32 level with operands read from the FP32 shadow of L (column-major views, no rounding
// on load): C -= X Y^T accumulated in FP32.
cudaError_t launch_gemm_simt_f32(double* C, int ldc, const float* X, int ldx, const float* Y, int ldy,
                                 int m, int n, int k, bool lower, cudaStream_t s);

// ---------------- tcgen05 FP16 GEMM (k_gemm_tc.cu) ----------------
// C[m x n] (FP64 master, column-major) -= scale * X Y^T with X = S[xr0.., k0..] (m x k) and
// Y = S[yr0.., k0..] (n x k) read from the row-major FP16 shadow S (lds), FP32 accumulation
// in TMEM.  Requires k0 % 8 == 0 and lds % 8 == 0.
bool tc_gemm_supported();
// occupancy: tiles per SM the tile-width rule aims for (the tree's tile_occupancy; 0 = 1).
cudaError_t launch_gemm_f16_tc(double* C, int ldc, const __half* S, int lds,
                               int xr0, int yr0, int k0, int m, int n, int k, bool lower,
                               double scale, unsigned* dev_err, cudaStream_t s, int occupancy = 0);

// ---------------- POTRS (k_potrs.cu) ----------------
constexpr int kPotrsBlock = 64;     // rows per block of the sweeps
constexpr int kPotrsMaxRhs = 16;    // right-hand sides per pair of sweeps
// device scratch of one solve of order n: the inverses of the 64 x 64 diagonal blocks
// (FP64), then two mailboxes (forward and backward sweep) of kPotrsMaxRhs columns each
constexpr size_t potrs_workspace_bytes(int n) {
  return (size_t)((n + kPotrsBlock - 1) / kPotrsBlock) * kPotrsBlock * (kPotrsBlock + 2 * kPotrsMaxRhs) * sizeof(double);
}
// B (n x nrhs) <- A^{-1} B with A = L L^T: forward then backward sweep, in FP64 (the products
// in double-float) or (fp32) in FP32 on FP32-rounded L and B.  ticket: device int scratch.
// work: device scratch of potrs_workspace_bytes(n), no initial contents needed (the solve
// empties its mailboxes itself).  A bounded wait that expires sets DEV_ERR_TIMEOUT in dev_err
// and leaves NaN in the unsolved rows of B.  Launches: one pre-pass plus potrs_sweeps(nrhs).
cudaError_t launch_potrs(const double* L, int ldl, double* B, int ldb, int n, int nrhs, bool fp32, void* work,
                         int* ticket, unsigned* dev_err, cudaStream_t s,
                         unsigned long long wait_limit_ns = kWaitTimeoutNs);
// One thread empties the mailbox entry *entry (device) and waits on it through the sweeps'
// bounded wait; nothing fills it, so after wait_limit_ns it sets DEV_ERR_TIMEOUT and writes
// the time it waited (ns) to *waited_ns (device).
cudaError_t launch_wait_probe(double* entry, unsigned long long wait_limit_ns, unsigned* dev_err,
                              unsigned long long* waited_ns, cudaStream_t s);
int potrs_sweeps(int nrhs);

// ---------------- utilities (k_util.cu) ----------------
// SM count of the current device, queried once per device
int device_sm_count();
// Function attributes (the opt-in shared memory size) belong to the current device.  A launch
// site keeps a mask of the devices it has configured; dev_bit() is the current device's bit
// (0 for devices >= 64, which are then configured on every call).
inline unsigned long long dev_bit() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0ull;
  return 1ull << d;
}
cudaError_t launch_fill_int(int* p, int v, int count, cudaStream_t s);
// seeded SPD test matrix: off-diagonal entries uniform in [-1, 1) (symmetric), n on the
// diagonal (strictly diagonally dominant); n <= 65535
cudaError_t launch_fill_spd_uniform(double* A, int lda, int n, unsigned long long seed, cudaStream_t s);
cudaError_t launch_finalize_info(int* info, cudaStream_t s);
cudaError_t launch_copy_lower(double* dst, int ldd, const double* src, int lds, int n, cudaStream_t s);
cudaError_t launch_copy_matrix(double* dst, int ldd, const double* src, int lds, int m, int n, cudaStream_t s);
// R = B - A X with A symmetric from its lower triangle (FP64). R, B, X: n x nrhs.
cudaError_t launch_residual(const double* A, int lda, const double* X, int ldx, const double* B, int ldb,
                            double* R, int ldr, int n, int nrhs, cudaStream_t s);
// out[j] = ||R[:, j]||_2^2 and out[nrhs + j] = ||B[:, j]||_2^2 (accumulated with atomics; zeroed here)
cudaError_t launch_col_norms2(const double* R, int ldr, const double* B, int ldb, int n, int nrhs,
                              double* out, cudaStream_t s);
cudaError_t launch_axpy_matrix(double* X, int ldx, const double* D, int ldd, int n, int nrhs, cudaStream_t s);
// out[0] += sum over lower triangle (sym weights) of (A - L L^T)^2, out[1] += ||A||_F^2
cudaError_t launch_backward_error(const double* A, int lda, const double* L, int ldl, int n,
                                  double* out, cudaStream_t s);
// E4M3 quantization of the finished panel A[r0:r0+m, c0:c0+128] (r0, c0 multiples of 128)
// into the FP8 shadows (each optional): S8, FP16 storage of 2^G s e4m3(x/s), and B8, the E4M3
// codes of e4m3(x/s) (bytes), both row-major with row stride lds; one power-of-two scale
// exponent per 128 x 128 tile into tile_exp[(row tile) * ntile_ld + (col tile)].
cudaError_t launch_quant_e4m3(const double* A, int ld, int r0, int m, int c0, int nc, __half* S8, unsigned char* B8,
                              int lds, int* tile_exp, int ntile_ld, int G, unsigned* err, cudaStream_t s);
// every 128 x 128 tile strictly below the diagonal tiles of A[off:off+nb, off:off+nb]
cudaError_t launch_quant_e4m3_lower(const double* A, int ld, int off, int nb, __half* S8, unsigned char* B8, int lds,
                                    int* tile_exp, int ntile_ld, int G, unsigned* err, cudaStream_t s);
// Operand copies for the standalone SYRK / TRSM: the m x k block X (column-major, ldx) into
// S16 row-major (S16[r * lds + c], round to nearest even; an entry beyond kF16Max sets
// DEV_ERR_RANGE16 in err) and into S32 column-major (S32[c * ld32 + r]).
cudaError_t launch_cast_f16_rows(const double* X, int ldx, int m, int k, __half* S16, int lds, unsigned* err,
                                 cudaStream_t s);
cudaError_t launch_cast_f32(const double* X, int ldx, int m, int k, float* S32, int ld32, cudaStream_t s);
// C[.., ..] -= X Y^T for an F8 level by block-scaled E4M3 MMAs (kind::mxf8f6f4, UE8M0 scale
// 2^e per 128 x 128 tile): X rows xr0.., Y rows yr0.., K columns k0.. of the row-major E4M3
// codes S (lds bytes per row), tile_exp as written by the quantization (ntile_ld tiles per
// row of tiles).  xr0, yr0, k0 multiples of 128; lds a multiple of 16.
cudaError_t launch_gemm_f8_tc(double* C, int ldc, const uint8_t* S, int lds, int xr0, int yr0, int k0, int m, int n,
                              int k, bool lower, const int* tile_exp, int ntile_ld, unsigned* dev_err, cudaStream_t s,
                              int occupancy = 0);
// TF32 split of an FP32-level block: hi = tf32(fp32(a)), lo = tf32(fp32(a) - hi), read from the
// column-major FP64 block A[r0.., c0..] (m x nc) and written row-major at [(r0 + i) ldh + c0 + j].
cudaError_t launch_split_tf32(const double* A, int lda, int r0, int m, int c0, int nc, float* H, float* Lo, int ldh,
                              cudaStream_t s);
// C[.., ..] -= X Y^T from TF32 splits (error-corrected FP32 GEMM on tcgen05, kind::tf32):
// X rows xr0.., Y rows yr0.., K columns k0.. of the row-major hi (H) / lo (Lo) arrays (ldh);
// k0 and ldh multiples of 4, H and Lo 16-byte aligned.  `lower` as for the FP16 GEMM.
cudaError_t launch_gemm_tf32x3_tc(double* C, int ldc, const float* H, const float* Lo, int ldh, int xr0, int yr0,
                                  int k0, int m, int n, int k, bool lower, unsigned* dev_err, cudaStream_t s,
                                  int occupancy = 0);
// Two-sided power-of-two diagonal scaling of the lower triangle of A (n x n): unscale = false
// computes e[i] = floor(ex_i / 2) from a_ii = m 2^ex_i and sets a_ij <- a_ij 2^-(e_i + e_j);
// unscale = true sets l_ij <- l_ij 2^(e_i) (the factor of the original matrix).  e: n ints.
cudaError_t launch_diag_scale(double* A, int lda, int n, int* e, bool unscale, cudaStream_t s);
// Krylov helpers (FP64 vectors of length n; V column-major with leading dimension ldv):
// out[j] = V[:, j] . w for j < nv (out device, zeroed here); w -= V[:, 0:nv] c (c device);
// y = a x, or y += a x when accumulate.
cudaError_t launch_multi_dot(const double* V, int ldv, int nv, const double* w, int n, double* out, cudaStream_t s);
cudaError_t launch_gemv_sub(double* w, const double* V, int ldv, int nv, const double* c, int n, cudaStream_t s);
cudaError_t launch_scale(double* y, const double* x, double a, int n, bool accumulate, cudaStream_t s);
// sets *flag = 1 if any diagonal entry of A exceeds `limit` (or is not finite)
cudaError_t launch_diag_check(const double* A, int lda, int n, double limit, int* flag, cudaStream_t s);

// ---------------- persistent batched factorization (k_batched.cu) ----------------
// One recorded operation of a system's factorization (the launches the recursion of Alg. 1-3
// would make), on that system's FP64 master:
//   BOP_POTRF: leaf POTRF of the diagonal block at offset a, order b, precision p;
//   BOP_TRSM:  leaf TRSM of rows [a, a+b), columns [c, c+d), FP64 if e else FP32;
//   BOP_GEMM:  A[a:a+b, c:c+d] -= A[a:a+b, e:e+f] A[c:c+d, e:e+f]^T at precision p, lower if g.
enum { BOP_POTRF = 1, BOP_TRSM = 2, BOP_GEMM = 3 };
struct BatchOp {
  int type, p, a, b, c, d, e, f, g;
};
struct BatchSys {
  double* A;          // the system's matrix (column-major, lda), overwritten with L
  int lda, n;
  int op0, op1;       // its operations: ops[op0 .. op1)
  int* info;          // device int: 0 or the failing column
  const double* src;  // when non-null, A's lower triangle is first copied from src (ldsrc)
  int ldsrc;
  float* s32;         // FP32 and FP16 copies of the finished off-diagonal entries (column-
  __half* s16;        // major, leading dimension n), read by the FP32 and FP16 GEMMs; null
                      // when the system's tree has neither precision
};
// Every system's operations by one persistent launch (one CTA per SM, systems taken from
// *ticket in array order).  ticket: device int scratch.
cudaError_t launch_batched_interp(const BatchOp* ops, const BatchSys* sys, int nsys, int* ticket, unsigned* err,
                                  cudaStream_t s);

// ---------------- learned policy (k_policy.cu) ----------------
int policy_nparam();
cudaError_t launch_rowsum(const double* A, int lda, int n, double* rowsum, double* stats, cudaStream_t s);
cudaError_t launch_lanczos_start(double* v, int n, cudaStream_t s);
// R = -A v (A symmetric from its lower triangle, FP32 arithmetic)
cudaError_t launch_symv32(const double* A, int lda, const double* v, double* R, int n, cudaStream_t s);
cudaError_t launch_lanczos_dot(const double* R, const double* v, int n, double* out, cudaStream_t s);
cudaError_t launch_lanczos_axpy(double* R, const double* v, const double* vp, int n, const double* alpha,
                                const double* beta, double* out, cudaStream_t s);
cudaError_t launch_lanczos_next(const double* w, double* vp, double* v, int n, const double* norm2, double* beta,
                                cudaStream_t s);
cudaError_t launch_mlp_forward(const float* p, int batch, const float* X, float* Z, cudaStream_t s);
cudaError_t launch_mlp_grad(const float* p, int batch, const float* X, const int* y, float* g, float* loss,
                            cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int t, float lr, cudaStream_t s);

}  // namespace hrp
