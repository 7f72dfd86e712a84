/*
 * hrp.h — C ABI of the hierarchical recursive precision (HRP) Cholesky library
 * for GB300 (sm_103a).
 *
 * The library factors a dense symmetric positive-definite matrix A = L L^T with the
 * nested recursive Cholesky of Carrica et al., "Hierarchical Recursive Precision for
 * Accelerating Symmetric Linear Solves on MXUs" (arXiv 2601.08082):
 *   - Alg. 1 Tree-POTRF_L, Alg. 2 Tree-TRSM_{R,L,T}, Alg. 3 Tree-SYRK_L (Sec. 3.2):
 *     POTRF, TRSM and SYRK are all split recursively down to GEMMs;
 *   - the tree-structured precision hierarchy of Sec. 3.3: low precision on large
 *     off-diagonal blocks, FP32/FP64 on the recursively refined diagonal;
 *   - the per-block quantization of Sec. 3.4 around every low-precision GEMM;
 * and solves A X = B with the factor (the "linear solve" of the title and abstract),
 * optionally refined in FP64 (mixed-precision iterative refinement, Sec. 1-2).
 *
 * Conventions (all entry points)
 *   - Matrices are column-major with a leading dimension (LAPACK style):
 *     entry (i, j) of A is A[i + j * lda], 0-based, lda >= max(1, n).
 *   - Pointers named d* are DEVICE pointers on the handle's device; other pointers are
 *     host pointers.  The caller owns every buffer it passes; the handle owns its
 *     workspace.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on it in order.  Functions documented as synchronous wait for the
 *     stream before returning (only to read back a status); *_async variants never wait.
 *   - Return value: hrp_status.  On HRP_ERR_INVALID_ARG, hrp_last_arg() returns the
 *     1-based position of the offending argument, negated (LAPACK's -i convention).
 *   - There is no CPU fallback: every step runs in this library's CUDA kernels.
 *   - The first call that needs a larger workspace allocates it (cudaMalloc); make one
 *     call of each size before capturing calls into a CUDA graph.
 *   - A handle's calls share its workspace (shadows, inverses, the solve's mailboxes): calls
 *     on one handle must be ordered on the GPU (one stream, or streams joined by events).
 *     Work that should run concurrently takes one handle per stream.  A handle is used by
 *     one host thread at a time.
 */
#ifndef HRP_H_
#define HRP_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HRP_OK = 0,
  HRP_ERR_INVALID_ARG = 1,     /* bad argument, see hrp_last_arg() */
  HRP_ERR_NOT_SPD = 2,         /* *info = 1-based global column of the first pivot that is not
                                  positive and finite (LAPACK POTRF's convention) */
  HRP_ERR_NO_CONVERGENCE = 3,  /* refinement did not reach tol within max_iter */
  HRP_ERR_ALLOC = 4,           /* device or host allocation failed */
  HRP_ERR_CUDA = 5,            /* a CUDA call failed; hrp_last_error() has the text */
  HRP_ERR_TIMEOUT = 6,         /* a bounded device-side wait expired (no trap, context usable) */
  HRP_ERR_UNSUPPORTED = 7,     /* valid request the library does not implement */
  HRP_ERR_RANGE = 8            /* input outside the range an FP16 tree handles without alpha > 1 */
} hrp_status;

/* Precisions of the tree (Sec. 3.3). HRP_F8E4M3 is OCP E4M3FN with per-tile scales. */
typedef enum { HRP_F64 = 0, HRP_F32 = 1, HRP_F16 = 2, HRP_F8E4M3 = 3 } hrp_prec;

#define HRP_MAX_DEPTH 16

/*
 * Precision tree (Sec. 3.3; notation of Sec. 4.2: a list from the outermost
 * off-diagonal level to the innermost diagonal).
 *   level[t], t < depth: precision of the off-diagonal TRSM/SYRK work of a node at
 *     recursion depth t; nodes deeper than depth-1 use level[depth-1].
 *   inner, inner_size: when inner_size > 0, every node of order <= inner_size runs
 *     entirely in `inner` (F64 or F32), e.g. "[F16,F16,F16,F16,F32|F64@128]".
 *   leaf: Alg. 1 base case size b (a diagonal block of order <= leaf is factored by the
 *     leaf POTRF kernel); 1 <= leaf <= 128.
 *   trsm_leaf, syrk_leaf: Alg. 2 / Alg. 3 base-case sizes (0 = leaf); trsm_leaf <= leaf.
 *   scale_block: tile edge of the FP8 power-of-two scales (128).
 *   trsm_compute: arithmetic of a leaf TRSM at a reduced-precision (F32/F16/F8) level:
 *     0 = FP32 (default), 1 = FP64.  Leaf TRSMs at F64 levels are always FP64.
 *   tile_occupancy: tile width rule of the FP16/FP8 tensor-core GEMMs: each launch takes
 *     the widest tile (256, 128, 64 or 32 columns) that still gives at least
 *     tile_occupancy tiles per SM (0 = 1).  1, 2 and 4 are meaningful; the autotuner
 *     chooses among them.
 * Split point of a node of order n (reading of "e.g. n1 = floor(n/2)"): n/2 rounded to
 * the nearest multiple of 128 for n >= 512, of 16 for 32 <= n < 512, floor(n/2) below.
 */
typedef struct {
  int depth;
  int level[HRP_MAX_DEPTH];
  int leaf;
  int inner;
  int inner_size;
  int trsm_leaf;
  int syrk_leaf;
  int scale_block;
  int trsm_compute;
  int tile_occupancy;
} hrp_tree;

typedef struct hrp_handle_s hrp_handle;

/* Create a handle bound to CUDA device `device`; *out receives it. */
hrp_status hrp_create(hrp_handle** out, int device);
/* Free the handle and all workspace it owns (synchronizes the device). */
hrp_status hrp_destroy(hrp_handle* h);

/* 1-based index (negated) of the last invalid argument, 0 if none. */
int hrp_last_arg(const hrp_handle* h);
/* Text of the last error on this handle (static storage owned by the handle). */
const char* hrp_last_error(const hrp_handle* h);
const char* hrp_status_string(hrp_status s);

/*
 * Parse a tree string "[P0,P1,...,Pd-1]" or "[P0,...,Pd-1|F64@S]" with P in
 * {F64,F32,F16,F8}; leaf as described above; trsm_leaf = syrk_leaf = 0, scale_block = 128.
 */
hrp_status hrp_tree_parse(const char* spec, int leaf, hrp_tree* out);
/* Print a tree in the same notation into buf (always NUL-terminated). Returns length. */
int hrp_tree_format(const hrp_tree* t, char* buf, size_t len);

/*
 * Factor A = L L^T (Alg. 1-3 with the tree's precisions).
 *   n >= 0; dA device, column-major, lda >= max(1,n). The lower triangle is read and
 *   overwritten with L (the computed values, held in FP64); the strict upper triangle
 *   is not touched.
 *   info: host int* (may be NULL). The call synchronizes `stream` once at the end to read
 *   it: 0, or the 1-based column of the first failing pivot (then HRP_ERR_NOT_SPD).
 */
hrp_status hrp_potrf(hrp_handle* h, const hrp_tree* tree, int n, double* dA, int lda,
                     int* info, void* stream);
/*
 * As hrp_potrf, but never synchronizes: d_info is a DEVICE int that receives 0 or the
 * failing column when the enqueued work completes. Capturable in a CUDA graph once the
 * workspace for n exists.
 */
hrp_status hrp_potrf_async(hrp_handle* h, const hrp_tree* tree, int n, double* dA, int lda,
                           int* d_info, void* stream);

/*
 * Solve A X = B given the factor from hrp_potrf (L in the lower triangle of dL):
 * forward substitution L Y = B, then backward L^T X = Y, in 64-row blocks with FP64
 * storage and sums; each block's 16-term partial products are formed in double-float
 * (a pair of binary32 values, about 2^-44 relative to the sum of |terms| at worst, against
 * about 2^-49 for FP64 arithmetic), which moves them off GB300's slow FP64 pipe.
 * dB (n x nrhs, ldb >= max(1,n)) is overwritten with X. Asynchronous.
 */
hrp_status hrp_potrs(hrp_handle* h, int n, int nrhs, const double* dL, int ldl,
                     double* dB, int ldb, void* stream);

/*
 * Factor + solve + FP64 iterative refinement.
 *   dA is NOT modified (the factor lives in the handle's workspace).
 *   X_0 = POTRS(B); repeat R = B - A X (FP64, A's lower triangle read as symmetric),
 *   D = POTRS(R), X += D, until max_j ||r_j||_2/||b_j||_2 <= tol or max_iter corrections.
 *   If the tree's factorization fails (info > 0) the call refactors with the fallback
 *   tree "[F32|F64@128]" and reports it in *used_fallback.  tree == NULL: the learned
 *   policy chooses the tree (see hrp_policy_set below).
 *   iters, resid, info, used_fallback: host pointers (may be NULL). Synchronous (one
 *   device->host read of the residual per iteration).
 */
hrp_status hrp_posv(hrp_handle* h, const hrp_tree* tree, int n, int nrhs,
                    const double* dA, int lda, const double* dB, int ldb,
                    double* dX, int ldx, int max_iter, double tol,
                    int* iters, double* resid, int* info, int* used_fallback, void* stream);

/*
 * Alg. 1 on a matrix in HOST memory: hrp_potrf_async with the transfer overlapped.  The lower
 * triangle of hA (column-major, leading dimension ldha) is copied into dA (lda) in blocks of
 * 128 columns, block b holding rows [128 b, n) of columns [128 b, 128 b + 128), on a copy
 * stream of the handle, in column order; each node of the recursion waits only for the
 * blocks it reads, so the leading blocks are factored while the rest is in flight, and half
 * of the matrix is transferred.  The copies start after the work queued on `stream` before
 * the call; every copy has completed before the work this call queues on `stream` does.
 * Entries of dA above the 128 x 128 diagonal blocks are not written.  hA should be
 * page-locked (cudaHostAlloc or cudaHostRegister): from pageable memory the copies are staged
 * through the driver and overlap nothing.  hA must stay unchanged until the copies are done:
 * synchronizing `stream` covers them, also after an error return.  Otherwise as
 * hrp_potrf_async: *d_info (device) as in hrp_potrf, no synchronization.
 */
hrp_status hrp_potrf_host(hrp_handle* h, const hrp_tree* tree, int n, const double* hA, int ldha, double* dA,
                          int lda, int* d_info, void* stream);

/*
 * Arithmetic of the FP64 leaves (Alg. 1 base case, the 128 x 128 leaf on an 8-CTA cluster).
 * The leaf's pivot chains, TRSM substitutions and rank-16 updates lie on the critical path of
 * the whole factorization, and FP64 operations take ~64 cycles on this GPU.
 *   mode 1: the leaf runs in double-float arithmetic (pairs of binary32, Dekker 1971; about
 *     48 significant bits, relative error of each operation a few units of 2^-48) on the FP32
 *     pipe.  The leaf is scaled by a power of two and converted exactly (hi) and to 2^-48
 *     (lo) from FP64 on load, and L is rounded back to FP64 on store.  A leaf with an entry
 *     that is not finite, or a diagonal entry or pivot that is not positive or falls below
 *     2^-36 times its largest diagonal entry, is factored again by the FP64 schedule in the
 *     same launch (bitwise the mode-0 result; a failing column is reported as in mode 0).
 *   mode 0: the leaf in FP64.
 *   mode -1 (default): mode 1 for trees with a level below FP64, mode 0 for all-FP64 trees.
 * Applies to hrp_potrf, hrp_potrf_async, hrp_posv and the stream-pool batched calls.
 */
hrp_status hrp_set_leaf_chain(hrp_handle* h, int mode);

/*
 * F8 levels (E4M3 with one power-of-two scale 2^e per 128 x 128 tile of L).  mode 0 (default):
 * the F8-level GEMMs are block-scaled E4M3 tensor-core products (kind::mxf8f6f4, one UE8M0
 * scale 127 + e per row and 32 K elements, constant over each tile), at the FP8 rate.  mode 1:
 * the same E4M3 values times 2^(e + 8), exact in FP16, multiplied by the FP16 GEMM and scaled
 * back by 2^-16 (FP16 rate).  Both form the exact products of the quantized operands with
 * FP32 accumulation.
 */
hrp_status hrp_set_f8_gemm(hrp_handle* h, int mode);

/*
 * FP32 levels on tensor cores (the paper names tensor-core FP32 regions as future work,
 * Sec. 5).  on = 0 (default): the FP32-level GEMMs of hrp_potrf, hrp_potrf_async, hrp_posv and
 * hrp_syrk run on the SIMT FP32 pipe.  on = 1: products of at least 2e6 multiply-adds with
 * K >= 32 run on tcgen05 by the error-corrected TF32 split of Ootomo and Yokota (2022): each
 * FP32 operand x is held as hi = tf32(x), lo = tf32(x - hi) (|x - hi - lo| <= 2^-22 |x|), the
 * product is hi hi^T + (hi lo^T + lo hi^T) with FP32 accumulation, the two parts in separate
 * accumulators, and the result is within 3 2^-22 |X||Y|^T plus the FP32 accumulation error of
 * the FP32 product.  The split arrays take 8 bytes per entry of L (n x ceil64(n) x 2 floats).
 * The batched calls and hrp_trsm keep the SIMT path.
 */
hrp_status hrp_set_fp32_split(hrp_handle* h, int on);

/*
 * Scaling before the recursion (dynamic quantization, the paper's future work for matrices of
 * extreme dynamic range, Sec. 4.5).  mode 0 (default): none; every FP16 operand is checked
 * against 65504 (Sec. 3.4 with alpha = 1, HRP_ERR_RANGE otherwise).  mode 1: hrp_potrf and
 * hrp_posv factor D^-1 A D^-1 with D = diag(2^e_i), e_i = floor(ex_i / 2) for
 * a_ii = m 2^ex_i (m in [0.5, 1)), so every scaled diagonal entry lies in [0.5, 2); the factor
 * returned is L = D L_hat.  Powers of two make both scalings exact (away from subnormals), and
 * every row meets the FP16 range at the scale of its own diagonal.
 */
hrp_status hrp_set_scaling(hrp_handle* h, int mode);

/*
 * Refinement of hrp_posv.  mode 0 (default): classical iterative refinement, each
 * correction an FP32 POTRS with the factor.  mode 1: GMRES-IR (Carson and Higham, the
 * refinement literature of the paper's Sec. 1-2): each correction d solves A d = r by
 * GMRES on M^{-1} A d = M^{-1} r (M = L L^T the computed factor, applied by an FP64 POTRS;
 * FP64 products with A) from d = 0, at most `restart` steps (1..60), stopped when the
 * preconditioned residual falls to inner_tol (0 < inner_tol < 1) of its start; it converges
 * where the classical iteration stalls or diverges (kappa(A) times the factor's error
 * above 1).  The outer loop, stopping rule and fallback tree are those of hrp_posv.
 * hrp_last_inner_iterations: GMRES steps of the last hrp_posv (0 in mode 0).
 */
hrp_status hrp_set_refinement(hrp_handle* h, int mode, int restart, double inner_tol);
long long hrp_last_inner_iterations(const hrp_handle* h);

/*
 * Relative backward error ||A - L L^T||_F / ||A||_F computed on the device in FP64
 * (A symmetric from its lower triangle in dA; L from the lower triangle of dL).
 * *out is a host double. Synchronous.
 */
hrp_status hrp_backward_error(hrp_handle* h, int n, const double* dA, int lda,
                              const double* dL, int ldl, double* out, void* stream);

/*
 * Timing mode (hrp_set_timing(h, 1)): every kernel the next factorizations enqueue is
 * bracketed by CUDA events on the call's stream, and the factorization synchronizes the
 * stream once at its end (so do not enable it while capturing a graph).
 * hrp_get_timing writes, for each kernel class c = 0..4 (leaf POTRF, leaf TRSM, tcgen05
 * GEMM (FP16, F8 and TF32-split levels), SIMT GEMM, other), the triple out[3c] = summed device milliseconds,
 * out[3c+1] = launches, out[3c+2] = algorithmic flops of the last factorization.
 * Returns the number of doubles written (<= n).
 */
hrp_status hrp_set_timing(hrp_handle* h, int enable);
int hrp_get_timing(hrp_handle* h, double* out, int n);

/*
 * The launches of the last factorization in timing mode, in enqueue order, four doubles each:
 * kernel class (as hrp_get_timing), stream (0: the critical stream, d: the lookahead side
 * stream of recursion depth d), start and end in milliseconds from the first launch's start
 * event.  Returns the number of doubles written (a multiple of 4, <= n).  The events around
 * every launch add a few microseconds each, so gaps read from it are upper bounds.
 */
int hrp_get_timeline(hrp_handle* h, double* out, int n);

/*
 * Lookahead (on by default): after a node's A11 is factored, the rows of its A21 that the
 * next diagonal block needs, and that block's share of the SYRK, run on the handle's
 * critical stream (highest priority); the remaining TRSM rows and SYRK blocks run on a side
 * stream of that recursion depth and are awaited only when the recursion reaches them, so
 * they overlap the leaf factorizations.  The arithmetic of every entry is unchanged.  The
 * streams fork from and join into the call's stream (capturable in a CUDA graph).
 * hrp_set_lookahead(h, 0) keeps every launch on the call's stream.
 */
hrp_status hrp_set_lookahead(hrp_handle* h, int enable);

/*
 * Autotuner for the recursion cut-offs of a tree: the base-case sizes b of Alg. 1
 * (leaf) and Alg. 2 (trsm_leaf), which the paper leaves as parameters (Sec. 3.2).  The
 * precision list, the inner region and trsm_compute are never changed.
 * hrp_autotune_candidates (host only, no device work): writes up to `cap` candidate trees
 *   into out and returns how many there are (-1 for an invalid tree): the given tree
 *   first, then leaf in {128, 64, 32} with trsm_leaf in {leaf, leaf/2}, then, for trees
 *   with an F16 or F8 level, each of those with tile_occupancy 2 and 4; no duplicates, at
 *   most 24.  A tree with an F8 level admits only leaf = trsm_leaf = 128 (its E4M3 tiles
 *   live on the 128 x 128 grid).
 * hrp_autotune: factors a seeded SPD matrix of order n (1 <= n <= 65535) drawn on the
 *   device (off-diagonal entries uniform in [-1, 1), n on the diagonal, the paper's
 *   synthetic generator of Sec. 4.1) with every candidate: one warm-up, then `reps`
 *   factorizations timed with CUDA events on `stream`, keeping the median.  A candidate
 *   counts only if it factors the matrix (info = 0) with a backward error at most
 *   4 x that of the given tree + 1e-15.  *out receives the fastest, *ms (may be NULL) its
 *   median milliseconds.  The choice is cached in the handle under (n, precision list,
 *   inner region, trsm_compute); a later call with that key returns it at once unless
 *   flags & 1 (re-tune).  Synchronous; allocates 2 n^2 doubles for the call's duration.
 *   Errors: the given tree's own failure (HRP_ERR_NOT_SPD, HRP_ERR_UNSUPPORTED, ...) is
 *   returned; other candidates that fail are skipped.
 */
int hrp_autotune_candidates(const hrp_tree* tree, hrp_tree* out, int cap);
/*
 * hrp_autotune_orders: hrp_autotune for each of the `count` orders in orders[] (host
 *   array).  The batched calls (hrp_potrf_batched, hrp_posv_batched) then give a system of
 *   order n the cut-offs and tile rule tuned at the largest tuned order <= n with the same
 *   precisions (its own tree's otherwise).  Synchronous.
 */
hrp_status hrp_autotune_orders(hrp_handle* h, const hrp_tree* tree, int count, const int* orders, int reps,
                               void* stream);
hrp_status hrp_autotune(hrp_handle* h, const hrp_tree* tree, int n, int reps, int flags, hrp_tree* out,
                        float* ms, void* stream);

/*
 * Batched factorization of `batch` independent systems (a many-systems workload; the
 * paper factors one matrix at a time).  Host arrays: trees[i] (the tree of
 * system i; entries may share one tree; F8 levels are not batched), n[i], dA[i] (device
 * pointer), lda[i].  trees == NULL, or trees[i] == NULL: the learned policy chooses that
 * system's tree (hrp_policy_predict on its features, F8 levels taken in FP16; the
 * fallback tree when no policy is loaded); the feature pass synchronizes `stream`, so
 * such a call cannot be captured in a graph.  d_info: DEVICE array of batch ints, info of each system as in
 * hrp_potrf.  Each system runs the recursion of Alg. 1-3 on one stream of an internal
 * pool forked from `stream` (longest systems first) and joined back into it; the call only
 * enqueues work (capturable into one CUDA graph once the workspace for these sizes exists).
 * That is batched mode 0 (the default).  Batched mode 1 (hrp_set_batched_mode): the same
 * recursion is recorded per system as a list of base cases and GEMMs (each at the precision
 * its tree gives it) and ONE persistent launch runs them: one CTA per SM takes the next
 * system (longest first) from an atomic ticket and executes its list in order; no CTA waits
 * on another.  Mode 1 runs every operation on CUDA cores (FP16 operands rounded on load,
 * FP32 accumulation; FP32 substitution for reduced-precision leaf solves).  The first call
 * with a given batch (orders, trees, pointers) uploads its lists to device memory that the
 * handle keeps for that batch until it is destroyed (36 bytes per operation); later calls
 * with the same batch, and graphs that capture them, reuse it.  Capturing a batch that was
 * never run returns HRP_ERR_INVALID_ARG.
 */
hrp_status hrp_potrf_batched(hrp_handle* h, const hrp_tree* const* trees, int batch, const int* n,
                             double* const* dA, const int* lda, int* d_info, void* stream);
/*
 * Batched POTRS (FP64): for each i, dB[i] (n[i] x nrhs, ldb[i]) <- A_i^{-1} dB[i] with the
 * factor in the lower triangle of dL[i].  Same stream pool and capture rules as above.
 */
hrp_status hrp_potrs_batched(hrp_handle* h, int batch, const int* n, double* const* dL, const int* ldl,
                             int nrhs, double* const* dB, const int* ldb, void* stream);
/* Batched factorization mode of the handle: 0 = stream pool, 1 = persistent launch (above;
   also used by the factorizations of hrp_posv_batched). */
hrp_status hrp_set_batched_mode(hrp_handle* h, int mode);

/*
 * Learned precision policy (not in the paper; an extension of it).  A small network
 * (MLP 12 -> 64 -> 64 -> 8, ReLU, FP32) maps cheap matrix features to one of eight
 * candidate trees (hrp_policy_tree); hrp_posv with tree == NULL uses it, and falls back
 * to the conservative tree (index 0, "[F32|F64@128]") when the chosen factorization fails.
 *
 * hrp_policy_features: the 12 features of the symmetric A (lower triangle of dA), host
 *   float feat[12]: log2 n; min, mean and fraction > 1 of the row dominance ratios
 *   a_ii / sum_{j!=i} |a_ij| (min clamped at 1e6); log10 ||A||_F; log10 of the diagonal
 *   max, min and their ratio; log10 of the extreme Ritz values of `lanczos_steps` Lanczos
 *   steps (start vector v_i ~ 1 + (i mod 7)/7), their ratio (condition estimate), and
 *   log10(n lambda_min / ||A||_F).  FP64 on the device; synchronous.
 * hrp_mlp_forward / hrp_mlp_grad / hrp_mlp_adam: the network's kernels on device arrays:
 *   params (hrp_mlp_param_count() = 5512 floats: W1 64x12, b1, W2 64x64, b2, W3 8x64, b3,
 *   row-major), X (batch x 12), logits Z (batch x 8), labels y (batch ints); grad gets the
 *   gradient of the mean softmax cross-entropy and *d_loss the loss; Adam with
 *   beta = (0.9, 0.999), eps 1e-8, bias-corrected at step `step` (1-based).  Asynchronous.
 * hrp_policy_set: install trained parameters (host arrays) and the input standardization
 *   (mean[12], scale[12]).
 * hrp_policy_load: the same from a file written by train_policy.py (JSON, format
 *   "hrp-policy-v1": "trees" must be this library's 8 candidate trees in order, "params"
 *   5512 numbers, "mean" and "scale" 12 each, optionally "min_n": [order] as for
 *   hrp_policy_set_min_order); HRP_ERR_INVALID_ARG (with hrp_last_error) when the file is
 *   missing or does not match.
 * hrp_policy_set_min_order: systems of order n < n_min take the fallback tree (index 0) without
 *   the feature pass, where the pass costs more than the policy saves (0, the default after
 *   hrp_policy_set: every order asks the policy).
 * hrp_policy_predict: the predicted tree for host feat[12] into *out and its index into
 *   *index (either may be NULL, not both); HRP_ERR_INVALID_ARG when no policy is loaded.
 * hrp_last_policy_choice: the index hrp_posv chose last (-1 if a tree was given).
 */
hrp_status hrp_policy_features(hrp_handle* h, int n, const double* dA, int lda, int lanczos_steps, float* feat,
                               void* stream);
hrp_status hrp_mlp_forward(hrp_handle* h, const float* d_params, int batch, const float* d_X, float* d_Z,
                           void* stream);
hrp_status hrp_mlp_grad(hrp_handle* h, const float* d_params, int batch, const float* d_X, const int* d_y,
                        float* d_grad, float* d_loss, void* stream);
hrp_status hrp_mlp_adam(hrp_handle* h, float* d_params, const float* d_grad, float* d_m, float* d_v, int step,
                        float lr, void* stream);
int hrp_mlp_param_count(void);
hrp_status hrp_policy_set(hrp_handle* h, const float* params, const float* mean, const float* scale);
hrp_status hrp_policy_load(hrp_handle* h, const char* path);
hrp_status hrp_policy_set_min_order(hrp_handle* h, int n_min);
hrp_status hrp_policy_predict(hrp_handle* h, const float* feat, hrp_tree* out, int* index);
hrp_status hrp_policy_tree(int index, hrp_tree* out);
int hrp_last_policy_choice(const hrp_handle* h);

/*
 * Batched hrp_posv: for each system i (host arrays as in hrp_potrf_batched, plus dB[i],
 * ldb[i], dX[i], ldx[i]; 1 <= nrhs <= 16): factor a copy of A_i with trees[i] (NULL: the
 * policy's choice, as above; dA[i] is not modified), refactor with "[F32|F64@128]" where
 * that fails or needs alpha > 1 (used_fallback[i] = 1), solve,
 * and refine in FP64 until ||b - A x||_2 / ||b||_2 <= tol per column or max_iter.  All
 * systems advance together, one round of refinement at a time, on the internal stream
 * pool.  info, iters, resid, used_fallback: host arrays of batch entries (may be NULL).
 * Synchronous (one device->host read per round).
 */
hrp_status hrp_posv_batched(hrp_handle* h, const hrp_tree* const* trees, int batch, const int* n,
                            double* const* dA, const int* lda, int nrhs, double* const* dB, const int* ldb,
                            double* const* dX, const int* ldx, int max_iter, double tol, int* info, int* iters,
                            double* resid, int* used_fallback, void* stream);

/*
 * Standalone recursive SYRK and TRSM (Alg. 3 and Alg. 2, the kernels of Sec. 4.2's SYRK and
 * TRSM experiments) with the tree's precision list applied to their own recursion: the GEMM
 * of a node at depth t runs at level[t] (deeper nodes at the last entry; a node of order <=
 * inner_size at `inner`) with FP32 accumulation below FP64, and a base case at its node's
 * precision (FP32 arithmetic for F16/F32 base cases unless trsm_compute = 1).  FP16 operands
 * are copies rounded to nearest even; one beyond 65504 is recorded as HRP_ERR_RANGE (read by
 * hrp_check).  F8 levels are not supported here.  Both calls only enqueue work.
 * hrp_syrk: C <- C - A A^T on the lower triangle of the n x n dC (ldc); dA is n x k (lda).
 *   Base case size: syrk_leaf (0 = leaf).  The strict upper triangle of C is not touched.
 * hrp_trsm: B <- B L^{-T} (TRSM_{R,L,T}: solves X L^T = B) for dB m x n (ldb) and the lower
 *   triangle of the n x n dL (ldl), which is not modified.  Base case: min(m, n) <= trsm_leaf
 *   (0 = leaf), trsm_leaf <= 128 unless m <= 128.
 * Workspace: an FP16 copy of A (n x k) or of [B; L] ((m + n) x n), and an FP32 copy when the
 * tree has F32 levels, in the handle.
 */
hrp_status hrp_syrk(hrp_handle* h, const hrp_tree* tree, int n, int k, const double* dA, int lda, double* dC, int ldc,
                    void* stream);
hrp_status hrp_trsm(hrp_handle* h, const hrp_tree* tree, int m, int n, const double* dL, int ldl, double* dB, int ldb,
                    void* stream);

/* Number of kernel launches enqueued by the last hrp_potrf/potrs/posv call. */
long long hrp_last_launch_count(const hrp_handle* h);

/*
 * Device-side status.  Kernels record failures that only the device sees in the handle's
 * status word: a bounded wait that expired (POTRS sweeps; the tcgen05 GEMM pipeline) and
 * an operand outside the FP16 / E4M3 range.  Synchronous calls read and clear it before
 * they return; asynchronous calls (hrp_potrf_async, hrp_potrs, the batched calls) leave it
 * for the next synchronous call or for hrp_check.
 * hrp_check: synchronizes `stream`, reads and clears the word; returns HRP_ERR_TIMEOUT,
 *   HRP_ERR_RANGE or HRP_OK.
 * hrp_set_wait_limit: the limit of the bounded waits in the handle's solves (POTRS
 *   sweeps), 1 us .. 2 s (the default).  A sweep whose wait expires writes NaN into the
 *   rows it could not solve and publishes them, so dependent rows come out NaN too.
 * hrp_wait_selftest: one device thread waits, through the sweeps' bounded-wait routine,
 *   on a mailbox entry that nothing fills, for `microseconds` (1 .. 2e6); the wait expires,
 *   the kernel records the timeout and returns, and the call reports HRP_ERR_TIMEOUT with
 *   *waited_us (host, may be NULL) the time the device waited.  The context stays usable.
 *   Synchronous.
 */
hrp_status hrp_check(hrp_handle* h, void* stream);
hrp_status hrp_set_wait_limit(hrp_handle* h, long long microseconds);
hrp_status hrp_wait_selftest(hrp_handle* h, long long microseconds, double* waited_us, void* stream);

/*
 * hrp_potrs_noalloc: the same solve as hrp_potrs (B <- A^{-1} B from the factor in the
 * lower triangle of dL, FP64, forward then backward substitution), for callers that may
 * not allocate device memory when they solve: applications whose memory is owned by
 * their own pool, loops where cudaMalloc's implicit synchronization is unacceptable, or
 * plugins handed buffers but no allocator.  The paper has no counterpart; this is a
 * property of the library, not of the method.
 *   - Takes no handle and allocates nothing: its scratch (diagonal-block inverses, the
 *     sweeps' mailboxes, a ticket) is one fixed device array inside the library, about
 *     6 MiB, which every GPU that loads the library keeps until the process exits.
 *   - n must be <= 8192 (the array's size); larger n returns HRP_ERR_INVALID_ARG, as do
 *     negative sizes, NULL buffers and leading dimensions < max(1, n).
 *   - The first call on a device (with that device current) looks up the array's device
 *     address and zeroes its ticket with a synchronous cudaMemset; make that first call
 *     before any stream capture.  Later calls only enqueue work on `stream`.
 *   - All calls share the one array: calls that overlap on the GPU (different streams,
 *     no ordering between them) race and must not be issued.
 *   - The call only enqueues work, so it cannot return a device-side failure: a bounded
 *     device wait that expires inside a sweep (it gives up after 2 s) leaves NaN in the
 *     rows of dB it could not solve and in every row that depends on them.  Check the
 *     result for NaN where that matters.
 */
hrp_status hrp_potrs_noalloc(int n, int nrhs, const double* dL, int ldl, double* dB, int ldb,
                             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HRP_H_ */
