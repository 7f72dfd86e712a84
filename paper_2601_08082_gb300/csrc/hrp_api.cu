// C ABI of the HRP library and the host-side recursion scheduler.
//
// The scheduler walks Alg. 1 (Tree-POTRF_L), Alg. 2 (Tree-TRSM_{R,L,T}) and Alg. 3
// (Tree-SYRK_L) on the host and enqueues one kernel per base case or GEMM on the caller's
// stream, choosing each kernel by the precision the tree assigns to the node (Sec. 3.3):
//   - leaf POTRF: FP64 or FP32 in shared memory (k_leaf.cu);
//   - leaf TRSM: FP64 substitution, or FP32 through the inverse of the diagonal leaf;
//   - GEMM at an F16 level: tcgen05 FP16 GEMM from the FP16 shadow (k_gemm_tc.cu),
//     at F32/F64 levels a SIMT GEMM on the FP64 master (k_gemm_simt.cu).
// Tree-SYRK is enqueued as ONE lower-triangle GEMM: every entry of C is produced by
// exactly one GEMM (or leaf SYRK) of the recursion with the full inner dimension and the
// node's precision, so the flattened launch performs the same arithmetic per entry.
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "hrp_internal.cuh"

namespace hrp {
// Lanczos steps of the policy's condition estimate (the training features use the same)
constexpr int kPolicyLanczosSteps = 10;
// kernel classes reported by hrp_get_timing
enum { CLS_POTRF = 0, CLS_TRSM = 1, CLS_GEMM_TC = 2, CLS_GEMM_SIMT = 3, CLS_OTHER = 4, kNumClasses = 5 };
}

struct hrp_handle_s {
  int device = 0;
  int last_arg = 0;
  char last_err[512] = {0};
  int* d_info = nullptr;       // internal info word
  unsigned* d_err = nullptr;   // device error flags
  int* d_ticket = nullptr;
  double* d_probe = nullptr;   // a mailbox entry nothing fills (hrp_wait_selftest) and the time waited
  unsigned long long wait_ns = hrp::kWaitTimeoutNs;   // limit of the solves' bounded waits
  __half* shadow = nullptr;
  size_t shadow_cap = 0;       // elements
  float* w32 = nullptr;
  size_t w32_cap = 0;          // elements
  __half* shadow8 = nullptr;   // E4M3 values (times 2^G, exact) in FP16 storage
  size_t shadow8_cap = 0;
  unsigned char* bytes8 = nullptr;   // E4M3 codes (row-major, ld lds) for the block-scaled MMAs
  size_t bytes8_cap = 0;
  // F8-level GEMMs: 0 = block-scaled E4M3 MMAs (FP8 rate, default), 1 = the E4M3 values in
  // FP16 storage on kind::f16 (FP16 rate; same products)
  int f8_gemm = 0;
  float* shadow32 = nullptr;   // FP32 copy of L (column-major, ld n) for the FP32-level GEMMs
  size_t shadow32_cap = 0;
  int* tile_exp = nullptr;     // power-of-two scale exponent of every 128 x 128 tile
  size_t tile_exp_cap = 0;
  double* fact = nullptr;      // posv factor copy
  size_t fact_cap = 0;
  double* work = nullptr;      // posv residual/correction
  size_t work_cap = 0;
  unsigned char* pwork = nullptr;  // POTRS diagonal-block inverses
  size_t pwork_cap = 0;
  double* d_norms = nullptr;   // 2 * 64 doubles
  double* h_norms = nullptr;   // pinned host mirror
  long long launches = 0;
  bool timing = false;
  // per-kernel-class timing of the last factorization (timing mode only)
  double cls_ms[hrp::kNumClasses] = {0};
  std::vector<double> timeline;   // timing mode: class, stream, start ms, end ms per launch
  double cls_launches[hrp::kNumClasses] = {0};
  double cls_flops[hrp::kNumClasses] = {0};
  std::vector<cudaEvent_t> events;
  // batched calls: a pool of streams and per-system workspace
  std::vector<cudaStream_t> bstreams;
  std::vector<cudaEvent_t> bevents;
  unsigned char* bwork = nullptr;
  size_t bwork_cap = 0;
  // learned policy: feature workspace and the (standardization-folded) MLP parameters
  double* fwork = nullptr;
  size_t fwork_cap = 0;
  float* policy = nullptr;     // device, 5512 floats
  float* pio = nullptr;        // device, 12 inputs + 8 logits
  bool policy_set = false;
  int last_choice = -1;
  // orders below this take the fallback tree without the feature pass (the pass would cost
  // more than the policy saves there); 0 = every order asks the policy
  int policy_min_n = 0;
  // autotuner: tuned tree and its median time by (precision list, inner region, trsm_compute)
  // and order n
  std::map<std::string, std::map<int, std::pair<hrp_tree, float>>> tune_cache;
  // lookahead: the critical stream (highest priority), side streams by recursion depth, and
  // a pool of events for the dependencies between them
  bool lookahead = true;
  std::vector<cudaStream_t> lstreams;
  std::vector<cudaEvent_t> levents;
  // hrp_potrf_host: the copy stream and one event per 128-column block of the copied matrix
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> col_events;
  // refinement of hrp_posv: 0 = classical (POTRS corrections), 1 = GMRES-IR
  int refine_mode = 0;
  int gmres_restart = 20;
  double gmres_tol = 1e-8;
  double* kwork = nullptr;     // GMRES basis and vectors
  size_t kwork_cap = 0;
  long long inner_steps = 0;   // GMRES steps of the last hrp_posv
  // scaling before the recursion: 0 = none (the static Sec. 3.4 rule, alpha = 1 checked),
  // 1 = two-sided power-of-two diagonal scaling (dynamic quantization)
  int scaling = 0;
  int* scale_exp = nullptr;
  size_t scale_exp_cap = 0;
  // FP32-level GEMMs: 0 = SIMT FP32 (default), 1 = error-corrected TF32 split on tcgen05
  int fp32_split = 0;
  // FP64 leaves' 16 x 16 diagonal-tile Cholesky: 1 = double-float on the FP32 pipe, 0 = FP64,
  // -1 (default) = double-float when the tree has a level below FP64, else FP64
  int leaf_chain = -1;
  float* split32 = nullptr;    // hi then lo, row-major (see Fact::h32)
  size_t split32_cap = 0;
  // batched factorization: 0 = one stream per system (default), 1 = one persistent launch
  int batched_mode = 0;
  // persistent launch plans: every distinct batch (its operation and system lists, byte for
  // byte) keeps its own device copy and ticket, so a graph that captured it stays valid
  struct Plan {
    std::string key;
    hrp::BatchOp* ops = nullptr;
    hrp::BatchSys* sys = nullptr;
    int* ticket = nullptr;
    int nsys = 0;
    unsigned char* shadows = nullptr;   // the systems' FP32 and FP16 shadows (owned by the plan)
  };
  std::vector<Plan> plans;
};

namespace hrp {
namespace {

hrp_status set_err(hrp_handle* h, hrp_status st, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->last_err, sizeof(h->last_err), fmt, ap);
    va_end(ap);
  }
  return st;
}
hrp_status bad_arg(hrp_handle* h, int pos, const char* what) {
  if (h) h->last_arg = -pos;
  return set_err(h, HRP_ERR_INVALID_ARG, "argument %d: %s", pos, what);
}

template <typename T>
hrp_status ensure(hrp_handle* h, T** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return HRP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (need == 0) return HRP_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_err(h, HRP_ERR_ALLOC, "cudaMalloc(%zu bytes) failed: %s", need * sizeof(T), cudaGetErrorString(e));
  }
  *cap = need;
  return HRP_OK;
}

int split(int n) {
  int q;
  if (n >= 512) q = 128;
  else if (n >= 32) q = 16;
  else return n / 2;
  int n1 = q * ((n + q) / (2 * q));
  if (n1 <= 0 || n1 >= n) return n / 2;
  return n1;
}

int node_prec(const hrp_tree* t, int depth, int n) {
  if (t->inner_size > 0 && n <= t->inner_size) return t->inner;
  int d = depth < t->depth ? depth : t->depth - 1;
  return t->level[d];
}

hrp_status validate_tree(hrp_handle* h, const hrp_tree* t, int pos) {
  if (!t) return bad_arg(h, pos, "tree is NULL");
  if (t->depth < 1 || t->depth > HRP_MAX_DEPTH) return bad_arg(h, pos, "tree depth out of range");
  for (int i = 0; i < t->depth; ++i)
    if (t->level[i] < HRP_F64 || t->level[i] > HRP_F8E4M3) return bad_arg(h, pos, "bad precision in tree");
  if (t->leaf < 1 || t->leaf > 128) return bad_arg(h, pos, "leaf must be in [1, 128]");
  if (t->inner_size < 0) return bad_arg(h, pos, "inner_size < 0");
  if (t->inner_size > 0 && t->inner != HRP_F64 && t->inner != HRP_F32) return bad_arg(h, pos, "inner must be F64 or F32");
  int tl = t->trsm_leaf ? t->trsm_leaf : t->leaf;
  if (tl < 1 || tl > t->leaf) return bad_arg(h, pos, "trsm_leaf must be in [1, leaf]");
  int sl = t->syrk_leaf ? t->syrk_leaf : t->leaf;
  if (sl < 1) return bad_arg(h, pos, "syrk_leaf < 0");
  if (t->trsm_compute != 0 && t->trsm_compute != 1) return bad_arg(h, pos, "trsm_compute must be 0 or 1");
  if (t->tile_occupancy < 0 || t->tile_occupancy > 8) return bad_arg(h, pos, "tile_occupancy must be in [0, 8]");
  if (t->level[t->depth - 1] == HRP_F8E4M3 && t->inner_size < t->leaf)
    return bad_arg(h, pos, "the innermost (diagonal) precision cannot be F8");
  return HRP_OK;
}

bool tree_has(const hrp_tree* t, int prec) {
  for (int i = 0; i < t->depth; ++i)
    if (t->level[i] == prec) return true;
  return t->inner_size > 0 && t->inner == prec;
}

// the autotuner's cache key: everything it never changes (precisions, inner region, TRSM
// arithmetic); the tuned cut-offs and tile rule are filed under it by order
std::string tune_key(const hrp_tree* t) {
  std::string k = "d=" + std::to_string(t->depth) + ";in=" + std::to_string(t->inner) + "@" +
                  std::to_string(t->inner_size) + ";tc=" + std::to_string(t->trsm_compute) + ";L=";
  for (int i = 0; i < t->depth; ++i) k += std::to_string(t->level[i]) + ",";
  return k;
}

// t with the cut-offs and tile rule tuned at the largest tuned order <= n (t unchanged if
// none was tuned for its precisions)
void apply_tuned(const hrp_handle* h, hrp_tree* t, int n) {
  auto it = h->tune_cache.find(tune_key(t));
  if (it == h->tune_cache.end() || it->second.empty()) return;
  auto jt = it->second.upper_bound(n);
  if (jt == it->second.begin()) return;
  --jt;
  t->leaf = jt->second.first.leaf;
  t->trsm_leaf = jt->second.first.trsm_leaf;
  t->syrk_leaf = jt->second.first.syrk_leaf;
  t->tile_occupancy = jt->second.first.tile_occupancy;
}

// ------------------------------------------------------------------------------------
// One factorization: the recursion of Alg. 1-3 turned into stream-ordered launches.
// ------------------------------------------------------------------------------------
// FP32-level products large enough to pay for the tensor-core kernel's fixed cost (TMEM
// allocation, barrier set-up, pipeline fill); smaller ones stay on the SIMT pipe
bool split_tc_worth(int m, int n, int k) { return k >= 32 && (double)m * n * k >= 2.0e6; }

struct Fact {
  hrp_handle* h;
  const hrp_tree* t;
  double* A;
  int lda;
  int n;
  int* info;
  cudaStream_t s;
  __half* shadow;       // null if no F16 level
  int lds;
  float* w32;           // null if every level is F64
  __half* shadow8;      // null if no F8 level, or if the F8 GEMMs read bytes8
  unsigned char* bytes8 = nullptr;   // E4M3 codes for the block-scaled F8 GEMMs
  int* tile_exp;
  float* shadow32;      // null: FP32-level GEMMs round their operands from the master
  int ld32;
  // TF32 split of every block finished by an F32 or F64 leaf TRSM (row-major, ld ldh): the
  // operands of the FP32-level GEMMs on tensor cores; null when they run on the SIMT pipe
  float* h32 = nullptr;
  float* l32 = nullptr;
  int ldh = 0;
  bool tc;
  std::map<int, int> leaves;  // leaf offset -> order (blocks with an FP32 inverse)
  // launches so far on each stream, and for each leaf offset the stream and number of the
  // launch that wrote its FP32 inverse
  std::map<cudaStream_t, long long> launch_no;
  std::map<int, std::pair<cudaStream_t, long long>> inv_by;
  cudaError_t err = cudaSuccess;
  long long launches = 0;
  // lookahead (see potrf): s is the stream of the next launch, main_s the critical stream;
  // side[d] takes the off-critical TRSM/SYRK work of nodes at depth d
  bool la = false;
  cudaStream_t main_s = nullptr;
  const std::vector<cudaStream_t>* side = nullptr;
  size_t ev_used = 0;
  std::map<cudaStream_t, bool> waited;   // the stream's next kernel follows a cross-stream wait
  int side_ctas = 0;
  // record mode (persistent batched launch): operations are appended here, nothing is launched
  std::vector<BatchOp>* rec = nullptr;
  // host input (hrp_potrf_host): event of the copy of each 128-column block (rows from the
  // block's diagonal down), and the last block each stream has waited for
  const std::vector<cudaEvent_t>* col_ev = nullptr;
  std::map<cudaStream_t, int> col_waited;
  // timing mode: an event pair around every launch, tagged with its class and flops
  struct Rec { int cls; size_t ev; double flops; int sidx; };
  std::vector<Rec> recs;
  int cur_cls = CLS_OTHER;
  double cur_flops = 0.0;
  size_t ev_next = 0;

  cudaEvent_t event(size_t i) {
    while (h->events.size() <= i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      h->events.push_back(e);
    }
    return h->events[i];
  }
  bool began = false;
  void begin(int cls, double flops) {
    cur_cls = cls;
    cur_flops = flops;
    began = false;
    LaunchCtx& lc = launch_ctx();
    auto w = waited.find(s);
    lc.pdl = !(w != waited.end() && w->second);
    if (w != waited.end()) w->second = false;
    lc.max_ctas = (la && s != main_s) ? side_ctas : 0;
    lc.leaf_df = h->leaf_chain == 1 ||
                 (h->leaf_chain < 0 && (tree_has(t, HRP_F32) || tree_has(t, HRP_F16) || tree_has(t, HRP_F8E4M3)));
    if (h->timing) {
      cudaEvent_t e = event(ev_next);
      began = e && cudaEventRecord(e, s) == cudaSuccess;
    }
  }
  void chk(cudaError_t e) {
    ++launches;
    ++launch_no[s];
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    if (h->timing && began) {
      cudaEvent_t e1 = event(ev_next + 1);
      if (e1 && cudaEventRecord(e1, s) == cudaSuccess) {
        int sidx = 0;
        if (la && side)
          for (size_t q = 0; q < side->size(); ++q)
            if ((*side)[q] == s) sidx = (int)q;
        recs.push_back({cur_cls, ev_next, cur_flops, sidx});
        ev_next += 2;
      }
    }
    began = false;
    cur_cls = CLS_OTHER;
    cur_flops = 0.0;
  }
  int tleaf() const { return t->trsm_leaf ? t->trsm_leaf : t->leaf; }

  void leaf_potrf(int off, int nb, int p) {
    if (rec) {
      rec->push_back(BatchOp{BOP_POTRF, p, off, nb, 0, 0, 0, 0, 0});
      return;
    }
    float* W = nullptr;
    if (w32) {
      W = w32 + (size_t)off * 128;
      leaves[off] = nb;
      inv_by[off] = {s, launch_no[s] + 1};
    }
    begin(CLS_POTRF, (double)nb * nb * nb / 3.0);
    chk(launch_potrf_leaf(A + (size_t)off * lda + off, lda, nb, off, p == HRP_F64, p == HRP_F16, W, 128, info, h->d_err, s));
  }

  void leaf_trsm(int r0, int m, int c0, int nc, int p) {
    if (rec) {
      rec->push_back(BatchOp{BOP_TRSM, p, r0, m, c0, nc, (p == HRP_F64 || t->trsm_compute == 1) ? 1 : 0, 0, 0});
      return;
    }
    double* Ab = A;
    __half* sh = shadow;
    begin(CLS_TRSM, (double)m * nc * nc);
    if (p == HRP_F64 || t->trsm_compute == 1) {
      chk(launch_trsm_leaf64(Ab, lda, r0, m, c0, nc, sh, lds, shadow32, ld32, info, h->d_err, s));
      quant8(r0, m, c0, nc, p);
      split_block(r0, m, c0, nc, p);
      return;
    }
    auto it = leaves.find(c0);
    if (w32 && it != leaves.end() && it->second == nc) {
      // the inverse is complete when this launch starts unless the previous launch on this
      // stream wrote it (a leaf on another stream was awaited through an event, which starts
      // the next launch here without programmatic overlap)
      const auto pr = inv_by.find(c0);
      const bool w_done = pr != inv_by.end() && (pr->second.first != s || pr->second.second < launch_no[s]);
      chk(launch_trsm_leaf32(Ab, lda, r0, m, c0, nc, w32 + (size_t)c0 * 128, 128, sh, lds, shadow32, ld32, info,
                             h->d_err, s, w_done));
    } else {
      chk(launch_trsm_leaf32_subst(Ab, lda, r0, m, c0, nc, sh, lds, shadow32, ld32, info, h->d_err, s));
    }
    quant8(r0, m, c0, nc, p);
    split_block(r0, m, c0, nc, p);
  }
  // the FP32-level GEMMs of a node read blocks finished inside it, by leaves of precision F32
  // (or F64 below an |F64@S cut-off)
  void split_block(int r0, int m, int c0, int nc, int p) {
    if (!h32 || (p != HRP_F32 && p != HRP_F64)) return;
    begin(CLS_OTHER, 0.0);
    chk(launch_split_tf32(A, lda, r0, m, c0, nc, h32, l32, ldh, s));
  }

  // FP8 levels: E4M3 tiles (scale per 128 x 128 tile) of what the F8-level GEMMs of a node
  // read: the panels of its A21 as the F8-level TRSM finishes them (quant8), and the
  // off-diagonal tiles of its L11 in one launch once L11 is factored (quant8_lower)
  static constexpr int kG = 8;   // storage upshift: entries are 2^8 s e4m3(x/s)
  void quant8(int r0, int m, int c0, int nc, int p) {
    if ((!shadow8 && !bytes8) || p != HRP_F8E4M3) return;
    begin(CLS_OTHER, 0.0);
    chk(launch_quant_e4m3(A, lda, r0, m, c0, nc, shadow8, bytes8, lds, tile_exp, n / 128, kG, h->d_err, s));
  }
  void quant8_lower(int off, int nb) {
    if ((!shadow8 && !bytes8) || nb < 256) return;
    begin(CLS_OTHER, 0.0);
    chk(launch_quant_e4m3_lower(A, lda, off, nb, shadow8, bytes8, lds, tile_exp, n / 128, kG, h->d_err, s));
  }

  // C = A[r0:r0+m, c0:c0+nd] -= X Y^T, X = A[r0:r0+m, k0:k0+k], Y = A[c0:c0+nd, k0:k0+k]
  void gemm(int p, int r0, int m, int c0, int nd, int k0, int k, bool lower) {
    if (m <= 0 || nd <= 0 || k <= 0) return;
    if (rec) {
      if (p == HRP_F8E4M3 && err == cudaSuccess) err = cudaErrorNotSupported;
      rec->push_back(BatchOp{BOP_GEMM, p, r0, m, c0, nd, k0, k, lower ? 1 : 0});
      return;
    }
    double* C = A + (size_t)c0 * lda + r0;
    const double* X = A + (size_t)k0 * lda + r0;
    const double* Y = A + (size_t)k0 * lda + c0;
    const double fl = lower ? (double)m * (m + 1) * k : 2.0 * m * nd * k;
    const bool split_tc = p == HRP_F32 && h32 && (k0 % 4) == 0 && split_tc_worth(m, nd, k);
    const bool use_tc = ((p == HRP_F16 || p == HRP_F8E4M3) && tc && (k0 % 8) == 0 && k >= 16) || split_tc;
    begin(use_tc ? CLS_GEMM_TC : CLS_GEMM_SIMT, fl);
    switch (p) {
      case HRP_F64: chk(launch_gemm_simt(C, lda, X, lda, Y, lda, m, nd, k, OpRound::F64, lower, s)); break;
      case HRP_F32:
        // every FP32-level operand is an off-diagonal block of L, finished by a leaf TRSM that
        // also wrote its FP32 rounding into the shadow
        if (split_tc)
          chk(launch_gemm_tf32x3_tc(C, lda, h32, l32, ldh, r0, c0, k0, m, nd, k, lower, h->d_err, s,
                                    t->tile_occupancy));
        else if (shadow32)
          chk(launch_gemm_simt_f32(C, lda, shadow32 + (size_t)k0 * ld32 + r0, ld32, shadow32 + (size_t)k0 * ld32 + c0,
                                   ld32, m, nd, k, lower, s));
        else
          chk(launch_gemm_simt(C, lda, X, lda, Y, lda, m, nd, k, OpRound::F32, lower, s));
        break;
      case HRP_F16:
        if (use_tc)
          chk(launch_gemm_f16_tc(C, lda, shadow, lds, r0, c0, k0, m, nd, k, lower, 1.0, h->d_err, s, t->tile_occupancy));
        else
          chk(launch_gemm_simt(C, lda, X, lda, Y, lda, m, nd, k, OpRound::F16, lower, s));
        break;
      case HRP_F8E4M3:
        if (tc && bytes8)
          chk(launch_gemm_f8_tc(C, lda, bytes8, lds, r0, c0, k0, m, nd, k, lower, tile_exp, n / 128, h->d_err, s,
                                t->tile_occupancy));
        else if (tc && shadow8 && (k0 % 8) == 0 && k >= 16)
          chk(launch_gemm_f16_tc(C, lda, shadow8, lds, r0, c0, k0, m, nd, k, lower, ldexp(1.0, -2 * kG), h->d_err, s,
                                 t->tile_occupancy));
        else if (err == cudaSuccess)
          err = cudaErrorNotSupported;
        break;
      default:
        if (err == cudaSuccess) err = cudaErrorNotSupported;
    }
  }

  // Alg. 2: B = A[r0:r0+m, c0:c0+nc] <- B L^{-T}, L = A[c0:c0+nc, c0:c0+nc].  The rows of B
  // are independent; when B is a slice of a taller block (lookahead), mdec is that block's
  // height, so the slice follows the block's own recursion (same base cases, same GEMMs).
  void trsm(int r0, int m, int c0, int nc, int p, int mdec = -1) {
    if (mdec < 0) mdec = m;
    if (std::min(mdec, nc) <= tleaf()) {
      leaf_trsm(r0, m, c0, nc, p);
      return;
    }
    int n1 = split(nc);
    trsm(r0, m, c0, n1, p, mdec);
    gemm(p, r0, m, c0 + n1, nc - n1, c0, n1, false);   // B2 -= B1 L21^T
    trsm(r0, m, c0 + n1, nc - n1, p, mdec);
  }

  // Alg. 3 flattened: C = A[c0:c0+nc, c0:c0+nc] (lower) -= X X^T, X = A[c0:c0+nc, a0:a0+k]
  void syrk(int c0, int nc, int a0, int k, int p) { gemm(p, c0, nc, c0, nc, a0, k, true); }

  // ---- cross-stream dependencies (lookahead) ----
  cudaEvent_t record(cudaStream_t on) {
    while (h->levents.size() <= ev_used) {
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        if (err == cudaSuccess) err = cudaErrorMemoryAllocation;
        return nullptr;
      }
      h->levents.push_back(e);
    }
    cudaEvent_t e = h->levents[ev_used++];
    cudaError_t r = cudaEventRecord(e, on);
    if (r != cudaSuccess && err == cudaSuccess) err = r;
    return e;
  }
  void wait(cudaStream_t on, cudaEvent_t e) {
    if (!e) return;
    cudaError_t r = cudaStreamWaitEvent(on, e, 0);
    if (r != cudaSuccess && err == cudaSuccess) err = r;
    waited[on] = true;
  }

  // host input: the next launch on s reads columns < col_end (rows from their diagonal down)
  static constexpr int kColBlock = 128;
  void need(int col_end) {
    if (!col_ev || col_ev->empty() || col_end <= 0) return;
    const int b = std::min((int)col_ev->size() - 1, (col_end - 1) / kColBlock);
    int& w = col_waited.emplace(s, -1).first->second;
    if (w >= b) return;
    wait(s, (*col_ev)[b]);
    w = b;
  }

  // Alg. 1.  `rest`: when non-null, the event after which everything of this node outside
  // its A11 block is up to date (A11 itself is up to date now, on the critical stream).
  //
  // Lookahead: the next node, Alg. 1 on A22, starts with its own A11 block, A22[0:m1, 0:m1]
  // (m1 = split(n2)), which needs only the top m1 rows of A21 solved (Alg. 2) and their share
  // of the SYRK (Alg. 3).  Those stay on the critical stream; the other rows of the TRSM and
  // the rest of the SYRK (A22's off-diagonal block and its trailing block) go to the side
  // stream of this depth, and A22's Alg. 1 waits for them only after its own A11.  Every
  // entry still receives the same updates with the same inner dimension and precision.
  void potrf(int off, int nb, int depth, cudaEvent_t rest = nullptr) {
    if (nb <= 0) return;
    int p = node_prec(t, depth, nb);
    if (nb <= t->leaf) {
      wait(s, rest);
      need(off + nb);
      leaf_potrf(off, nb, p);
      return;
    }
    int n1 = split(nb), n2 = nb - n1;
    potrf(off, n1, depth + 1);
    wait(s, rest);
    if (p == HRP_F8E4M3) quant8_lower(off, n1);
    const int m1 = n2 > t->leaf ? split(n2) : n2;
    if (!la || m1 >= n2 || depth + 1 >= (int)side->size()) {
      trsm(off + n1, n2, off, n1, p);              // A21 lies in the columns of A11: copied
      need(off + nb);
      syrk(off + n1, n2, off, n1, p);
      potrf(off + n1, n2, depth + 1);
      return;
    }
    cudaStream_t ss = (*side)[depth + 1];
    const int r0 = off + n1, rb = off + n1 + m1, mb = n2 - m1;
    wait(ss, record(s));                         // L11 (and its FP32 inverses) are final
    trsm(r0, m1, off, n1, p, n2);                // top rows of A21: critical
    cudaEvent_t top = record(s);
    need(r0 + m1);
    syrk(r0, m1, off, n1, p);                    // A22[0:m1, 0:m1] -= A21_top A21_top^T
    s = ss;                                      // side: the rest of Alg. 2 and Alg. 3
    trsm(rb, mb, off, n1, p, n2);
    wait(ss, top);
    need(r0 + m1);
    gemm(p, rb, mb, r0, m1, off, n1, false);     // A22[m1:, 0:m1] -= A21_bot A21_top^T
    need(off + nb);
    syrk(rb, mb, off, n1, p);                    // A22[m1:, m1:] (lower) -= A21_bot A21_bot^T
    cudaEvent_t done = record(ss);
    s = main_s;
    potrf(off + n1, n2, depth + 1, done);
  }
};

hrp_status cuda_status(hrp_handle* h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HRP_OK;
  if (e == cudaErrorNotSupported) return set_err(h, HRP_ERR_UNSUPPORTED, "%s: precision not supported by this library", where);
  return set_err(h, HRP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

void collect_timing(hrp_handle* h, const Fact& f) {
  for (int c = 0; c < kNumClasses; ++c) h->cls_ms[c] = h->cls_launches[c] = h->cls_flops[c] = 0.0;
  h->timeline.clear();
  for (const auto& r : f.recs) {
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, h->events[f.recs[0].ev], h->events[r.ev]) == cudaSuccess &&
        cudaEventElapsedTime(&t1, h->events[f.recs[0].ev], h->events[r.ev + 1]) == cudaSuccess) {
      h->timeline.push_back(r.cls);
      h->timeline.push_back(r.sidx);
      h->timeline.push_back(t0);
      h->timeline.push_back(t1);
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->events[r.ev], h->events[r.ev + 1]) == cudaSuccess) h->cls_ms[r.cls] += ms;
    h->cls_launches[r.cls] += 1.0;
    h->cls_flops[r.cls] += r.flops;
  }
  cudaGetLastError();   // a failed elapsed-time query must not leak into the next launch check
}

// The lookahead streams of the handle: [0] with the highest priority (the critical path),
// [1..] side streams by recursion depth, deeper ones at higher priority than shallower ones
// (their work is needed sooner), all below [0].
hrp_status lookahead_streams(hrp_handle* h) {
  constexpr int kStreams = 12;
  if ((int)h->lstreams.size() >= kStreams) return HRP_OK;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  while ((int)h->lstreams.size() < kStreams) {
    const int i = (int)h->lstreams.size();
    // numerically lower is higher priority: [0] = greatest; side depth d from least upwards
    int prio = greatest;
    if (i > 0) prio = std::max(greatest + 1, least - (i - 1) / 2);
    if (greatest == least) prio = least;
    cudaStream_t st;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess)
      return set_err(h, HRP_ERR_CUDA, "lookahead stream");
    h->lstreams.push_back(st);
  }
  return HRP_OK;
}

hrp_status potrf_enqueue(hrp_handle* h, const hrp_tree* t, int n, double* dA, int lda, int* d_info, cudaStream_t s,
                         const std::vector<cudaEvent_t>* col_ev = nullptr) {
  hrp_status st;
  const bool has8 = tree_has(t, HRP_F8E4M3);
  if (has8) {
    // E4M3 tiles live on the global 128 x 128 grid: every node must split on it
    bool pow2 = n >= 128 && (n % 128) == 0 && (((n / 128) & (n / 128 - 1)) == 0);
    int tl = t->trsm_leaf ? t->trsm_leaf : t->leaf;
    if (n > 0 && (!pow2 || t->leaf != 128 || tl != 128))
      return set_err(h, HRP_ERR_UNSUPPORTED, "an F8 level needs n = 128 * 2^k and leaf = trsm_leaf = 128");
  }
  Fact f{};
  f.h = h;
  f.t = t;
  f.A = dA;
  f.lda = lda;
  f.n = n;
  f.info = d_info;
  f.s = s;
  f.tc = tc_gemm_supported();
  f.shadow = nullptr;
  f.shadow8 = nullptr;
  f.tile_exp = nullptr;
  f.lds = (n + 63) / 64 * 64;
  f.w32 = nullptr;
  if (tree_has(t, HRP_F16)) {
    if ((st = ensure(h, &h->shadow, &h->shadow_cap, (size_t)n * f.lds)) != HRP_OK) return st;
    f.shadow = h->shadow;
  }
  if (has8 && n > 0 && h->f8_gemm == 0 && f.tc) {
    if ((st = ensure(h, &h->bytes8, &h->bytes8_cap, (size_t)n * f.lds)) != HRP_OK) return st;
    const size_t nt = (size_t)(n / 128);
    if ((st = ensure(h, &h->tile_exp, &h->tile_exp_cap, nt * nt)) != HRP_OK) return st;
    f.bytes8 = h->bytes8;
    f.tile_exp = h->tile_exp;
  } else if (has8 && n > 0) {
    if ((st = ensure(h, &h->shadow8, &h->shadow8_cap, (size_t)n * f.lds)) != HRP_OK) return st;
    const size_t nt = (size_t)(n / 128);
    if ((st = ensure(h, &h->tile_exp, &h->tile_exp_cap, nt * nt)) != HRP_OK) return st;
    f.shadow8 = h->shadow8;
    f.tile_exp = h->tile_exp;
  }
  if (tree_has(t, HRP_F32) || tree_has(t, HRP_F16) || has8) {
    if ((st = ensure(h, &h->w32, &h->w32_cap, (size_t)n * 128 + 128 * 128)) != HRP_OK) return st;
    f.w32 = h->w32;
  }
  f.shadow32 = nullptr;
  f.ld32 = n;
  if (h->fp32_split && f.tc && tree_has(t, HRP_F32) && n > 0) {
    f.ldh = f.lds;
    if ((st = ensure(h, &h->split32, &h->split32_cap, 2 * (size_t)n * f.ldh)) != HRP_OK) return st;
    f.h32 = h->split32;
    f.l32 = h->split32 + (size_t)n * f.ldh;
  }
  if (tree_has(t, HRP_F32) && n > 0) {
    if ((st = ensure(h, &h->shadow32, &h->shadow32_cap, (size_t)n * n)) != HRP_OK) return st;
    f.shadow32 = h->shadow32;
  }
  // lookahead needs a node whose A22 splits again (n2 > leaf)
  f.la = h->lookahead && n > 2 * t->leaf + 128;
  if (f.la && (st = lookahead_streams(h)) != HRP_OK) return st;
  if (f.la) {
    f.side = &h->lstreams;                 // [0] is the critical stream, [d] the side stream of depth d
    f.main_s = h->lstreams[0];
    f.side_ctas = std::max(1, device_sm_count() - 16);
    f.wait(f.main_s, f.record(s));          // fork from the caller's stream
    f.s = f.main_s;
  } else {
    f.main_s = s;
  }
  const bool scaled = h->scaling == 1 && n > 0;
  if (scaled && (st = ensure(h, &h->scale_exp, &h->scale_exp_cap, (size_t)n)) != HRP_OK) return st;
  f.col_ev = col_ev;
  f.begin(CLS_OTHER, 0.0);
  f.chk(launch_fill_int(d_info, INT_MAX, 1, f.s));
  if (scaled) f.need(n);                      // the scaling reads the whole matrix
  if (scaled) {                               // A_hat = D^-1 A D^-1, D = diag(2^e_i)
    f.begin(CLS_OTHER, 0.0);
    f.chk(launch_diag_scale(dA, lda, n, h->scale_exp, false, f.s));
  }
  f.potrf(0, n, 0);
  if (scaled) {                               // L = D L_hat
    f.begin(CLS_OTHER, 0.0);
    f.chk(launch_diag_scale(dA, lda, n, h->scale_exp, true, f.s));
  }
  f.need(n);                                  // every copy is done when the call's work is
  f.begin(CLS_OTHER, 0.0);
  f.chk(launch_finalize_info(d_info, f.s));
  if (f.la) {
    f.wait(s, f.record(f.main_s));          // join: every side stream was joined into it
    f.s = s;
  }
  launch_ctx() = LaunchCtx{};
  h->launches = f.launches;
  if (h->timing && f.err == cudaSuccess) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(h, e, "hrp_potrf timing");
    collect_timing(h, f);
  }
  return cuda_status(h, f.err, "hrp_potrf");
}

hrp_status check_dev_err(hrp_handle* h, cudaStream_t s) {
  unsigned e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_status(h, ce, "device status");
  if (e & DEV_ERR_TIMEOUT) {
    cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), s);
    return set_err(h, HRP_ERR_TIMEOUT, "a bounded device wait expired");
  }
  if (e & DEV_ERR_RANGE) {
    cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), s);
    return set_err(h, HRP_ERR_RANGE, "an E4M3 tile fell outside the exact FP16 storage window");
  }
  if (e & DEV_ERR_RANGE16) {
    cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), s);
    return set_err(h, HRP_ERR_RANGE,
                   "an FP16 operand exceeds 65504: the Sec. 3.4 scale alpha would be > 1 (use an F32 tree)");
  }
  return HRP_OK;
}

}  // namespace

// The learned policy's tree for the system (n, dA, lda): its features, the network's choice
// (index 0, the fallback tree, when no policy is loaded), with F8 levels taken in FP16 when
// n is not 128 * 2^k or when no_f8 (the batched calls do not run F8 levels).  Synchronous.
hrp_status policy_choose(hrp_handle* h, int n, const double* dA, int lda, bool no_f8, hrp_tree* out, int* idx,
                         void* stream) {
  int k = 0;
  if (h->policy_set && n >= h->policy_min_n) {
    float feat[12];
    hrp_status fs = hrp_policy_features(h, n, dA, lda, kPolicyLanczosSteps, feat, stream);
    if (fs != HRP_OK) return fs;
    if ((fs = hrp_policy_predict(h, feat, nullptr, &k)) != HRP_OK) return fs;
  }
  hrp_policy_tree(k, out);
  const bool pow2 = n >= 128 && n % 128 == 0 && (((n / 128) & (n / 128 - 1)) == 0);
  if (no_f8 || !pow2)
    for (int i = 0; i < out->depth; ++i)
      if (out->level[i] == HRP_F8E4M3) out->level[i] = HRP_F16;
  if (idx) *idx = k;
  return HRP_OK;
}

}  // namespace hrp

using namespace hrp;

extern "C" {

const char* hrp_status_string(hrp_status s) {
  switch (s) {
    case HRP_OK: return "HRP_OK";
    case HRP_ERR_INVALID_ARG: return "HRP_ERR_INVALID_ARG";
    case HRP_ERR_NOT_SPD: return "HRP_ERR_NOT_SPD";
    case HRP_ERR_NO_CONVERGENCE: return "HRP_ERR_NO_CONVERGENCE";
    case HRP_ERR_ALLOC: return "HRP_ERR_ALLOC";
    case HRP_ERR_CUDA: return "HRP_ERR_CUDA";
    case HRP_ERR_TIMEOUT: return "HRP_ERR_TIMEOUT";
    case HRP_ERR_UNSUPPORTED: return "HRP_ERR_UNSUPPORTED";
    case HRP_ERR_RANGE: return "HRP_ERR_RANGE";
  }
  return "HRP_ERR_UNKNOWN";
}

hrp_status hrp_create(hrp_handle** out, int device) {
  if (!out) return HRP_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return HRP_ERR_CUDA;
  if (device < 0 || device >= count) return HRP_ERR_INVALID_ARG;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return HRP_ERR_CUDA;
  hrp_handle* h = new (std::nothrow) hrp_handle_s();
  if (!h) return HRP_ERR_ALLOC;
  h->device = device;
  bool ok = cudaMalloc(&h->d_info, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_err, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&h->d_ticket, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_probe, 4 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&h->d_norms, sizeof(double) * 128) == cudaSuccess &&
            cudaMallocHost(&h->h_norms, sizeof(double) * 128) == cudaSuccess;
  if (!ok || cudaMemset(h->d_err, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->d_probe, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    hrp_destroy(h);
    return HRP_ERR_ALLOC;
  }
  *out = h;
  return HRP_OK;
}

hrp_status hrp_destroy(hrp_handle* h) {
  if (!h) return HRP_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->d_info);
  cudaFree(h->d_err);
  cudaFree(h->d_ticket);
  cudaFree(h->d_probe);
  cudaFree(h->shadow);
  cudaFree(h->w32);
  cudaFree(h->shadow8);
  cudaFree(h->bytes8);
  cudaFree(h->shadow32);
  cudaFree(h->tile_exp);
  cudaFree(h->fact);
  cudaFree(h->work);
  cudaFree(h->d_norms);
  cudaFree(h->pwork);
  if (h->h_norms) cudaFreeHost(h->h_norms);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  for (cudaEvent_t e : h->bevents) cudaEventDestroy(e);
  for (cudaStream_t st : h->bstreams) cudaStreamDestroy(st);
  for (cudaStream_t st : h->lstreams) cudaStreamDestroy(st);
  for (cudaEvent_t e : h->levents) cudaEventDestroy(e);
  for (cudaEvent_t e : h->col_events) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  cudaFree(h->bwork);
  cudaFree(h->fwork);
  cudaFree(h->kwork);
  cudaFree(h->scale_exp);
  cudaFree(h->split32);
  for (auto& pl : h->plans) {
    cudaFree(pl.ops);
    cudaFree(pl.sys);
    cudaFree(pl.ticket);
    cudaFree(pl.shadows);
  }
  cudaFree(h->policy);
  cudaFree(h->pio);
  delete h;
  return HRP_OK;
}

int hrp_last_arg(const hrp_handle* h) { return h ? h->last_arg : 0; }
const char* hrp_last_error(const hrp_handle* h) { return h ? h->last_err : ""; }

hrp_status hrp_tree_parse(const char* spec, int leaf, hrp_tree* out) {
  if (!spec || !out) return HRP_ERR_INVALID_ARG;
  hrp_tree t;
  memset(&t, 0, sizeof(t));
  t.leaf = leaf;
  t.scale_block = 128;
  const char* p = spec;
  while (*p == ' ') ++p;
  if (*p != '[') return HRP_ERR_INVALID_ARG;
  ++p;
  bool inner_part = false;
  while (true) {
    while (*p == ' ' || *p == ',') ++p;
    if (*p == ']') { ++p; break; }
    if (*p == '|') { inner_part = true; ++p; continue; }
    int prec;
    if (!strncmp(p, "F64", 3)) { prec = HRP_F64; p += 3; }
    else if (!strncmp(p, "F32", 3)) { prec = HRP_F32; p += 3; }
    else if (!strncmp(p, "F16", 3)) { prec = HRP_F16; p += 3; }
    else if (!strncmp(p, "F8E4M3", 6)) { prec = HRP_F8E4M3; p += 6; }
    else if (!strncmp(p, "E4M3", 4)) { prec = HRP_F8E4M3; p += 4; }
    else if (!strncmp(p, "F8", 2)) { prec = HRP_F8E4M3; p += 2; }
    else return HRP_ERR_INVALID_ARG;
    if (inner_part) {
      while (*p == ' ') ++p;
      if (*p != '@' || (prec != HRP_F64 && prec != HRP_F32)) return HRP_ERR_INVALID_ARG;
      ++p;
      char* endp = nullptr;
      long v = strtol(p, &endp, 10);
      if (endp == p || v <= 0) return HRP_ERR_INVALID_ARG;
      p = endp;
      t.inner = prec;
      t.inner_size = (int)v;
      while (*p == ' ') ++p;
      if (*p != ']') return HRP_ERR_INVALID_ARG;
      continue;
    }
    if (t.depth >= HRP_MAX_DEPTH) return HRP_ERR_INVALID_ARG;
    t.level[t.depth++] = prec;
  }
  while (*p == ' ') ++p;
  if (*p != '\0' || t.depth == 0) return HRP_ERR_INVALID_ARG;
  *out = t;
  return HRP_OK;
}

int hrp_tree_format(const hrp_tree* t, char* buf, size_t len) {
  static const char* names[] = {"F64", "F32", "F16", "F8"};
  std::string s = "[";
  for (int i = 0; t && i < t->depth; ++i) {
    if (i) s += ",";
    int l = t->level[i];
    s += (l >= 0 && l <= 3) ? names[l] : "?";
  }
  if (t && t->inner_size > 0) {
    s += "|";
    s += (t->inner >= 0 && t->inner <= 3) ? names[t->inner] : "?";
    s += "@" + std::to_string(t->inner_size);
  }
  s += "]";
  if (buf && len) {
    strncpy(buf, s.c_str(), len - 1);
    buf[len - 1] = '\0';
  }
  return (int)s.size();
}

hrp_status hrp_potrf_async(hrp_handle* h, const hrp_tree* tree, int n, double* dA, int lda, int* d_info, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (n < 0) return bad_arg(h, 3, "n < 0");
  if (n > 0 && !dA) return bad_arg(h, 4, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 5, "lda < max(1, n)");
  if (!d_info) return bad_arg(h, 6, "d_info is NULL");
  cudaSetDevice(h->device);
  return potrf_enqueue(h, tree, n, dA, lda, d_info, static_cast<cudaStream_t>(stream));
}

hrp_status hrp_potrf_host(hrp_handle* h, const hrp_tree* tree, int n, const double* hA, int ldha, double* dA, int lda,
                          int* d_info, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (n < 0) return bad_arg(h, 3, "n < 0");
  if (n > 0 && !hA) return bad_arg(h, 4, "hA is NULL");
  if (ldha < (n > 1 ? n : 1)) return bad_arg(h, 5, "ldha < max(1, n)");
  if (n > 0 && !dA) return bad_arg(h, 6, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 7, "lda < max(1, n)");
  if (!d_info) return bad_arg(h, 8, "d_info is NULL");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr int kBlk = 128;                 // Fact::kColBlock
  const int nblk = (n + kBlk - 1) / kBlk;
  if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return set_err(h, HRP_ERR_CUDA, "hrp_potrf_host: copy stream");
  while ((int)h->col_events.size() < nblk + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return set_err(h, HRP_ERR_CUDA, "hrp_potrf_host: events");
    h->col_events.push_back(e);
  }
  // the copies start after the work queued on the caller's stream before this call (it may
  // still use dA); block b carries rows [128 b, n) of columns [128 b, 128 b + 128)
  cudaEvent_t fork = h->col_events[nblk];
  cudaError_t e = cudaEventRecord(fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, fork, 0);
  for (int b = 0; b < nblk && e == cudaSuccess; ++b) {
    const int c0 = b * kBlk, nc = std::min(kBlk, n - c0);
    e = cudaMemcpy2DAsync(dA + (size_t)c0 * lda + c0, (size_t)lda * sizeof(double), hA + (size_t)c0 * ldha + c0,
                          (size_t)ldha * sizeof(double), (size_t)(n - c0) * sizeof(double), nc, cudaMemcpyHostToDevice,
                          h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->col_events[b], h->copy_stream);
  }
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_potrf_host: copies");
  const std::vector<cudaEvent_t> ev(h->col_events.begin(), h->col_events.begin() + nblk);
  st = potrf_enqueue(h, tree, n, dA, lda, d_info, s, &ev);
  // on an error the factorization may have enqueued nothing that waits for the copies: the
  // caller's stream still does, so synchronizing it covers every use of hA and dA
  if (st != HRP_OK && nblk > 0) cudaStreamWaitEvent(s, ev.back(), 0);
  return st;
}

hrp_status hrp_potrf(hrp_handle* h, const hrp_tree* tree, int n, double* dA, int lda, int* info, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (n < 0) return bad_arg(h, 3, "n < 0");
  if (n > 0 && !dA) return bad_arg(h, 4, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 5, "lda < max(1, n)");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = potrf_enqueue(h, tree, n, dA, lda, h->d_info, s);
  if (st != HRP_OK) return st;
  int hinfo = 0;
  cudaError_t e = cudaMemcpyAsync(&hinfo, h->d_info, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_potrf");
  if ((st = check_dev_err(h, s)) != HRP_OK) return st;
  if (info) *info = hinfo;
  if (hinfo) return set_err(h, HRP_ERR_NOT_SPD, "leading minor of order %d is not positive definite", hinfo);
  return HRP_OK;
}


static hrp_status potrs_impl(hrp_handle* h, int n, int nrhs, const double* dL, int ldl, double* dB, int ldb,
                             bool fp32, cudaStream_t s) {
  hrp_status st;
  if ((st = ensure(h, &h->pwork, &h->pwork_cap, potrs_workspace_bytes(n))) != HRP_OK) return st;
  cudaError_t e = launch_potrs(dL, ldl, dB, ldb, n, nrhs, fp32, h->pwork, h->d_ticket, h->d_err, s, h->wait_ns);
  h->launches += 1 + potrs_sweeps(nrhs);
  return cuda_status(h, e, "hrp_potrs");
}

hrp_status hrp_potrs(hrp_handle* h, int n, int nrhs, const double* dL, int ldl, double* dB, int ldb, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (n < 0) return bad_arg(h, 2, "n < 0");
  if (nrhs < 0) return bad_arg(h, 3, "nrhs < 0");
  if (n > 0 && !dL) return bad_arg(h, 4, "dL is NULL");
  if (ldl < (n > 1 ? n : 1)) return bad_arg(h, 5, "ldl < max(1, n)");
  if (n > 0 && nrhs > 0 && !dB) return bad_arg(h, 6, "dB is NULL");
  if (ldb < (n > 1 ? n : 1)) return bad_arg(h, 7, "ldb < max(1, n)");
  cudaSetDevice(h->device);
  h->launches = 0;
  return potrs_impl(h, n, nrhs, dL, ldl, dB, ldb, false, static_cast<cudaStream_t>(stream));
}

// One GMRES-IR correction for one right-hand side (Carson and Higham): x += d, where d solves
// A d = r by GMRES on M^{-1} A d = M^{-1} r from d = 0 with M = L L^T the factor in h->fact,
// applied by the FP64 POTRS; classical Gram-Schmidt twice, Givens rotations on the host,
// stop at |g_k| <= gmres_tol * beta or after gmres_restart steps.  Matrix-vector products
// in FP64 from A's lower triangle.  Synchronous (a few 8-byte reads per step).
static hrp_status gmres_correction(hrp_handle* h, const double* dA, int lda, int n, const double* r, double* x,
                                   cudaStream_t s) {
  const int m = h->gmres_restart;
  hrp_status st = ensure(h, &h->kwork, &h->kwork_cap, (size_t)(m + 1) * n + 2 * (size_t)n + 2 * (m + 1));
  if (st != HRP_OK) return st;
  double* V = h->kwork;
  double* w = V + (size_t)(m + 1) * n;
  double* zero = w + n;
  double* hd = zero + n;
  double* hh = h->h_norms;                       // pinned host mirror (128 doubles)
  cudaError_t e = cudaMemsetAsync(zero, 0, sizeof(double) * n, s);
  auto sync_read = [&](int cnt) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(hh, hd, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  };
  // v0 = M^{-1} r / beta
  if (e == cudaSuccess) e = cudaMemcpyAsync(V, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_status(h, e, "gmres");
  if ((st = potrs_impl(h, n, 1, h->fact, n, V, n, false, s)) != HRP_OK) return st;
  e = launch_multi_dot(V, n, 1, V, n, hd, s);
  sync_read(1);
  if (e != cudaSuccess) return cuda_status(h, e, "gmres");
  const double beta = sqrt(hh[0]);
  if (!(beta > 0.0) || !std::isfinite(beta)) return HRP_OK;   // nothing to correct (or NaN: left to the caller)
  e = launch_scale(V, V, 1.0 / beta, n, false, s);
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)j * (m + 1) + i]; };
  g[0] = beta;
  int k = 0;
  while (k < m && e == cudaSuccess) {
    double* vk = V + (size_t)k * n;
    // w = M^{-1} A v_k (the residual kernel gives -A v_k from a zero right-hand side)
    e = launch_residual(dA, lda, vk, n, zero, n, w, n, n, 1, s);
    if (e == cudaSuccess) e = launch_scale(w, w, -1.0, n, false, s);
    if (e != cudaSuccess) break;
    if ((st = potrs_impl(h, n, 1, h->fact, n, w, n, false, s)) != HRP_OK) return st;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      e = launch_multi_dot(V, n, k + 1, w, n, hd, s);
      if (e == cudaSuccess) e = launch_gemv_sub(w, V, n, k + 1, hd, n, s);
      sync_read(k + 1);
      for (int i = 0; i <= k; ++i) Hat(i, k) += hh[i];
    }
    if (e == cudaSuccess) e = launch_multi_dot(w, n, 1, w, n, hd, s);
    sync_read(1);
    if (e != cudaSuccess) break;
    const double hn = sqrt(hh[0]);
    Hat(k + 1, k) = hn;
    for (int i = 0; i < k; ++i) {                 // earlier rotations on the new column
      const double a = Hat(i, k), b = Hat(i + 1, k);
      Hat(i, k) = cs[i] * a + sn[i] * b;
      Hat(i + 1, k) = -sn[i] * a + cs[i] * b;
    }
    const double a = Hat(k, k), b = Hat(k + 1, k), rho = std::hypot(a, b);
    cs[k] = rho > 0 ? a / rho : 1.0;
    sn[k] = rho > 0 ? b / rho : 0.0;
    Hat(k, k) = rho;
    Hat(k + 1, k) = 0.0;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    if (hn > 0.0) e = launch_scale(V + (size_t)(k + 1) * n, w, 1.0 / hn, n, false, s);
    ++k;
    if (!(fabs(g[k]) > h->gmres_tol * beta) || !(hn > 0.0)) break;
  }
  if (e != cudaSuccess) return cuda_status(h, e, "gmres");
  // y from the rotated (upper triangular) H, then x += V y
  std::vector<double> y(k, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int j = i + 1; j < k; ++j) t -= Hat(i, j) * y[j];
    y[i] = t / Hat(i, i);
  }
  for (int i = 0; i < k; ++i) hh[i] = -y[i];
  e = cudaMemcpyAsync(hd, hh, sizeof(double) * k, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_gemv_sub(x, V, n, k, hd, n, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);        // hh is reused by the caller
  h->inner_steps += k;
  return cuda_status(h, e, "gmres");
}

hrp_status hrp_posv(hrp_handle* h, const hrp_tree* tree, int n, int nrhs, const double* dA, int lda, const double* dB,
                    int ldb, double* dX, int ldx, int max_iter, double tol, int* iters, double* resid, int* info,
                    int* used_fallback, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_tree chosen;
  h->last_choice = -1;
  if (!tree && n > 0 && dA && lda >= n) {
    // no tree given: the learned policy picks one (the fallback tree if none is loaded)
    int idx = 0;
    hrp_status fs = policy_choose(h, n, dA, lda, false, &chosen, &idx, stream);
    if (fs != HRP_OK) return fs;
    h->last_choice = idx;
    tree = &chosen;
  }
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (n < 0) return bad_arg(h, 3, "n < 0");
  if (nrhs < 0 || nrhs > 64) return bad_arg(h, 4, "nrhs must be in [0, 64]");
  if (n > 0 && !dA) return bad_arg(h, 5, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 6, "lda < max(1, n)");
  if (n > 0 && nrhs > 0 && !dB) return bad_arg(h, 7, "dB is NULL");
  if (ldb < (n > 1 ? n : 1)) return bad_arg(h, 8, "ldb < max(1, n)");
  if (n > 0 && nrhs > 0 && !dX) return bad_arg(h, 9, "dX is NULL");
  if (ldx < (n > 1 ? n : 1)) return bad_arg(h, 10, "ldx < max(1, n)");
  if (max_iter < 0) return bad_arg(h, 11, "max_iter < 0");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (iters) *iters = 0;
  if (resid) *resid = 0.0;
  if (info) *info = 0;
  if (used_fallback) *used_fallback = 0;
  h->inner_steps = 0;
  if (n == 0 || nrhs == 0) return HRP_OK;
  if ((st = ensure(h, &h->fact, &h->fact_cap, (size_t)n * n)) != HRP_OK) return st;
  if ((st = ensure(h, &h->work, &h->work_cap, (size_t)n * nrhs)) != HRP_OK) return st;
  if (!tree) return set_err(h, HRP_ERR_INVALID_ARG, "no tree");
  cudaError_t e;
  hrp_tree fallback;
  hrp_tree_parse("[F32|F64@128]", 128, &fallback);
  const hrp_tree* use = tree;
  int hinfo = 0, it = 0;
  double worst = 0.0;
  // attempt 0 uses the requested tree; attempt 1 (if needed) the conservative fallback:
  // taken when the factorization fails (info > 0) or refinement diverges or stalls
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      use = &fallback;
      if (used_fallback) *used_fallback = 1;
    }
    if ((e = launch_copy_lower(h->fact, n, dA, lda, n, s)) != cudaSuccess) return cuda_status(h, e, "hrp_posv");
    if ((st = potrf_enqueue(h, use, n, h->fact, n, h->d_info, s)) != HRP_OK) return st;
    e = cudaMemcpyAsync(&hinfo, h->d_info, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(h, e, "hrp_posv");
    // an operand outside the FP16 (or E4M3 storage) range: the tree cannot factor this
    // matrix without alpha > 1, so the fallback tree takes over
    if ((st = check_dev_err(h, s)) == HRP_ERR_RANGE && attempt == 0) continue;
    if (st != HRP_OK) return st;
    if (hinfo) continue;
    // X0 = POTRS(B) in FP32
    if ((e = launch_copy_matrix(dX, ldx, dB, ldb, n, nrhs, s)) != cudaSuccess) return cuda_status(h, e, "hrp_posv");
    if ((st = potrs_impl(h, n, nrhs, h->fact, n, dX, ldx, true, s)) != HRP_OK) return st;
    it = 0;
    double prev = 1e300;
    bool diverged = false;
    while (true) {
      if ((e = launch_residual(dA, lda, dX, ldx, dB, ldb, h->work, n, n, nrhs, s)) != cudaSuccess)
        return cuda_status(h, e, "hrp_posv residual");
      if ((e = launch_col_norms2(h->work, n, dB, ldb, n, nrhs, h->d_norms, s)) != cudaSuccess)
        return cuda_status(h, e, "hrp_posv norms");
      e = cudaMemcpyAsync(h->h_norms, h->d_norms, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_status(h, e, "hrp_posv");
      worst = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        double rb = h->h_norms[nrhs + c] > 0 ? sqrt(h->h_norms[c] / h->h_norms[nrhs + c]) : sqrt(h->h_norms[c]);
        if (!(rb <= worst)) worst = rb;   // NaN propagates
      }
      // a solve whose bounded wait expired leaves NaN rows: report it, do not refine on
      if (worst != worst && (st = check_dev_err(h, s)) != HRP_OK) return st;
      if (worst <= tol || it >= max_iter) break;
      if (!(worst < prev)) { diverged = true; break; }   // no decrease: this factor will not get there
      prev = worst;
      if (h->refine_mode == 1) {
        for (int c = 0; c < nrhs; ++c)
          if ((st = gmres_correction(h, dA, lda, n, h->work + (size_t)c * n, dX + (size_t)c * ldx, s)) != HRP_OK)
            return st;
      } else {
        if ((st = potrs_impl(h, n, nrhs, h->fact, n, h->work, n, true, s)) != HRP_OK) return st;
        if ((e = launch_axpy_matrix(dX, ldx, h->work, n, n, nrhs, s)) != cudaSuccess)
          return cuda_status(h, e, "hrp_posv");
      }
      ++it;
    }
    if (worst <= tol || (!diverged && attempt == 1)) break;
    if (attempt == 1) break;
  }
  if (info) *info = hinfo;
  if (hinfo) return set_err(h, HRP_ERR_NOT_SPD, "factorization failed at column %d (fallback tree too)", hinfo);
  if (iters) *iters = it;
  if (resid) *resid = worst;
  if ((st = check_dev_err(h, s)) != HRP_OK) return st;
  if (!(worst <= tol)) return set_err(h, HRP_ERR_NO_CONVERGENCE, "residual %.3e after %d corrections", worst, it);
  return HRP_OK;
}

hrp_status hrp_backward_error(hrp_handle* h, int n, const double* dA, int lda, const double* dL, int ldl, double* out,
                              void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (n < 0) return bad_arg(h, 2, "n < 0");
  if (n > 0 && !dA) return bad_arg(h, 3, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 4, "lda < max(1, n)");
  if (n > 0 && !dL) return bad_arg(h, 5, "dL is NULL");
  if (ldl < (n > 1 ? n : 1)) return bad_arg(h, 6, "ldl < max(1, n)");
  if (!out) return bad_arg(h, 7, "out is NULL");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *out = 0.0;
  if (n == 0) return HRP_OK;
  cudaError_t e = cudaMemsetAsync(h->d_norms, 0, 2 * sizeof(double), s);
  if (e == cudaSuccess) e = launch_backward_error(dA, lda, dL, ldl, n, h->d_norms, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_norms, h->d_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_backward_error");
  *out = h->h_norms[1] > 0 ? sqrt(h->h_norms[0] / h->h_norms[1]) : sqrt(h->h_norms[0]);
  return HRP_OK;
}

int hrp_autotune_candidates(const hrp_tree* tree, hrp_tree* out, int cap) {
  if (!tree || cap < 0 || (cap > 0 && !out)) return -1;
  if (validate_tree(nullptr, tree, 1) != HRP_OK) return -1;
  std::vector<hrp_tree> c;
  auto add = [&](int leaf, int tl) {
    hrp_tree t = *tree;
    t.leaf = leaf;
    t.trsm_leaf = (tl == leaf) ? 0 : tl;
    for (const auto& u : c)
      if (u.leaf == t.leaf && (u.trsm_leaf ? u.trsm_leaf : u.leaf) == (t.trsm_leaf ? t.trsm_leaf : t.leaf) &&
          u.tile_occupancy == t.tile_occupancy)
        return;
    if (validate_tree(nullptr, &t, 1) == HRP_OK) c.push_back(t);
  };
  add(tree->leaf, tree->trsm_leaf ? tree->trsm_leaf : tree->leaf);   // the given tree first
  if (!tree_has(tree, HRP_F8E4M3)) {                                 // F8 trees: 128 / 128 only
    for (int leaf : {128, 64, 32}) {
      add(leaf, leaf);
      add(leaf, leaf / 2);
    }
  }
  // the tensor-core tile rule: the same cut-offs with 2 and 4 tiles per SM
  if (tree_has(tree, HRP_F16) || tree_has(tree, HRP_F8E4M3)) {
    const size_t base = c.size();
    for (int occ : {2, 4})
      for (size_t i = 0; i < base; ++i) {
        hrp_tree t = c[i];
        if ((t.tile_occupancy ? t.tile_occupancy : 1) == occ) continue;
        t.tile_occupancy = occ;
        bool dup = false;
        for (const auto& u : c)
          dup |= u.leaf == t.leaf && u.trsm_leaf == t.trsm_leaf && u.tile_occupancy == t.tile_occupancy;
        if (!dup && validate_tree(nullptr, &t, 1) == HRP_OK) c.push_back(t);
      }
  }
  for (int i = 0; i < (int)c.size() && i < cap; ++i) out[i] = c[i];
  return (int)c.size();
}

hrp_status hrp_autotune(hrp_handle* h, const hrp_tree* tree, int n, int reps, int flags, hrp_tree* out, float* ms,
                        void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (n < 1 || n > 65535) return bad_arg(h, 3, "n must be in [1, 65535]");
  if (reps < 1) return bad_arg(h, 4, "reps < 1");
  if (!out) return bad_arg(h, 6, "out is NULL");
  const std::string key = tune_key(tree);
  if (!(flags & 1)) {
    auto it = h->tune_cache.find(key);
    if (it != h->tune_cache.end()) {
      auto jt = it->second.find(n);
      if (jt != it->second.end()) {
        *out = jt->second.first;
        if (ms) *ms = jt->second.second;
        return HRP_OK;
      }
    }
  }
  hrp_tree cand[32];
  const int nc = std::min(hrp_autotune_candidates(tree, cand, 32), 32);
  if (nc < 1) return set_err(h, HRP_ERR_INVALID_ARG, "no valid candidate tree");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *base = nullptr, *work = nullptr;
  const size_t bytes = (size_t)n * n * sizeof(double);
  if (cudaMalloc(&base, bytes) != cudaSuccess || cudaMalloc(&work, bytes) != cudaSuccess) {
    cudaFree(base);
    cudaGetLastError();
    return set_err(h, HRP_ERR_ALLOC, "autotune: cudaMalloc of 2 x %zu bytes failed", bytes);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto fail = [&](hrp_status x) {
    cudaFree(base);
    cudaFree(work);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return x;
  };
  cudaError_t ce = launch_fill_spd_uniform(base, n, n, 0x2601008082ull + (unsigned long long)n, s);
  if (ce != cudaSuccess) return fail(cuda_status(h, ce, "autotune generator"));
  int best = -1;
  float best_ms = 0.f;
  double be_ref = -1.0;
  for (int c = 0; c < nc; ++c) {
    std::vector<float> t;
    int info = 0;
    for (int r = 0; r <= reps; ++r) {                     // r = 0: warm-up (workspace, caches)
      ce = cudaMemcpyAsync(work, base, bytes, cudaMemcpyDeviceToDevice, s);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
      if (ce != cudaSuccess) return fail(cuda_status(h, ce, "autotune"));
      st = potrf_enqueue(h, &cand[c], n, work, n, h->d_info, s);
      if (st != HRP_OK) break;
      ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(&info, h->d_info, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) return fail(cuda_status(h, ce, "autotune"));
      if ((st = check_dev_err(h, s)) != HRP_OK || info != 0) break;
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r > 0) t.push_back(x);
    }
    if (st == HRP_ERR_CUDA) return fail(st);              // the context may be unusable
    if (st != HRP_OK || info != 0 || (int)t.size() != reps) {
      if (c == 0) return fail(st != HRP_OK ? st : set_err(h, HRP_ERR_NOT_SPD, "autotune: the given tree failed"));
      continue;
    }
    double be = 0.0;
    if ((st = hrp_backward_error(h, n, base, n, work, n, &be, stream)) != HRP_OK) return fail(st);
    if (c == 0) be_ref = be;
    else if (!(be <= 4.0 * be_ref + 1e-15)) continue;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    const float med = t[reps / 2];
    if (best < 0 || med < best_ms) {
      best = c;
      best_ms = med;
    }
  }
  fail(HRP_OK);
  *out = cand[best];
  if (ms) *ms = best_ms;
  h->tune_cache[key][n] = {cand[best], best_ms};
  return HRP_OK;
}

hrp_status hrp_autotune_orders(hrp_handle* h, const hrp_tree* tree, int count, const int* orders, int reps,
                               void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (count < 0) return bad_arg(h, 3, "count < 0");
  if (count > 0 && !orders) return bad_arg(h, 4, "orders is NULL");
  for (int i = 0; i < count; ++i) {
    hrp_tree out;
    hrp_status st = hrp_autotune(h, tree, orders[i], reps, 0, &out, nullptr, stream);
    if (st != HRP_OK) return st;
  }
  return HRP_OK;
}

hrp_status hrp_set_timing(hrp_handle* h, int enable) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->timing = enable != 0;
  return HRP_OK;
}

hrp_status hrp_set_refinement(hrp_handle* h, int mode, int restart, double inner_tol) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (mode != 0 && mode != 1) return bad_arg(h, 2, "mode must be 0 (classical) or 1 (GMRES)");
  if (restart < 1 || restart > 60) return bad_arg(h, 3, "restart must be in [1, 60]");
  if (!(inner_tol > 0.0 && inner_tol < 1.0)) return bad_arg(h, 4, "inner_tol must be in (0, 1)");
  h->refine_mode = mode;
  h->gmres_restart = restart;
  h->gmres_tol = inner_tol;
  return HRP_OK;
}

long long hrp_last_inner_iterations(const hrp_handle* h) { return h ? h->inner_steps : 0; }

hrp_status hrp_set_leaf_chain(hrp_handle* h, int mode) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (mode < -1 || mode > 1) return bad_arg(h, 2, "mode must be -1 (by tree), 0 (FP64) or 1 (double-float)");
  h->leaf_chain = mode;
  return HRP_OK;
}

hrp_status hrp_set_f8_gemm(hrp_handle* h, int mode) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (mode != 0 && mode != 1) return bad_arg(h, 2, "mode must be 0 (block-scaled E4M3) or 1 (FP16 storage)");
  h->f8_gemm = mode;
  return HRP_OK;
}

hrp_status hrp_set_fp32_split(hrp_handle* h, int on) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (on != 0 && on != 1) return bad_arg(h, 2, "on must be 0 (SIMT FP32) or 1 (TF32 split on tensor cores)");
  h->fp32_split = on;
  return HRP_OK;
}

hrp_status hrp_set_scaling(hrp_handle* h, int mode) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (mode != 0 && mode != 1) return bad_arg(h, 2, "mode must be 0 (static) or 1 (diagonal scaling)");
  h->scaling = mode;
  return HRP_OK;
}

hrp_status hrp_set_batched_mode(hrp_handle* h, int mode) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (mode != 0 && mode != 1) return bad_arg(h, 2, "mode must be 0 (stream pool) or 1 (persistent)");
  h->batched_mode = mode;
  return HRP_OK;
}

hrp_status hrp_set_lookahead(hrp_handle* h, int enable) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->lookahead = enable != 0;
  return HRP_OK;
}

int hrp_get_timing(hrp_handle* h, double* out, int n) {
  if (!h || !out) return 0;
  int w = 0;
  for (int c = 0; c < kNumClasses && w + 3 <= n; ++c) {
    out[w++] = h->cls_ms[c];
    out[w++] = h->cls_launches[c];
    out[w++] = h->cls_flops[c];
  }
  return w;
}

int hrp_get_timeline(hrp_handle* h, double* out, int n) {
  if (!h || !out) return 0;
  const int w = std::min(n - n % 4, (int)h->timeline.size());
  for (int i = 0; i < w; ++i) out[i] = h->timeline[i];
  return w;
}

long long hrp_last_launch_count(const hrp_handle* h) { return h ? h->launches : 0; }

hrp_status hrp_check(hrp_handle* h, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  return check_dev_err(h, static_cast<cudaStream_t>(stream));
}

hrp_status hrp_set_wait_limit(hrp_handle* h, long long microseconds) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (microseconds < 1 || microseconds > 2000000) return bad_arg(h, 2, "limit must be in [1, 2000000] us");
  h->wait_ns = (unsigned long long)microseconds * 1000ull;
  return HRP_OK;
}

hrp_status hrp_wait_selftest(hrp_handle* h, long long microseconds, double* waited_us, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (microseconds < 1 || microseconds > 2000000) return bad_arg(h, 2, "limit must be in [1, 2000000] us");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  hrp_status st = check_dev_err(h, s);           // report what earlier calls left first
  if (st != HRP_OK) return st;
  // d_probe[0] is the mailbox entry (emptied by the probe); d_probe[1] receives the time waited
  unsigned long long* out = reinterpret_cast<unsigned long long*>(h->d_probe + 1);
  cudaError_t e = launch_wait_probe(h->d_probe, (unsigned long long)microseconds * 1000ull, h->d_err, out, s);
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, out, sizeof(ns), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_wait_selftest");
  if (waited_us) *waited_us = ns * 1e-3;
  return check_dev_err(h, s);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batched factorization and solve: many independent systems of different orders.
// Each system runs the same recursion as hrp_potrf on one stream of a pool forked from
// the caller's stream (systems assigned longest-processing-time first by n^3), with its
// own slice of workspace, and the pool is joined back into the caller's stream.  The
// whole call only enqueues work, so it can be captured into one CUDA graph.
// ---------------------------------------------------------------------------------------
namespace hrp {
namespace {

constexpr int kBatchStreams = 32;

struct SysWork {
  size_t shadow, w32, pinv, ticket, fact, res;   // byte offsets into h->bwork
  int lds;
};

// per-system workspace; nrhs_ir > 0 adds an n x n factor copy and an n x nrhs residual
hrp_status batch_prepare(hrp_handle* h, int batch, const int* n, std::vector<SysWork>& ws, bool need_factor_ws,
                         int nrhs_ir = 0) {
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  ws.resize(batch);
  for (int i = 0; i < batch; ++i) {
    const int ni = n[i];
    SysWork& w = ws[i];
    w.lds = (ni + 63) / 64 * 64;
    w.shadow = need_factor_ws ? take((size_t)ni * w.lds * sizeof(__half)) : 0;
    w.w32 = need_factor_ws ? take(((size_t)ni * 128 + 128 * 128) * sizeof(float)) : 0;
    w.pinv = take(potrs_workspace_bytes(ni));
    w.ticket = take(sizeof(int));
    w.fact = nrhs_ir ? take(sizeof(double) * (size_t)ni * ni) : 0;
    w.res = nrhs_ir ? take(sizeof(double) * (size_t)ni * nrhs_ir + sizeof(double) * 2 * nrhs_ir) : 0;
  }
  unsigned char* old = h->bwork;
  size_t old_cap = h->bwork_cap;
  hrp_status st = ensure(h, &h->bwork, &h->bwork_cap, off);
  if (st != HRP_OK) return st;
  if (h->bwork != old || h->bwork_cap != old_cap) {
    // zero the tickets (and everything else) of the fresh workspace
    if (cudaMemset(h->bwork, 0, h->bwork_cap) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "batch workspace");
  }
  while ((int)h->bstreams.size() < kBatchStreams) {
    cudaStream_t st2;
    if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "stream");
    h->bstreams.push_back(st2);
  }
  while ((int)h->bevents.size() < kBatchStreams + 1) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "event");
    h->bevents.push_back(ev);
  }
  return HRP_OK;
}

// longest processing time first: stream of each system
std::vector<int> lpt_assign(int batch, const int* n, int nstreams) {
  std::vector<int> order(batch), which(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<double> load(nstreams, 0.0);
  for (int i : order) {
    int best = 0;
    for (int k = 1; k < nstreams; ++k)
      if (load[k] < load[best]) best = k;
    which[i] = best;
    load[best] += (double)n[i] * n[i] * n[i];
  }
  return which;
}

hrp_status fork(hrp_handle* h, cudaStream_t s) {
  if (cudaEventRecord(h->bevents[kBatchStreams], s) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "fork");
  for (int k = 0; k < kBatchStreams; ++k)
    if (cudaStreamWaitEvent(h->bstreams[k], h->bevents[kBatchStreams], 0) != cudaSuccess)
      return set_err(h, HRP_ERR_CUDA, "fork");
  return HRP_OK;
}
hrp_status join(hrp_handle* h, cudaStream_t s) {
  for (int k = 0; k < kBatchStreams; ++k) {
    if (cudaEventRecord(h->bevents[k], h->bstreams[k]) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "join");
    if (cudaStreamWaitEvent(s, h->bevents[k], 0) != cudaSuccess) return set_err(h, HRP_ERR_CUDA, "join");
  }
  return HRP_OK;
}

hrp_status check_batch_args(hrp_handle* h, int batch, const int* n, double* const* dA, const int* lda);

// The tree of every system: trees[i], or the learned policy's choice where trees (the
// array) or trees[i] is NULL (F8 levels taken in FP16: the batched calls do not run them).
hrp_status batch_trees(hrp_handle* h, const hrp_tree* const* trees, int batch, const int* n, double* const* dA,
                       const int* lda, std::vector<hrp_tree>& chosen, std::vector<const hrp_tree*>& out,
                       void* stream) {
  chosen.assign(batch, hrp_tree{});
  out.assign(batch, nullptr);
  for (int i = 0; i < batch; ++i) {
    if (trees && trees[i]) {
      chosen[i] = *trees[i];
    } else if (n[i] > 0) {
      hrp_status st = policy_choose(h, n[i], dA[i], lda[i], true, &chosen[i], nullptr, stream);
      if (st != HRP_OK) return st;
    } else {
      hrp_policy_tree(0, &chosen[i]);
    }
    apply_tuned(h, &chosen[i], n[i]);         // cut-offs tuned for this order, if any
    out[i] = &chosen[i];
  }
  return HRP_OK;
}

// One system of a persistent batched launch.
struct PSys {
  const hrp_tree* tree;
  int n;
  double* A;
  int lda;
  const double* src;   // non-null: factor a copy of src's lower triangle into A
  int ldsrc;
  int* info;
};

// Records every system's operations (the recursion of Alg. 1-3 with its tree), orders the
// systems longest first, and enqueues the one persistent launch on the batch's plan (its
// device copy of the lists, uploaded on the first call with this batch).  Capturable once
// the plan exists.
hrp_status enqueue_persistent(hrp_handle* h, const std::vector<PSys>& sys, cudaStream_t s, long long* launches) {
  std::vector<int> order(sys.size());
  for (size_t i = 0; i < sys.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sys[a].n > sys[b].n; });
  std::vector<BatchOp> ops;
  std::vector<BatchSys> bs;
  size_t shadow_bytes = 0;
  for (int i : order) {
    const PSys& q = sys[i];
    if (q.n <= 0) continue;
    Fact f{};
    f.h = h;
    f.t = q.tree;
    f.A = q.A;
    f.lda = q.lda;
    f.n = q.n;
    f.info = q.info;
    f.rec = &ops;
    const int op0 = (int)ops.size();
    f.potrf(0, q.n, 0);
    if (f.err != cudaSuccess) return cuda_status(h, f.err, "batched (persistent)");
    const bool shad = tree_has(q.tree, HRP_F32) || tree_has(q.tree, HRP_F16);
    // shadow offsets (bytes from the plan's shadow block) ride in the pointers until the plan
    // allocates the block: FP32 then FP16, each n x n, 256-byte aligned
    float* s32 = nullptr;
    __half* s16 = nullptr;
    if (shad) {
      s32 = reinterpret_cast<float*>(shadow_bytes + 1);
      shadow_bytes += ((size_t)q.n * q.n * sizeof(float) + 255) / 256 * 256;
      s16 = reinterpret_cast<__half*>(shadow_bytes + 1);
      shadow_bytes += ((size_t)q.n * q.n * sizeof(__half) + 255) / 256 * 256;
    }
    bs.push_back(BatchSys{q.A, q.lda, q.n, op0, (int)ops.size(), q.info, q.src, q.ldsrc, s32, s16});
  }
  // systems of order 0: info = 0
  for (const PSys& q : sys)
    if (q.n <= 0) {
      cudaError_t e = launch_fill_int(q.info, 0, 1, s);
      if (e != cudaSuccess) return cuda_status(h, e, "batched (persistent)");
    }
  if (bs.empty()) return HRP_OK;
  const size_t bytes_ops = ops.size() * sizeof(BatchOp), bytes_sys = bs.size() * sizeof(BatchSys);
  // the key holds the shadow offsets (not yet addresses): the same batch finds its plan
  std::string key(bytes_ops + bytes_sys, '\0');
  memcpy(&key[0], ops.data(), bytes_ops);
  memcpy(&key[bytes_ops], bs.data(), bytes_sys);
  hrp_handle_s::Plan* plan = nullptr;
  for (auto& pl : h->plans)
    if (pl.key == key) plan = &pl;
  if (!plan) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
      return set_err(h, HRP_ERR_INVALID_ARG,
                     "batched (persistent): make one call with this batch before capturing it in a graph");
    hrp_handle_s::Plan pl;
    pl.key = key;
    pl.nsys = (int)bs.size();
    if (cudaMalloc(&pl.ops, bytes_ops) != cudaSuccess || cudaMalloc(&pl.sys, bytes_sys) != cudaSuccess ||
        cudaMalloc(&pl.ticket, sizeof(int)) != cudaSuccess ||
        (shadow_bytes && cudaMalloc(&pl.shadows, shadow_bytes) != cudaSuccess)) {
      cudaFree(pl.ops);
      cudaFree(pl.sys);
      cudaFree(pl.ticket);
      cudaGetLastError();
      return set_err(h, HRP_ERR_ALLOC, "batched (persistent): plan buffers");
    }
    for (auto& b : bs)                    // offsets -> addresses in the plan's shadow block
      if (b.s32) {
        b.s32 = reinterpret_cast<float*>(pl.shadows + (reinterpret_cast<uintptr_t>(b.s32) - 1));
        b.s16 = reinterpret_cast<__half*>(pl.shadows + (reinterpret_cast<uintptr_t>(b.s16) - 1));
      }
    // from pageable memory: the call returns once the bytes are staged, before they are used
    cudaError_t e = cudaMemcpyAsync(pl.ops, ops.data(), bytes_ops, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl.sys, bs.data(), bytes_sys, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaFree(pl.ops);
      cudaFree(pl.sys);
      cudaFree(pl.ticket);
      return cuda_status(h, e, "batched (persistent)");
    }
    h->plans.push_back(std::move(pl));
    plan = &h->plans.back();
  }
  cudaError_t e = launch_batched_interp(plan->ops, plan->sys, plan->nsys, plan->ticket, h->d_err, s);
  if (launches) *launches = 1;
  return cuda_status(h, e, "batched (persistent)");
}

hrp_status check_batch_args(hrp_handle* h, int batch, const int* n, double* const* dA, const int* lda) {
  if (batch < 0) return bad_arg(h, 3, "batch < 0");
  if (batch > 0 && (!n || !dA || !lda)) return bad_arg(h, 4, "NULL array");
  for (int i = 0; i < batch; ++i) {
    if (n[i] < 0) return bad_arg(h, 4, "n[i] < 0");
    if (n[i] > 0 && !dA[i]) return bad_arg(h, 5, "dA[i] is NULL");
    if (lda[i] < (n[i] > 1 ? n[i] : 1)) return bad_arg(h, 6, "lda[i] < max(1, n[i])");
  }
  return HRP_OK;
}

}  // namespace
}  // namespace hrp

extern "C" {

hrp_status hrp_potrf_batched(hrp_handle* h, const hrp_tree* const* trees_in, int batch, const int* n,
                             double* const* dA, const int* lda, int* d_info, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = check_batch_args(h, batch, n, dA, lda);
  if (st != HRP_OK) return st;
  if (batch > 0 && !d_info) return bad_arg(h, 7, "d_info is NULL");
  std::vector<hrp_tree> chosen;
  std::vector<const hrp_tree*> tv;
  if ((st = batch_trees(h, trees_in, batch, n, dA, lda, chosen, tv, stream)) != HRP_OK) return st;
  const hrp_tree* const* trees = tv.data();
  for (int i = 0; i < batch; ++i) {
    if ((st = validate_tree(h, trees[i], 2)) != HRP_OK) return st;
    if (tree_has(trees[i], HRP_F8E4M3)) return set_err(h, HRP_ERR_UNSUPPORTED, "F8 levels are not batched");
  }
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->batched_mode == 1) {
    if (batch == 0) return HRP_OK;
    std::vector<PSys> ps(batch);
    for (int i = 0; i < batch; ++i) ps[i] = PSys{trees[i], n[i], dA[i], lda[i], nullptr, 0, d_info + i};
    h->launches = 0;
    return enqueue_persistent(h, ps, s, &h->launches);
  }
  std::vector<SysWork> ws;
  if ((st = batch_prepare(h, batch, n, ws, true)) != HRP_OK) return st;
  if (batch == 0) return HRP_OK;
  const bool tc = tc_gemm_supported();
  std::vector<int> which = lpt_assign(batch, n, kBatchStreams);
  if ((st = fork(h, s)) != HRP_OK) return st;
  long long launches = 0;
  const bool timing = h->timing;
  h->timing = false;                       // per-launch event timing is not used in batches
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < batch; ++i) {
    Fact f{};
    f.h = h;
    f.t = trees[i];
    f.A = dA[i];
    f.lda = lda[i];
    f.n = n[i];
    f.info = d_info + i;
    f.s = h->bstreams[which[i]];
    f.tc = tc;
    f.lds = ws[i].lds;
    f.shadow = tree_has(f.t, HRP_F16) ? reinterpret_cast<__half*>(h->bwork + ws[i].shadow) : nullptr;
    f.shadow8 = nullptr;
    f.tile_exp = nullptr;
    f.w32 = (tree_has(f.t, HRP_F32) || tree_has(f.t, HRP_F16)) ? reinterpret_cast<float*>(h->bwork + ws[i].w32)
                                                                : nullptr;
    f.begin(CLS_OTHER, 0.0);
    f.chk(launch_fill_int(f.info, INT_MAX, 1, f.s));
    f.potrf(0, f.n, 0);
    f.begin(CLS_OTHER, 0.0);
    f.chk(launch_finalize_info(f.info, f.s));
    launches += f.launches;
    if (f.err != cudaSuccess && err == cudaSuccess) err = f.err;
  }
  h->timing = timing;
  if ((st = join(h, s)) != HRP_OK) return st;
  h->launches = launches;
  return cuda_status(h, err, "hrp_potrf_batched");
}

hrp_status hrp_potrs_batched(hrp_handle* h, int batch, const int* n, double* const* dL, const int* ldl, int nrhs,
                             double* const* dB, const int* ldb, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = check_batch_args(h, batch, n, dL, ldl);
  if (st != HRP_OK) return st;
  if (nrhs < 0) return bad_arg(h, 6, "nrhs < 0");
  if (batch > 0 && nrhs > 0 && (!dB || !ldb)) return bad_arg(h, 7, "dB/ldb is NULL");
  for (int i = 0; i < batch && nrhs > 0; ++i)
    if ((n[i] > 0 && !dB[i]) || ldb[i] < (n[i] > 1 ? n[i] : 1)) return bad_arg(h, 7, "dB[i] / ldb[i]");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<SysWork> ws;
  if ((st = batch_prepare(h, batch, n, ws, true)) != HRP_OK) return st;
  if (batch == 0 || nrhs == 0) return HRP_OK;
  std::vector<int> which = lpt_assign(batch, n, kBatchStreams);
  if ((st = fork(h, s)) != HRP_OK) return st;
  cudaError_t err = cudaSuccess;
  long long launches = 0;
  for (int i = 0; i < batch; ++i) {
    if (n[i] == 0) continue;
    cudaStream_t si = h->bstreams[which[i]];
    cudaError_t e = launch_potrs(dL[i], ldl[i], dB[i], ldb[i], n[i], nrhs, false, h->bwork + ws[i].pinv,
                                 reinterpret_cast<int*>(h->bwork + ws[i].ticket), h->d_err, si, h->wait_ns);
    launches += 1 + potrs_sweeps(nrhs);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  if ((st = join(h, s)) != HRP_OK) return st;
  h->launches = launches;
  return cuda_status(h, err, "hrp_potrs_batched");
}

}  // extern "C"


// ---------------------------------------------------------------------------------------
// Learned precision policy: features, MLP, and the table of candidate trees.
// ---------------------------------------------------------------------------------------
namespace hrp {
namespace {

const char* kPolicyTrees[8] = {
    "[F32|F64@128]",                 // 0: the conservative fallback
    "[F16,F32|F64@128]",
    "[F16,F16,F32|F64@128]",
    "[F16,F16,F16,F32|F64@128]",
    "[F16,F16,F16,F16,F32|F64@128]",
    "[F16,F16,F16,F16,F16,F32|F64@128]",
    "[F8,F16,F32|F64@128]",
    "[F8,F16,F16,F16,F32|F64@128]",
};

// The array following "key": in a JSON text (the policy file's flat layout: one array of
// numbers, or of strings without escapes, per key).  False if the key or the array is missing
// or malformed.
size_t json_array_start(const std::string& t, const char* key) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = t.find(k);
  if (p == std::string::npos) return std::string::npos;
  p = t.find_first_not_of(" \t\r\n", p + k.size());
  if (p == std::string::npos || t[p] != ':') return std::string::npos;
  p = t.find_first_not_of(" \t\r\n", p + 1);
  if (p == std::string::npos || t[p] != '[') return std::string::npos;
  return p + 1;
}
bool json_numbers(const std::string& t, const char* key, std::vector<float>& out) {
  size_t p = json_array_start(t, key);
  if (p == std::string::npos) return false;
  out.clear();
  const char* c = t.c_str() + p;
  while (true) {
    while (*c == ' ' || *c == ',' || *c == '\n' || *c == '\r' || *c == '\t') ++c;
    if (*c == ']') return true;
    char* end = nullptr;
    const double v = strtod(c, &end);
    if (end == c) return false;
    out.push_back((float)v);
    c = end;
  }
}
bool json_strings(const std::string& t, const char* key, std::vector<std::string>& out) {
  size_t p = json_array_start(t, key);
  if (p == std::string::npos) return false;
  out.clear();
  while (true) {
    p = t.find_first_not_of(" ,\t\r\n", p);
    if (p == std::string::npos) return false;
    if (t[p] == ']') return true;
    if (t[p] != '"') return false;
    const size_t q = t.find('"', p + 1);
    if (q == std::string::npos) return false;
    out.push_back(t.substr(p + 1, q - p - 1));
    p = q + 1;
  }
}

// number of eigenvalues of the symmetric tridiagonal (a, b) smaller than x (Sturm count)
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    q = a[i] - x - (i ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}
// k-th smallest eigenvalue (0-based) by bisection inside the Gershgorin interval
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double r = (i ? fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(fabs(lo), fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace
}  // namespace hrp

extern "C" {

hrp_status hrp_policy_features(hrp_handle* h, int n, const double* dA, int lda, int lanczos_steps, float* feat,
                               void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (n < 1) return bad_arg(h, 2, "n < 1");
  if (!dA) return bad_arg(h, 3, "dA is NULL");
  if (lda < n) return bad_arg(h, 4, "lda < n");
  if (lanczos_steps < 1) return bad_arg(h, 5, "lanczos_steps < 1");
  if (!feat) return bad_arg(h, 6, "feat is NULL");
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  hrp_status st;
  if ((st = ensure(h, &h->fwork, &h->fwork_cap, (size_t)5 * n + 16)) != HRP_OK) return st;
  double* rowsum = h->fwork;
  double* v = rowsum + n;
  double* vp = v + n;
  double* R = vp + n;
  double* zero = R + n;
  double* sc = zero + n;               // 16 scalars
  double init[8] = {0.0, 1e300, 0.0, 0.0, 1e300, 0.0, 0.0, 0.0};
  cudaError_t e = cudaMemsetAsync(rowsum, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(vp, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sc, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_rowsum(dA, lda, n, rowsum, sc, s);
  double stats[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(stats, sc, sizeof(stats), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_policy_features");
  // Lanczos: alpha_j, beta_j stay on the device; one read at the end
  const int k = std::min(lanczos_steps, n);
  if ((st = ensure(h, &h->fwork, &h->fwork_cap, (size_t)5 * n + 16 + 3 * (size_t)k)) != HRP_OK) return st;
  rowsum = h->fwork;
  v = rowsum + n;
  vp = v + n;
  R = vp + n;
  zero = R + n;
  sc = zero + n;
  double* dal = sc + 16;          // alpha_j
  double* dn2 = dal + k;          // ||w_j||^2
  double* dbe = dn2 + k;          // beta_{j+1}
  e = launch_lanczos_start(v, n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(vp, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dal, 0, sizeof(double) * 3 * k, s);
  for (int j = 0; j < k && e == cudaSuccess; ++j) {
    e = launch_symv32(dA, lda, v, R, n, s);                             // R = -A v
    if (e == cudaSuccess) e = launch_lanczos_dot(R, v, n, dal + j, s);
    if (e == cudaSuccess) e = launch_lanczos_axpy(R, v, vp, n, dal + j, j ? dbe + j - 1 : nullptr, dn2 + j, s);
    if (e == cudaSuccess && j + 1 < k) e = launch_lanczos_next(R, vp, v, n, dn2 + j, dbe + j, s);
  }
  std::vector<double> al(k), be;
  std::vector<double> bev(k);
  if (e == cudaSuccess) e = cudaMemcpyAsync(al.data(), dal, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bev.data(), dbe, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_policy_features lanczos");
  // stop at a breakdown (beta = 0): the Krylov space is exhausted
  int kk = k;
  for (int j = 0; j + 1 < k; ++j)
    if (!(bev[j] > 0.0)) { kk = j + 1; break; }
  al.resize(kk);
  be.assign(bev.begin(), bev.begin() + (kk - 1));
  const double lmin = tridiag_eig(al, be, 0), lmax = tridiag_eig(al, be, (int)al.size() - 1);
  const double fro = sqrt(stats[0]);
  auto lg = [](double x) { return log10(std::max(x, 1e-300)); };
  double f[12];
  f[0] = log2((double)n);
  f[1] = std::min(stats[1], 1e6);
  f[2] = stats[2] / n;
  f[3] = stats[3] / n;
  f[4] = lg(fro);
  f[5] = lg(stats[5]);
  f[6] = lg(stats[4]);
  f[7] = f[5] - f[6];
  f[8] = lg(lmax);
  f[9] = lg(lmin);
  f[10] = f[8] - f[9];
  f[11] = lg(n * std::max(lmin, 1e-300) / fro);
  for (int i = 0; i < 12; ++i) feat[i] = (float)f[i];
  return HRP_OK;
}

hrp_status hrp_mlp_forward(hrp_handle* h, const float* d_params, int batch, const float* d_X, float* d_Z,
                           void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  if (!d_params || batch < 0 || (batch > 0 && (!d_X || !d_Z))) return bad_arg(h, 2, "bad MLP argument");
  cudaSetDevice(h->device);
  return cuda_status(h, launch_mlp_forward(d_params, batch, d_X, d_Z, static_cast<cudaStream_t>(stream)),
                     "hrp_mlp_forward");
}

hrp_status hrp_mlp_grad(hrp_handle* h, const float* d_params, int batch, const float* d_X, const int* d_y,
                        float* d_grad, float* d_loss, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  if (!d_params || batch < 0 || !d_grad || !d_loss || (batch > 0 && (!d_X || !d_y)))
    return bad_arg(h, 2, "bad MLP argument");
  cudaSetDevice(h->device);
  return cuda_status(h, launch_mlp_grad(d_params, batch, d_X, d_y, d_grad, d_loss, static_cast<cudaStream_t>(stream)),
                     "hrp_mlp_grad");
}

hrp_status hrp_mlp_adam(hrp_handle* h, float* d_params, const float* d_grad, float* d_m, float* d_v, int step,
                        float lr, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  if (!d_params || !d_grad || !d_m || !d_v || step < 1) return bad_arg(h, 2, "bad Adam argument");
  cudaSetDevice(h->device);
  return cuda_status(h, launch_adam(d_params, d_grad, d_m, d_v, step, lr, static_cast<cudaStream_t>(stream)),
                     "hrp_mlp_adam");
}

int hrp_mlp_param_count(void) { return policy_nparam(); }

hrp_status hrp_policy_set(hrp_handle* h, const float* params, const float* mean, const float* scale) {
  if (!h) return HRP_ERR_INVALID_ARG;
  if (!params || !mean || !scale) return bad_arg(h, 2, "NULL policy array");
  cudaSetDevice(h->device);
  const int np = policy_nparam();
  // fold the input standardization x' = (x - mean) / scale into the first layer
  std::vector<float> p(params, params + np);
  for (int j = 0; j < 64; ++j) {
    double b = p[64 * 12 + j];
    for (int k = 0; k < 12; ++k) {
      const double w = params[j * 12 + k] / (double)scale[k];
      p[j * 12 + k] = (float)w;
      b -= w * mean[k];
    }
    p[64 * 12 + j] = (float)b;
  }
  size_t cap = h->policy ? (size_t)np : 0;
  hrp_status st = ensure(h, &h->policy, &cap, (size_t)np);
  if (st != HRP_OK) return st;
  size_t cap2 = h->pio ? 32 : 0;
  if ((st = ensure(h, &h->pio, &cap2, 32)) != HRP_OK) return st;
  if (cudaMemcpy(h->policy, p.data(), sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(h, HRP_ERR_CUDA, "hrp_policy_set");
  h->policy_set = true;
  h->policy_min_n = 0;
  return HRP_OK;
}

hrp_status hrp_policy_predict(hrp_handle* h, const float* feat, hrp_tree* out, int* index) {
  if (!h) return HRP_ERR_INVALID_ARG;
  if (!feat) return bad_arg(h, 2, "feat is NULL");
  if (!out && !index) return bad_arg(h, 3, "out and index are both NULL");
  if (!h->policy_set) return set_err(h, HRP_ERR_INVALID_ARG, "no policy loaded (hrp_policy_set)");
  cudaSetDevice(h->device);
  float z[8];
  cudaError_t e = cudaMemcpy(h->pio, feat, 12 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_mlp_forward(h->policy, 1, h->pio, h->pio + 16, 0);
  if (e == cudaSuccess) e = cudaMemcpy(z, h->pio + 16, sizeof(z), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(h, e, "hrp_policy_predict");
  int best = 0;
  for (int i = 1; i < 8; ++i)
    if (z[i] > z[best]) best = i;
  if (index) *index = best;
  if (out) return hrp_policy_tree(best, out);
  return HRP_OK;
}

hrp_status hrp_policy_tree(int index, hrp_tree* out) {
  if (index < 0 || index >= 8 || !out) return HRP_ERR_INVALID_ARG;
  return hrp_tree_parse(kPolicyTrees[index], 128, out);
}

hrp_status hrp_policy_load(hrp_handle* h, const char* path) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (!path) return bad_arg(h, 2, "path is NULL");
  FILE* f = fopen(path, "rb");
  if (!f) return set_err(h, HRP_ERR_INVALID_ARG, "cannot open %s", path);
  std::string text;
  char buf[65536];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  if (text.find("\"hrp-policy-v1\"") == std::string::npos)
    return set_err(h, HRP_ERR_INVALID_ARG, "%s: not an hrp-policy-v1 file", path);
  // the candidate trees the weights were trained for must be this library's, in order
  std::vector<std::string> trees;
  if (!json_strings(text, "trees", trees) || trees.size() != 8)
    return set_err(h, HRP_ERR_INVALID_ARG, "%s: \"trees\" must list 8 trees", path);
  for (int i = 0; i < 8; ++i) {
    hrp_tree a, b;
    if (hrp_tree_parse(trees[i].c_str(), 128, &a) != HRP_OK || hrp_tree_parse(kPolicyTrees[i], 128, &b) != HRP_OK ||
        memcmp(&a, &b, sizeof(a)) != 0)
      return set_err(h, HRP_ERR_INVALID_ARG, "%s: tree %d is %s, this library's is %s", path, i, trees[i].c_str(),
                     kPolicyTrees[i]);
  }
  std::vector<float> params, mean, scale;
  if (!json_numbers(text, "params", params) || (int)params.size() != policy_nparam())
    return set_err(h, HRP_ERR_INVALID_ARG, "%s: \"params\" must hold %d numbers", path, policy_nparam());
  if (!json_numbers(text, "mean", mean) || mean.size() != 12 || !json_numbers(text, "scale", scale) ||
      scale.size() != 12)
    return set_err(h, HRP_ERR_INVALID_ARG, "%s: \"mean\" and \"scale\" must hold 12 numbers each", path);
  for (float v : scale)
    if (!(v > 0.f)) return set_err(h, HRP_ERR_INVALID_ARG, "%s: a scale is not positive", path);
  // optional "min_n": [order], the smallest order at which the policy paid for its features
  std::vector<float> min_n;
  int gate = 0;
  if (json_numbers(text, "min_n", min_n)) {
    if (min_n.size() != 1 || !(min_n[0] >= 0.f) || !(min_n[0] <= 2147483647.f))
      return set_err(h, HRP_ERR_INVALID_ARG, "%s: \"min_n\" must hold one order >= 0", path);
    gate = (int)min_n[0];
  }
  hrp_status st = hrp_policy_set(h, params.data(), mean.data(), scale.data());
  if (st == HRP_OK) h->policy_min_n = gate;
  return st;
}

hrp_status hrp_policy_set_min_order(hrp_handle* h, int n_min) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  if (n_min < 0) return bad_arg(h, 2, "n_min < 0");
  h->policy_min_n = n_min;
  return HRP_OK;
}

int hrp_last_policy_choice(const hrp_handle* h) { return h ? h->last_choice : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batched solve with FP64 iterative refinement (the many-systems counterpart of hrp_posv).
// ---------------------------------------------------------------------------------------
extern "C" hrp_status hrp_posv_batched(hrp_handle* h, const hrp_tree* const* trees_in, int batch, const int* n,
                                       double* const* dA, const int* lda, int nrhs, double* const* dB, const int* ldb,
                                       double* const* dX, const int* ldx, int max_iter, double tol, int* info,
                                       int* iters, double* resid, int* used_fallback, void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = check_batch_args(h, batch, n, dA, lda);
  if (st != HRP_OK) return st;
  if (nrhs < 1 || nrhs > 16) return bad_arg(h, 7, "nrhs must be in [1, 16]");
  if (batch > 0 && (!dB || !ldb || !dX || !ldx)) return bad_arg(h, 8, "NULL B or X arrays");
  std::vector<hrp_tree> chosen;
  std::vector<const hrp_tree*> tv;
  if ((st = batch_trees(h, trees_in, batch, n, dA, lda, chosen, tv, stream)) != HRP_OK) return st;
  const hrp_tree* const* trees = tv.data();
  for (int i = 0; i < batch; ++i) {
    if ((st = validate_tree(h, trees[i], 2)) != HRP_OK) return st;
    if (tree_has(trees[i], HRP_F8E4M3)) return set_err(h, HRP_ERR_UNSUPPORTED, "F8 levels are not batched");
    if (ldb[i] < std::max(1, n[i]) || ldx[i] < std::max(1, n[i])) return bad_arg(h, 9, "ldb/ldx");
  }
  cudaSetDevice(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<SysWork> ws;
  if ((st = batch_prepare(h, batch, n, ws, true, nrhs)) != HRP_OK) return st;
  if (batch == 0) return HRP_OK;
  int* d_info = nullptr;
  if (cudaMalloc(&d_info, sizeof(int) * batch) != cudaSuccess) return set_err(h, HRP_ERR_ALLOC, "info array");
  std::vector<int> hinfo(batch, 0), fb(batch, 0), its(batch, 0), done(batch, 0), fresh(batch, 1), restart;
  std::vector<double> res(batch, 1e300);
  std::vector<double> norms(2 * nrhs);
  hrp_tree fallback;
  hrp_tree_parse("[F32|F64@128]", 128, &fallback);
  const bool tc = tc_gemm_supported();
  std::vector<int> which = lpt_assign(batch, n, kBatchStreams);
  auto fact_of = [&](int i) { return reinterpret_cast<double*>(h->bwork + ws[i].fact); };
  auto res_of = [&](int i) { return reinterpret_cast<double*>(h->bwork + ws[i].res); };
  cudaError_t err = cudaSuccess;
  auto note = [&](cudaError_t e) { if (e != cudaSuccess && err == cudaSuccess) err = e; };
  const bool timing = h->timing;
  h->timing = false;
  // factor copies of every system (mixed trees), then the fallback tree where that failed
  for (int pass = 0; pass < 2 && err == cudaSuccess; ++pass) {
    if (h->batched_mode == 1) {
      std::vector<PSys> ps;
      for (int i = 0; i < batch; ++i) {
        if (n[i] == 0 || (pass == 1 && hinfo[i] == 0)) continue;
        ps.push_back(PSys{pass == 0 ? trees[i] : &fallback, n[i], fact_of(i), n[i], dA[i], lda[i], d_info + i});
        if (pass == 1) fb[i] = 1;
      }
      if ((st = enqueue_persistent(h, ps, s, nullptr)) != HRP_OK) break;
    } else {
    if ((st = fork(h, s)) != HRP_OK) break;
    for (int i = 0; i < batch; ++i) {
      if (n[i] == 0 || (pass == 1 && hinfo[i] == 0)) continue;
      cudaStream_t si = h->bstreams[which[i]];
      note(launch_copy_lower(fact_of(i), n[i], dA[i], lda[i], n[i], si));
      Fact f{};
      f.h = h;
      f.t = pass == 0 ? trees[i] : &fallback;
      f.A = fact_of(i);
      f.lda = n[i];
      f.n = n[i];
      f.info = d_info + i;
      f.s = si;
      f.tc = tc;
      f.lds = ws[i].lds;
      f.shadow = tree_has(f.t, HRP_F16) ? reinterpret_cast<__half*>(h->bwork + ws[i].shadow) : nullptr;
      f.w32 = reinterpret_cast<float*>(h->bwork + ws[i].w32);
      f.begin(CLS_OTHER, 0.0);
      f.chk(launch_fill_int(f.info, INT_MAX, 1, si));
      f.potrf(0, n[i], 0);
      f.begin(CLS_OTHER, 0.0);
      f.chk(launch_finalize_info(f.info, si));
      note(f.err);
      if (pass == 1) fb[i] = 1;
    }
    if ((st = join(h, s)) != HRP_OK) break;
    }
    note(cudaMemcpyAsync(hinfo.data(), d_info, sizeof(int) * batch, cudaMemcpyDeviceToHost, s));
    note(cudaStreamSynchronize(s));
    if (err != cudaSuccess) break;
    st = check_dev_err(h, s);
    if (st == HRP_ERR_RANGE && pass == 0) {
      // some FP16 operand needs alpha > 1: the systems with FP16 levels take the fallback tree
      st = HRP_OK;
      for (int i = 0; i < batch; ++i)
        if (n[i] > 0 && tree_has(trees[i], HRP_F16)) hinfo[i] = -1;
    }
    if (st != HRP_OK) break;
    bool any = false;
    for (int i = 0; i < batch; ++i) any |= hinfo[i] != 0;
    if (!any) break;
  }
  h->timing = timing;
  // X0 = POTRS(B) in FP32, then rounds of refinement over the systems not yet converged
  for (int it = 0; st == HRP_OK && err == cudaSuccess; ++it) {
    if ((st = fork(h, s)) != HRP_OK) break;
    for (int i = 0; i < batch; ++i) {
      if (n[i] == 0 || hinfo[i] != 0 || done[i]) continue;
      cudaStream_t si = h->bstreams[which[i]];
      double* R = res_of(i);
      if (fresh[i]) {
        fresh[i] = 0;
        note(launch_copy_matrix(dX[i], ldx[i], dB[i], ldb[i], n[i], nrhs, si));
        note(launch_potrs(fact_of(i), n[i], dX[i], ldx[i], n[i], nrhs, true, h->bwork + ws[i].pinv,
                          reinterpret_cast<int*>(h->bwork + ws[i].ticket), h->d_err, si, h->wait_ns));
      } else {
        note(launch_potrs(fact_of(i), n[i], R, n[i], n[i], nrhs, true, h->bwork + ws[i].pinv,
                          reinterpret_cast<int*>(h->bwork + ws[i].ticket), h->d_err, si, h->wait_ns));
        note(launch_axpy_matrix(dX[i], ldx[i], R, n[i], n[i], nrhs, si));
        ++its[i];
      }
      note(launch_residual(dA[i], lda[i], dX[i], ldx[i], dB[i], ldb[i], R, n[i], n[i], nrhs, si));
      note(launch_col_norms2(R, n[i], dB[i], ldb[i], n[i], nrhs, R + (size_t)n[i] * nrhs, si));
    }
    if ((st = join(h, s)) != HRP_OK) break;
    note(cudaStreamSynchronize(s));
    if (err != cudaSuccess) break;
    if ((st = check_dev_err(h, s)) != HRP_OK) break;       // a solve's bounded wait expired
    bool all = true;
    for (int i = 0; i < batch; ++i) {
      if (n[i] == 0 || hinfo[i] != 0 || done[i]) continue;
      note(cudaMemcpy(norms.data(), res_of(i) + (size_t)n[i] * nrhs, sizeof(double) * 2 * nrhs,
                      cudaMemcpyDeviceToHost));
      double worst = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        const double rb = norms[nrhs + c] > 0 ? sqrt(norms[c] / norms[nrhs + c]) : sqrt(norms[c]);
        if (!(rb <= worst)) worst = rb;
      }
      const bool stalled = its[i] > 0 && !(worst < res[i]);
      res[i] = worst;
      if (worst <= tol || (its[i] >= max_iter && fb[i]) || (stalled && fb[i])) {
        done[i] = 1;
      } else if ((stalled || its[i] >= max_iter) && !fb[i]) {
        restart.push_back(i);          // this factor will not get there: fallback tree
        all = false;
      } else {
        all = false;
      }
    }
    if (!restart.empty() && h->batched_mode == 1) {
      std::vector<PSys> ps;
      for (int i : restart) {
        ps.push_back(PSys{&fallback, n[i], fact_of(i), n[i], dA[i], lda[i], d_info + i});
        fb[i] = 1;
        fresh[i] = 1;
        its[i] = 0;
        res[i] = 1e300;
      }
      if ((st = enqueue_persistent(h, ps, s, nullptr)) != HRP_OK) break;
      note(cudaMemcpyAsync(hinfo.data(), d_info, sizeof(int) * batch, cudaMemcpyDeviceToHost, s));
      note(cudaStreamSynchronize(s));
      if (err == cudaSuccess && (st = check_dev_err(h, s)) != HRP_OK) break;
      restart.clear();
    }
    if (!restart.empty()) {
      // refactor the stalled systems with the fallback tree; they restart their solve
      if ((st = fork(h, s)) != HRP_OK) break;
      for (int i : restart) {
        cudaStream_t si = h->bstreams[which[i]];
        note(launch_copy_lower(fact_of(i), n[i], dA[i], lda[i], n[i], si));
        Fact f{};
        f.h = h;
        f.t = &fallback;
        f.A = fact_of(i);
        f.lda = n[i];
        f.n = n[i];
        f.info = d_info + i;
        f.s = si;
        f.tc = tc;
        f.lds = ws[i].lds;
        f.shadow = nullptr;
        f.w32 = reinterpret_cast<float*>(h->bwork + ws[i].w32);
        f.begin(CLS_OTHER, 0.0);
        f.chk(launch_fill_int(f.info, INT_MAX, 1, si));
        f.potrf(0, n[i], 0);
        f.begin(CLS_OTHER, 0.0);
        f.chk(launch_finalize_info(f.info, si));
        note(f.err);
        fb[i] = 1;
        fresh[i] = 1;
        its[i] = 0;
        res[i] = 1e300;
      }
      if ((st = join(h, s)) != HRP_OK) break;
      note(cudaMemcpyAsync(hinfo.data(), d_info, sizeof(int) * batch, cudaMemcpyDeviceToHost, s));
      note(cudaStreamSynchronize(s));
      if (err == cudaSuccess && (st = check_dev_err(h, s)) != HRP_OK) break;
      restart.clear();
    }
    if (all) break;
  }
  cudaFree(d_info);
  bool conv = true, spd = true;
  for (int i = 0; i < batch; ++i) {
    if (info) info[i] = hinfo[i];
    if (iters) iters[i] = its[i];
    if (resid) resid[i] = res[i];
    if (used_fallback) used_fallback[i] = fb[i];
    spd &= hinfo[i] == 0;
    conv &= (hinfo[i] != 0) || n[i] == 0 || res[i] <= tol;
  }
  if (st != HRP_OK) return st;
  if (err != cudaSuccess) return cuda_status(h, err, "hrp_posv_batched");
  if (!spd) return set_err(h, HRP_ERR_NOT_SPD, "a system failed with the fallback tree too");
  if (!conv) return set_err(h, HRP_ERR_NO_CONVERGENCE, "a system did not reach tol");
  return HRP_OK;
}

// ---------------------------------------------------------------------------------------
// Standalone Tree-SYRK (Alg. 3) and Tree-TRSM (Alg. 2) with the precision list applied to
// their own recursion (Sec. 4.2's SYRK and TRSM experiments): the GEMM of a node at
// recursion depth t runs at level[t] (nodes deeper than the list use its last entry; a
// node of order <= inner_size uses `inner`), and the base case at the precision of its node.
// ---------------------------------------------------------------------------------------
namespace hrp {
namespace {

struct Blas3 {
  hrp_handle* h;
  const hrp_tree* t;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  long long launches = 0;
  void chk(cudaError_t e) {
    ++launches;
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  int prec(int depth, int order) const { return node_prec(t, depth, order); }
};

// C (n x n lower, ldc) -= A A^T with A n x k (lda).  S16: row-major FP16 copy of A (lds), A32:
// column-major FP32 copy (ld32), each present when the tree has that precision.
struct SyrkRun : Blas3 {
  double* C;
  int ldc;
  const double* A;
  int lda, k;
  const __half* S16;
  int lds;
  const float* A32;
  int ld32;
  const float* h32 = nullptr;    // TF32 split of A (row-major, ldh), when FP32 levels run on tcgen05
  const float* l32 = nullptr;
  int ldh = 0;
  bool tc;
  int base() const { return t->syrk_leaf ? t->syrk_leaf : t->leaf; }
  // C[r0:r0+m, c0:c0+nd] -= A[r0:r0+m, :] A[c0:c0+nd, :]^T at precision p
  void gemm(int p, int r0, int m, int c0, int nd, bool lower) {
    double* Cb = C + (size_t)c0 * ldc + r0;
    switch (p) {
      case HRP_F64:
        chk(launch_gemm_simt(Cb, ldc, A + r0, lda, A + c0, lda, m, nd, k, OpRound::F64, lower, s));
        break;
      case HRP_F32:
        if (h32 && split_tc_worth(m, nd, k))
          chk(launch_gemm_tf32x3_tc(Cb, ldc, h32, l32, ldh, r0, c0, 0, m, nd, k, lower, h->d_err, s));
        else
          chk(launch_gemm_simt_f32(Cb, ldc, A32 + r0, ld32, A32 + c0, ld32, m, nd, k, lower, s));
        break;
      case HRP_F16:
        if (tc && k >= 16) chk(launch_gemm_f16_tc(Cb, ldc, S16, lds, r0, c0, 0, m, nd, k, lower, 1.0, h->d_err, s));
        else chk(launch_gemm_simt(Cb, ldc, A + r0, lda, A + c0, lda, m, nd, k, OpRound::F16, lower, s));
        break;
      default:
        if (err == cudaSuccess) err = cudaErrorNotSupported;
    }
  }
  void rec(int c0, int nc, int depth) {
    if (nc <= 0) return;
    const int p = prec(depth, nc);
    if (nc <= base()) {                          // base case: the lower triangle of one GEMM
      gemm(p, c0, nc, c0, nc, true);
      return;
    }
    const int n1 = split(nc), n2 = nc - n1;
    rec(c0, n1, depth + 1);
    gemm(p, c0 + n1, n2, c0, n1, false);         // C21 -= A2 A1^T
    rec(c0 + n1, n2, depth + 1);
  }
};

// B (m x n, ldb) <- B L^{-T} with L n x n lower (ldl).  S16: row-major FP16 rows [0, m) hold B's
// solved columns (written by the base cases), rows [m, m + n) L; B32 / L32: column-major FP32
// copies (ld m and n).
struct TrsmRun : Blas3 {
  double* B;
  int ldb, m;
  const double* L;
  int ldl;
  __half* S16;
  int lds;
  float* B32;
  const float* L32;
  bool tc;
  int* info;
  int tleaf() const { return t->trsm_leaf ? t->trsm_leaf : t->leaf; }
  void leaf(int c0, int nc, int p) {
    if (p == HRP_F64 || t->trsm_compute == 1)
      chk(launch_trsm_leaf64(B, ldb, 0, m, c0, nc, S16, lds, B32, m, info, h->d_err, s, L, ldl));
    else
      chk(launch_trsm_leaf32_subst(B, ldb, 0, m, c0, nc, S16, lds, B32, m, info, h->d_err, s, L, ldl));
  }
  // B[:, c0+n1 : c0+nc] -= B[:, c0 : c0+n1] L[c0+n1 : c0+nc, c0 : c0+n1]^T at precision p
  void gemm(int p, int c0, int n1, int n2) {
    double* Cb = B + (size_t)(c0 + n1) * ldb;
    switch (p) {
      case HRP_F64:
        chk(launch_gemm_simt(Cb, ldb, B + (size_t)c0 * ldb, ldb, L + (size_t)c0 * ldl + c0 + n1, ldl, m, n2, n1,
                             OpRound::F64, false, s));
        break;
      case HRP_F32:
        chk(launch_gemm_simt_f32(Cb, ldb, B32 + (size_t)c0 * m, m, L32 + (size_t)c0 * t_n + c0 + n1, t_n, m, n2, n1,
                                 false, s));
        break;
      case HRP_F16:
        if (tc && c0 % 8 == 0 && n1 >= 16)
          chk(launch_gemm_f16_tc(Cb, ldb, S16, lds, 0, m + c0 + n1, c0, m, n2, n1, false, 1.0, h->d_err, s));
        else
          chk(launch_gemm_simt(Cb, ldb, B + (size_t)c0 * ldb, ldb, L + (size_t)c0 * ldl + c0 + n1, ldl, m, n2, n1,
                               OpRound::F16, false, s));
        break;
      default:
        if (err == cudaSuccess) err = cudaErrorNotSupported;
    }
  }
  int t_n = 0;                                   // order of L (leading dimension of L32)
  void rec(int c0, int nc, int depth) {
    const int p = prec(depth, nc);
    if (std::min(m, nc) <= tleaf()) {
      leaf(c0, nc, p);
      return;
    }
    const int n1 = split(nc), n2 = nc - n1;
    rec(c0, n1, depth + 1);
    gemm(p, c0, n1, n2);
    rec(c0 + n1, n2, depth + 1);
  }
};

hrp_status blas3_tree_check(hrp_handle* h, const hrp_tree* tree) {
  hrp_status st = validate_tree(h, tree, 2);
  if (st != HRP_OK) return st;
  if (tree_has(tree, HRP_F8E4M3)) return set_err(h, HRP_ERR_UNSUPPORTED, "F8 levels need the factorization's tiles");
  return HRP_OK;
}

}  // namespace
}  // namespace hrp

extern "C" {

hrp_status hrp_syrk(hrp_handle* h, const hrp_tree* tree, int n, int k, const double* dA, int lda, double* dC, int ldc,
                    void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = blas3_tree_check(h, tree);
  if (st != HRP_OK) return st;
  if (n < 0) return bad_arg(h, 3, "n < 0");
  if (k < 0) return bad_arg(h, 4, "k < 0");
  if (n > 0 && k > 0 && !dA) return bad_arg(h, 5, "dA is NULL");
  if (lda < (n > 1 ? n : 1)) return bad_arg(h, 6, "lda < max(1, n)");
  if (n > 0 && !dC) return bad_arg(h, 7, "dC is NULL");
  if (ldc < (n > 1 ? n : 1)) return bad_arg(h, 8, "ldc < max(1, n)");
  if (n == 0 || k == 0) return HRP_OK;
  cudaSetDevice(h->device);
  SyrkRun r{};
  r.h = h;
  r.t = tree;
  r.s = static_cast<cudaStream_t>(stream);
  r.C = dC;
  r.ldc = ldc;
  r.A = dA;
  r.lda = lda;
  r.k = k;
  r.tc = tc_gemm_supported();
  r.lds = (k + 63) / 64 * 64;
  r.ld32 = n;
  if (tree_has(tree, HRP_F16)) {
    if ((st = ensure(h, &h->shadow, &h->shadow_cap, (size_t)n * r.lds)) != HRP_OK) return st;
    r.S16 = h->shadow;
    r.chk(launch_cast_f16_rows(dA, lda, n, k, h->shadow, r.lds, h->d_err, r.s));
  }
  if (tree_has(tree, HRP_F32)) {
    if ((st = ensure(h, &h->shadow32, &h->shadow32_cap, (size_t)n * k)) != HRP_OK) return st;
    r.A32 = h->shadow32;
    r.chk(launch_cast_f32(dA, lda, n, k, h->shadow32, n, r.s));
    if (h->fp32_split && r.tc) {
      r.ldh = (k + 63) / 64 * 64;
      if ((st = ensure(h, &h->split32, &h->split32_cap, 2 * (size_t)n * r.ldh)) != HRP_OK) return st;
      r.h32 = h->split32;
      r.l32 = h->split32 + (size_t)n * r.ldh;
      r.chk(launch_split_tf32(dA, lda, 0, n, 0, k, h->split32, h->split32 + (size_t)n * r.ldh, r.ldh, r.s));
    }
  }
  r.rec(0, n, 0);
  launch_ctx() = LaunchCtx{};
  h->launches = r.launches;
  return cuda_status(h, r.err, "hrp_syrk");
}

hrp_status hrp_trsm(hrp_handle* h, const hrp_tree* tree, int m, int n, const double* dL, int ldl, double* dB, int ldb,
                    void* stream) {
  if (!h) return HRP_ERR_INVALID_ARG;
  h->last_arg = 0;
  hrp_status st = blas3_tree_check(h, tree);
  if (st != HRP_OK) return st;
  if (m < 0) return bad_arg(h, 3, "m < 0");
  if (n < 0) return bad_arg(h, 4, "n < 0");
  if (n > 0 && !dL) return bad_arg(h, 5, "dL is NULL");
  if (ldl < (n > 1 ? n : 1)) return bad_arg(h, 6, "ldl < max(1, n)");
  if (m > 0 && n > 0 && !dB) return bad_arg(h, 7, "dB is NULL");
  if (ldb < (m > 1 ? m : 1)) return bad_arg(h, 8, "ldb < max(1, m)");
  if (m == 0 || n == 0) return HRP_OK;
  const int tl = tree->trsm_leaf ? tree->trsm_leaf : tree->leaf;
  if (tl > 128 && m > 128) return bad_arg(h, 2, "trsm_leaf must be <= 128");
  cudaSetDevice(h->device);
  TrsmRun r{};
  r.h = h;
  r.t = tree;
  r.s = static_cast<cudaStream_t>(stream);
  r.B = dB;
  r.ldb = ldb;
  r.m = m;
  r.L = dL;
  r.ldl = ldl;
  r.t_n = n;
  r.tc = tc_gemm_supported();
  r.lds = (n + 63) / 64 * 64;
  r.info = h->d_info;
  r.chk(launch_fill_int(h->d_info, INT_MAX, 1, r.s));
  if (tree_has(tree, HRP_F16)) {
    if ((st = ensure(h, &h->shadow, &h->shadow_cap, (size_t)(m + n) * r.lds)) != HRP_OK) return st;
    r.S16 = h->shadow;
    r.chk(launch_cast_f16_rows(dL, ldl, n, n, h->shadow + (size_t)m * r.lds, r.lds, h->d_err, r.s));
  }
  if (tree_has(tree, HRP_F32)) {
    if ((st = ensure(h, &h->shadow32, &h->shadow32_cap, (size_t)m * n + (size_t)n * n)) != HRP_OK) return st;
    r.B32 = h->shadow32;
    r.L32 = h->shadow32 + (size_t)m * n;
    r.chk(launch_cast_f32(dL, ldl, n, n, h->shadow32 + (size_t)m * n, n, r.s));
  }
  r.rec(0, n, 0);
  launch_ctx() = LaunchCtx{};
  h->launches = r.launches;
  return cuda_status(h, r.err, "hrp_trsm");
}

}  // extern "C"
