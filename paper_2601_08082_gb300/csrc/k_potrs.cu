// POTRS: solve A X = B with the Cholesky factor, L Y = B then L^T X = Y.
//
// Two launches per sweep pair plus one pre-pass:
//   1. inverse pre-pass: every 64 x 64 diagonal block L_rr is inverted in parallel (one
//      CTA per block, right-looking, all columns at once), W_r = L_rr^{-1}.
//   2. forward sweep: the rows are cut into 64-row blocks; each CTA takes the next block
//      in sweep order from an atomic ticket (every block it waits for belongs to a CTA
//      that started earlier and is resident: no deadlock).  As soon as a solved block
//      appears in the sweep's mailbox the CTA accumulates its off-diagonal product, 4
//      threads per row each over 16 columns; at the end y_r = W_r (b_r - sum_j L_rj y_j)
//      is a small matrix product, so no division sits on the dependency chain between
//      blocks.
//   3. backward sweep, the same with L^T: x_r = W_r^T (y_r - sum_{j>r} L_jr^T x_j).
// Mailboxes: a solved block is handed on through a copy of its rows in a mailbox, one per
// sweep direction (16 columns x the padded order), whose entries hold kEmpty until their
// value is stored.  A consumer polls the values themselves: one round trip, and the producer
// needs no fence.  kEmpty is a NaN that no arithmetic produces (a stored value with that
// bit pattern is replaced by the canonical NaN).  The pre-pass empties the forward mailbox,
// each forward sweep the backward one and each backward sweep the forward one, in stream
// order, so a solve captured in a CUDA graph needs no host-side reset between replays.
// All waits are bounded by %globaltimer: on expiry the CTA records DEV_ERR_TIMEOUT, writes
// NaN into its own block of the solution and still publishes it, so blocks downstream turn
// NaN as well instead of waiting in turn; no entry is left unpublished.
#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int PB = kPotrsBlock;
constexpr int PT = 256;
constexpr int MAX_RHS = kPotrsMaxRhs;
constexpr unsigned long long kEmpty = 0xffffffffffffffffull;   // an empty mailbox entry

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// publish v in a mailbox entry (never as the bit pattern of an empty entry)
__device__ __forceinline__ void post(double* p, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (b == kEmpty) b = 0x7ff8000000000000ull;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}
// the value of mailbox entry *p once it is stored; false (out = NaN) when limit_ns of
// %globaltimer pass first
__device__ bool poll_entry(const double* p, unsigned long long limit_ns, double& out) {
  unsigned long long b = ld_relaxed64(p);
  if (b == kEmpty) {
    const unsigned long long t0 = gtimer();
    while (b == kEmpty) {
      for (int k = 0; k < 16 && b == kEmpty; ++k) {
        __nanosleep(64);
        b = ld_relaxed64(p);
      }
      if (b == kEmpty && gtimer() - t0 > limit_ns) {
        out = __longlong_as_double(0x7ff8000000000000ll);
        return false;
      }
    }
  }
  out = __longlong_as_double((long long)b);
  return true;
}
// empty the 16 mailbox columns of rows R0 .. R0 + 63
__device__ __forceinline__ void empty_rows(double* mb, int mbld, int R0, int tid) {
  for (int idx = tid; idx < MAX_RHS * PB; idx += PT)
    mb[(size_t)(idx / PB) * mbld + R0 + idx % PB] = __longlong_as_double((long long)kEmpty);
}
// One thread empties *entry and then waits on it through the sweeps' poll_entry; nothing
// fills it, so the wait must expire after limit_ns, record DEV_ERR_TIMEOUT and return.
// out[0] = the time waited.
__global__ void wait_probe_kernel(double* entry, unsigned long long limit_ns, unsigned* err, unsigned long long* out) {
  if (threadIdx.x != 0) return;
  *reinterpret_cast<volatile unsigned long long*>(entry) = kEmpty;
  const unsigned long long t0 = gtimer();
  double v;
  if (!poll_entry(entry, limit_ns, v)) atomicOr(err, DEV_ERR_TIMEOUT);
  out[0] = gtimer() - t0;
}

// ---- 1. W_r = L_rr^{-1} for every 64-row diagonal block (one CTA each) ----
template <typename T>
__global__ void __launch_bounds__(PT)
potrs_diag_inverse_kernel(const double* __restrict__ L, int ldl, int n, T* __restrict__ W, double* __restrict__ mb_fwd,
                          int mbld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*Ls)[PB + 1] = reinterpret_cast<T (*)[PB + 1]>(smem_raw);               // Ls[i][k] = L(R0+i, R0+k)
  T (*Ws)[PB + 1] = reinterpret_cast<T (*)[PB + 1]>(smem_raw + sizeof(T) * PB * (PB + 1));  // W(i, c)
  __shared__ T rinv[PB];
  const int r = blockIdx.x, R0 = r * PB, rows = min(PB, n - R0);
  const int tid = threadIdx.x;
  empty_rows(mb_fwd, mbld, R0, tid);           // the forward sweep's mailbox, for this solve
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

// ---- double-float arithmetic for the link of the FP64 sweeps ----
// On this GPU one SM retires under two FP64 lane-FMAs per clock, so the two 64 x 64 products
// that sit on the block-to-block chain (the newest block's contribution and the product with
// W_r) would cost ~2.4 us per link in FP64.  They run on the FP32 pipe instead: an operand x
// of one thread's 16 is carried as the pair hi + lo of binary32 values equal to x 2^-s, s the
// largest binary exponent among those 16, so that no pair leaves binary32's range; the
// products are summed by Dot2 (Ogita, Rump and Oishi, 2005: TwoSum on the running sum, the
// rounding errors and low-order cross terms gathered in a second word) and each thread's
// partial sum is widened back to binary64 exactly, then reduced in FP64.  The pair keeps 48
// of x's 53 significand bits (a relative error below 2^-47); entries below 2^-74 of the
// thread's largest are dropped, and a NaN or infinity turns the result NaN.
struct fpair {
  float hi, lo;
};

// largest unbiased binary exponent among v (0 when all are zero or subnormal)
__device__ __forceinline__ int scale_of16(const double (&v)[16]) {
  int mx = 0;
#pragma unroll
  for (int q = 0; q < 16; ++q) mx = max(mx, (int)((unsigned long long)__double_as_longlong(v[q]) >> 52) & 0x7ff);
  return mx == 0 ? 0 : mx - 1023;
}

// x 2^-s as a pair, by integer operations on the bit fields: hi = the sign and the leading 24
// significand bits (truncated), lo = the remaining 29 bits rounded to binary32
__device__ __forceinline__ fpair split_scaled(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0x7ff) return {__uint_as_float(0x7fc00000u), 0.0f};
  const int e = E - 1023 - s;
  if (E == 0 || e < -74) return {0.0f, 0.0f};
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  const float lo = __uint2float_rn((unsigned)(m & 0x1fffffffu)) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
  return {hi, __uint_as_float(__float_as_uint(lo) | sgn)};
}

// f 2^off as a binary64, exactly (zero and subnormal f give 0, a NaN or infinity gives NaN)
__device__ __forceinline__ double widen_scaled(float f, int off) {
  const unsigned u = __float_as_uint(f);
  const int E = (int)((u >> 23) & 0xff);
  if (E == 0) return 0.0;
  if (E == 0xff) return __longlong_as_double(0x7ff8000000000000ll);
  const int Ed = E - 127 + 1023 + off;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if (Ed <= 0) return 0.0;
  if (Ed >= 0x7ff) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull));
  return __longlong_as_double((long long)(sgn | ((unsigned long long)Ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// (s, c) += a b, Dot2 step
__device__ __forceinline__ void dot2_step(float& s, float& c, fpair a, fpair b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                  // a.hi b.hi = p + e exactly
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s + p, bb = t - s;
  c += ((s - (t - bb)) + (p - bb)) + e;
  s = t;
}

// sum_q a_q v_q for this thread's 16 pairs a (scale sa) and 16 pairs v (scale sv)
__device__ __forceinline__ double dot16_df(const fpair (&a)[16], int sa, const fpair* __restrict__ v, int sv) {
  float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;   // even and odd q: two independent chains
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    dot2_step(s0, c0, a[q], v[q]);
    dot2_step(s1, c1, a[q + 1], v[q + 1]);
  }
  const float s = s0 + s1, bb = s - s0;
  const float c = (c0 + c1) + ((s0 - (s - bb)) + (s1 - bb));
  return widen_scaled(s, sa + sv) + widen_scaled(c, sa + sv);
}

// x as a pair scaled by the largest exponent among the 32 lanes of its warp (the entries of two
// 16-entry column chunks); every lane of the warp must call it
__device__ __forceinline__ fpair split_chunk(double x, int& s) {
  // one warp-wide reduction: the scale is shared by the warp's two chunks (any common
  // power of two keeps the pairs exact; the group only sets which entries count as negligible)
  const int ex = (int)__reduce_max_sync(0xffffffffu, (unsigned)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff));
  s = ex == 0 ? 0 : ex - 1023;
  return split_scaled(x, s);
}

// ---- 2/3. sweeps ----
// With T = double every 16-term partial product runs in double-float as above, and the sums
// across chunks and blocks in FP64; the link between consecutive blocks is one product with
// M_r (formed at the CTA's start).  With T = float (the correction solves of the refinement)
// every product is binary32.  NR (1, 4 or 16) bounds the right-hand sides of one launch, which
// sizes the accumulators: a 1-RHS solve does not carry 16 of them through the sweep.
template <typename T, bool FWD, int NR>
__global__ void __launch_bounds__(PT, 1)
potrs_sweep_kernel(const double* __restrict__ L, int ldl, const T* __restrict__ W, double* __restrict__ B, int ldb,
                   int n, int nrhs, int* __restrict__ ticket, double* __restrict__ mb, double* __restrict__ mb_next,
                   int mbld, unsigned* __restrict__ err, unsigned long long limit_ns) {
  constexpr bool kDF = sizeof(T) == sizeof(double);
  __shared__ T yS[NR][PB];               // solved block of another CTA; later the reduced rhs
  __shared__ T part[4][NR][PB];          // per-chunk partial sums
  __shared__ int s_r, s_abort;
  __shared__ int vsc[NR][PB / 16];       // double-float: scale of each 16-entry chunk of the staged vector
  T (*accS)[PB] = yS;
  fpair (*vP)[PB] = reinterpret_cast<fpair (*)[PB]>(&yS[0][0]);   // double-float: the staged vector as pairs
  const int tid = threadIdx.x;
  const int nb = (n + PB - 1) / PB;
  if (tid == 0) {
    const int t = atomicAdd(ticket, 1);
    s_r = FWD ? t : nb - 1 - t;
    s_abort = 0;
  }
  __syncthreads();
  const int r = s_r, R0 = r * PB, rows = min(PB, n - R0);
  const int i = tid % PB, ch = tid / PB;           // row i, k-chunk ch (16 columns each)
  empty_rows(mb_next, mbld, R0, tid);              // the next sweep's mailbox (no one reads it now)
  T acc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = (T)0;

  // this block's right-hand side does not depend on other blocks either: its DRAM latency
  // stays off the block-to-block chain (thread tid holds entries tid + PT u)
  constexpr int kBU = (NR * PB + PT - 1) / PT;
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
  // this thread's 16 entries of the factor block L_rj (forward) or L_jr^T (backward)
  auto load_l = [&](int j, T (&lv)[16]) {
    const int J0 = j * PB, jrows = min(PB, n - J0);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int kk = ch * 16 + q;
      if (FWD) lv[q] = (kk < jrows && i < rows) ? (T)L[(size_t)(J0 + kk) * ldl + R0 + i] : (T)0;
      else lv[q] = (kk < jrows && i < rows) ? (T)L[(size_t)(R0 + i) * ldl + J0 + kk] : (T)0;
    }
  };
  // this block's solution (or NaN) into B and into the mailbox
  auto publish = [&](int ii, int c, double v) {
    B[(size_t)c * ldb + R0 + ii] = v;
    post(mb + (size_t)c * mbld + R0 + ii, v);
  };
  // wait for block j's entries and stage them in yS (as pairs in vP for double-float); false
  // when a wait expired (the block is then marked NaN and published, and the caller returns)
  auto await_block = [&](int j) -> bool {
    const int J0 = j * PB, jrows = min(PB, n - J0);
    bool ok = true;
    for (int idx = tid; idx < nrhs * PB; idx += PT) {   // nrhs * PB: whole warps
      const int kk = idx % PB, c = idx / PB;
      double v = 0.0;
      if (kk < jrows) ok &= poll_entry(mb + (size_t)c * mbld + J0 + kk, limit_ns, v);
      if constexpr (kDF) {
        int sv;
        vP[c][kk] = split_chunk(v, sv);
        if ((kk & 15) == 0) vsc[c][kk >> 4] = sv;
      } else {
        yS[c][kk] = (T)v;
      }
    }
    if (!ok) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();
    if (s_abort) {
      // this block cannot be solved: NaN marks it (and, through the products, every block
      // that depends on it); publishing it spares those blocks a wait of their own
      for (int idx = tid; idx < nrhs * PB; idx += PT) {
        const int ii = idx % PB, c = idx / PB;
        if (ii < rows) publish(ii, c, __longlong_as_double(0x7ff8000000000000ll));
      }
      return false;
    }
    return true;
  };
  // dependencies in the order they complete: j = 0, 1, .. (forward), nb-1, nb-2, .. (backward)
  const int ndep = FWD ? r : nb - 1 - r;
  if constexpr (kDF) {
    // The link is y_r = v_r - M_r y_j (j = r - 1 forward, r + 1 backward), with
    // v_r = W_r (b_r - the older blocks' products) formed before block j is solved and
    // M_r = W_r L_rj (forward) or W_r^T L_jr^T (backward) formed here at the start: one product
    // sits on the chain instead of two with a reduction between them.  Shared memory first holds
    // both factors of M_r as pairs ([m][i] and [m][k]), then this thread's pairs of W_r and M_r.
    extern __shared__ __align__(16) unsigned char dsm[];
    fpair* Wsp = reinterpret_cast<fpair*>(dsm);
    fpair* Lsp = Wsp + PB * PB;
    __shared__ int sWi[PB], sLk[PB];
    const int jl = FWD ? r - 1 : r + 1;         // the link's block (ndep > 0)
    int smr = 0;
    if (ndep > 0) {
      if (tid < PB) sWi[tid] = sLk[tid] = 0;
      __syncthreads();
      const int JL0 = jl * PB, jlrows = min(PB, n - JL0);
      T wvv[16], lvv[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + PT * u, ia = idx / PB, ib = idx % PB;
        wvv[u] = Wr[ia * PB + ib];              // W_r(ib, ia): operand (i, m) = (ib, ia) forward, (ia, ib) backward
        if (FWD) lvv[u] = (ib < rows && ia < jlrows) ? L[(size_t)(JL0 + ia) * ldl + R0 + ib] : 0.0;   // L_rj(m=ib, k=ia)
        else lvv[u] = (ia < rows && ib < jlrows) ? L[(size_t)(R0 + ia) * ldl + JL0 + ib] : 0.0;      // L_jr(k=ib, m=ia)
        const int ew = (int)(((unsigned long long)__double_as_longlong(wvv[u]) >> 52) & 0x7ff);
        const int el = (int)(((unsigned long long)__double_as_longlong(lvv[u]) >> 52) & 0x7ff);
        atomicMax(&sWi[FWD ? ib : ia], ew);
        atomicMax(&sLk[FWD ? ia : ib], el);
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + PT * u, ia = idx / PB, ib = idx % PB;
        const int iw = FWD ? ib : ia, mw = FWD ? ia : ib, kl = FWD ? ia : ib, ml = FWD ? ib : ia;
        const int ew = sWi[iw], el = sLk[kl];
        Wsp[mw * PB + iw] = split_scaled(wvv[u], ew == 0 ? 0 : ew - 1023);
        Lsp[ml * PB + kl] = split_scaled(lvv[u], el == 0 ? 0 : el - 1023);
      }
      __syncthreads();
      // M(i, k) for the 16 k of this thread's chunk: sum over m of W(i, m) L(m, k), the zero
      // triangle of W skipped by whole warps
      float ms[16], mc[16];
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) ms[kq] = mc[kq] = 0.0f;
      const int i0 = i & ~31;
      const int mlo = FWD ? 0 : i0, mhi = FWD ? min(PB, i0 + 32) : PB;
#pragma unroll 2
      for (int m = mlo; m < mhi; ++m) {
        const fpair w = Wsp[m * PB + i];
#pragma unroll
        for (int kq = 0; kq < 16; ++kq) dot2_step(ms[kq], mc[kq], w, Lsp[m * PB + ch * 16 + kq]);
      }
      const int swi = sWi[i] == 0 ? 0 : sWi[i] - 1023;
      T md[16];
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) {
        const int el = sLk[ch * 16 + kq], off = swi + (el == 0 ? 0 : el - 1023);
        md[kq] = widen_scaled(ms[kq], off) + widen_scaled(mc[kq], off);
      }
      smr = scale_of16(md);
      __syncthreads();                          // the factors are consumed
#pragma unroll
      for (int q = 0; q < 16; ++q) Lsp[q * PT + tid] = split_scaled(md[q], smr);
    }
    const int sw = scale_of16(wv);
#pragma unroll
    for (int q = 0; q < 16; ++q) Wsp[q * PT + tid] = split_scaled(wv[q], sw);

    // One loop body serves every product: steps it < nfar add the product with block j(it) to
    // acc (its factor entries fetched one step ahead), step nfar forms v_r, step nfar + 1 the
    // link.
    // The backward sweep's factor entries L_jr(k, i) lie along k in memory while a thread's
    // 16 run along k for one i: they are loaded coalesced (a warp along k), turned into pairs
    // there (the chunk scale by shuffles) and passed to their threads through Ps[k][i].
    const int nfar = max(ndep - 1, 0);
    constexpr int kPsLd = PB + 1;
    fpair* Ps = Lsp + PB * PB;                 // [k][i], ld kPsLd (backward)
    __shared__ int Psc[PB][PB / 16];           // scale of (i, chunk) (backward)
    T lv[16];
    fpair ap[16];
    int sa = 0;
    auto kind_of = [&](int it) { return it < nfar ? 0 : (it == nfar ? 1 : 2); };
    auto fetch = [&](int it) {
      if (it >= nfar) return;
      if (FWD) {
        load_l(it, lv);
      } else {
        const int J0 = (nb - 1 - it) * PB, jrows = min(PB, n - J0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int idx = tid + PT * u, ia = idx / PB, kb = idx % PB;
          lv[u] = (ia < rows && kb < jrows) ? L[(size_t)(R0 + ia) * ldl + J0 + kb] : 0.0;
        }
      }
    };
    auto stage = [&](int it) {                // backward: lv (fetched for step it) into Ps
      if constexpr (!FWD) {
        if (it >= nfar) return;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int idx = tid + PT * u, ia = idx / PB, kb = idx % PB;
          int sc;
          Ps[kb * kPsLd + ia] = split_chunk(lv[u], sc);
          if ((kb & 15) == 0) Psc[ia][kb >> 4] = sc;
        }
      }
    };
    auto to_pairs = [&](int kd) {
      if (kd == 0 && FWD) {
        sa = scale_of16(lv);
#pragma unroll
        for (int q = 0; q < 16; ++q) ap[q] = split_scaled(lv[q], sa);
      } else if (kd == 0) {
        sa = Psc[i][ch];
#pragma unroll
        for (int q = 0; q < 16; ++q) ap[q] = Ps[(ch * 16 + q) * kPsLd + i];
      } else {
        const fpair* src = kd == 1 ? Wsp : Lsp;
        sa = kd == 1 ? sw : smr;
#pragma unroll
        for (int q = 0; q < 16; ++q) ap[q] = src[q * PT + tid];
      }
    };
    T vr[kBU];
    fetch(0);
    stage(0);
    __syncthreads();
    to_pairs(kind_of(0));
#pragma unroll 1
    for (int it = 0; it <= ndep; ++it) {
      const int kd = kind_of(it);
      if (kd == 0) {
        fetch(it + 1);
        if (!await_block(FWD ? it : nb - 1 - it)) return;
      } else if (kd == 1) {
        // reduce the four chunks, subtract from the right-hand side
#pragma unroll
        for (int c = 0; c < NR; ++c)
          if (c < nrhs) part[ch][c][i] = acc[c];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kBU; ++u) {
          const int idx = tid + PT * u, ii = idx % PB, c = idx / PB;
          if (c >= nrhs) break;   // whole warps leave (and issue no FP64 work) here
          {
            int sv;
            vP[c][ii] = split_chunk(bpre[u] - ((part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii])), sv);
            if ((ii & 15) == 0) vsc[c][ii >> 4] = sv;
          }
        }
        __syncthreads();
      } else {
        if (!await_block(jl)) return;
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        if (c < nrhs) {
          const double d = dot16_df(ap, sa, &vP[c][ch * 16], vsc[c][ch]);
          if (kd == 0) acc[c] += d;
          else part[ch][c][i] = d;
        }
      }
      stage(it + 1);
      __syncthreads();
      if (kd == 1) {
#pragma unroll
        for (int u = 0; u < kBU; ++u) {
          const int idx = tid + PT * u, ii = idx % PB, c = idx / PB;
          if (c >= nrhs) break;   // the SM retires few FP64 warp instructions: idle warps issue none
          vr[u] = (part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii]);
        }
      }
      if (it < ndep) to_pairs(kind_of(it + 1));
    }
    // the block's solution: v_r less the link's product
#pragma unroll
    for (int u = 0; u < kBU; ++u) {
      const int idx = tid + PT * u, ii = idx % PB, c = idx / PB;
      if (c >= nrhs) break;
      if (ii < rows)
        publish(ii, c, ndep > 0 ? vr[u] - ((part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii])) : vr[u]);
    }
  } else {
    for (int jj = 0; jj < ndep; ++jj) {
      const int j = FWD ? jj : nb - 1 - jj;
      // this thread's 16 factor entries do not depend on the mailbox: load them first
      T lv[16];
      load_l(j, lv);
      if (!await_block(j)) return;
#pragma unroll
      for (int c = 0; c < NR; ++c) {
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
    for (int c = 0; c < NR; ++c)
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
    for (int c = 0; c < NR; ++c) {
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
      if (ii < rows) publish(ii, c, (double)((part[0][c][ii] + part[1][c][ii]) + (part[2][c][ii] + part[3][c][ii])));
    }
  }
}

template <typename T, int NR>
cudaError_t sweep_smem_attr(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(potrs_sweep_kernel<T, true, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(potrs_sweep_kernel<T, false, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <typename T, int NR>
cudaError_t launch_sweep(bool fwd, int nb, size_t dsmem, cudaStream_t s, const double* L, int ldl, const T* W, double* B,
                         int ldb, int n, int nc, int* ticket, double* mb, double* mb_next, int mbld, unsigned* err,
                         unsigned long long limit_ns) {
  if (fwd)
    potrs_sweep_kernel<T, true, NR><<<nb, PT, dsmem, s>>>(L, ldl, W, B, ldb, n, nc, ticket, mb, mb_next, mbld, err, limit_ns);
  else
    potrs_sweep_kernel<T, false, NR><<<nb, PT, dsmem, s>>>(L, ldl, W, B, ldb, n, nc, ticket, mb, mb_next, mbld, err, limit_ns);
  return cudaGetLastError();
}

template <typename T>
cudaError_t potrs_t(const double* L, int ldl, double* B, int ldb, int n, int nrhs, void* work, int* ticket,
                    unsigned* err, unsigned long long limit_ns, cudaStream_t s) {
  const int nb = (n + PB - 1) / PB;
  T* W = static_cast<T*>(work);
  // the mailboxes follow the inverses (sized for FP64 inverses in either precision)
  const int mbld = nb * PB;
  double* mbf = reinterpret_cast<double*>(static_cast<unsigned char*>(work) + (size_t)nb * PB * PB * sizeof(double));
  double* mbb = mbf + (size_t)MAX_RHS * mbld;
  const size_t smem = 2 * sizeof(T) * PB * (PB + 1);
  static unsigned long long attr_mask = 0;
  const unsigned long long attr_bit = dev_bit();
  cudaError_t e;
  // the FP64 sweeps stage both factors of M_r as pairs (2 x 64 x 64 x 8 bytes), then the
  // backward sweep's factor blocks (64 x 65 pairs)
  const size_t dsmem = sizeof(T) == sizeof(double) ? 2 * sizeof(float) * (2 * PB * PB + PB * (PB + 1)) : 0;
  if (!(attr_mask & attr_bit)) {
    if ((e = cudaFuncSetAttribute(potrs_diag_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    if (dsmem > 0) {
      if ((e = sweep_smem_attr<T, 1>((int)dsmem)) != cudaSuccess) return e;
      if ((e = sweep_smem_attr<T, 4>((int)dsmem)) != cudaSuccess) return e;
      if ((e = sweep_smem_attr<T, MAX_RHS>((int)dsmem)) != cudaSuccess) return e;
    }
    attr_mask |= attr_bit;
  }
  potrs_diag_inverse_kernel<T><<<nb, PT, smem, s>>>(L, ldl, n, W, mbf, mbld);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int c0 = 0; c0 < nrhs; c0 += MAX_RHS) {
    const int nc = nrhs - c0 < MAX_RHS ? nrhs - c0 : MAX_RHS;
    double* Bc = B + (size_t)c0 * ldb;
    for (int pass = 0; pass < 2; ++pass) {
      if ((e = cudaMemsetAsync(ticket, 0, sizeof(int), s)) != cudaSuccess) return e;
      double* mb = pass == 0 ? mbf : mbb;
      double* mb_next = pass == 0 ? mbb : mbf;
      if (nc == 1)
        e = launch_sweep<T, 1>(pass == 0, nb, dsmem, s, L, ldl, W, Bc, ldb, n, nc, ticket, mb, mb_next, mbld, err, limit_ns);
      else if (nc <= 4)
        e = launch_sweep<T, 4>(pass == 0, nb, dsmem, s, L, ldl, W, Bc, ldb, n, nc, ticket, mb, mb_next, mbld, err, limit_ns);
      else
        e = launch_sweep<T, MAX_RHS>(pass == 0, nb, dsmem, s, L, ldl, W, Bc, ldb, n, nc, ticket, mb, mb_next, mbld, err,
                                     limit_ns);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_potrs(const double* L, int ldl, double* B, int ldb, int n, int nrhs, bool fp32, void* work,
                         int* ticket, unsigned* dev_err, cudaStream_t s, unsigned long long wait_limit_ns) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (fp32) return potrs_t<float>(L, ldl, B, ldb, n, nrhs, work, ticket, dev_err, wait_limit_ns, s);
  return potrs_t<double>(L, ldl, B, ldb, n, nrhs, work, ticket, dev_err, wait_limit_ns, s);
}

cudaError_t launch_wait_probe(double* entry, unsigned long long limit_ns, unsigned* dev_err,
                              unsigned long long* waited_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(entry, limit_ns, dev_err, waited_ns);
  return cudaGetLastError();
}

// two sweeps per chunk of MAX_RHS columns (written without forming nrhs + MAX_RHS - 1)
int potrs_sweeps(int nrhs) { return 2 * (nrhs / MAX_RHS + (nrhs % MAX_RHS != 0)); }

}  // namespace hrp
