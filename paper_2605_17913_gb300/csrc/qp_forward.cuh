// qp_forward.cuh -- batched implicit-complementarity IPM (Alg. 1, Alg. 2).
// One CTA solves one QP.  On chip (kBig = false) every per-instance array
// lives in shared memory; the large-problem variant (kBig) keeps K, G, Y, C
// in a per-instance global workspace with 16-byte aligned rows, stages G'WG's
// rows and the back substitutions' factor blocks in shared memory by bulk
// copies, and reads the matrices in its residuals and products by coalesced
// warp row sweeps.  kCoh: the same solver run by the persistent serving
// kernel, which reads memory reused across requests through L2.
//
// Newton system.  eq. 14 (symmetric, every block bounded):
//   [ Q - G'G   G'     A' ] [dx]     [ rho1 ]   rho1 = r_t - G'(r_i + r_z - r_s)
//   [ G        -B_-    0  ] [dv] = - [ rho2 ]   rho2 = r_i - r_s - c r_kappa
//   [ A         0      0  ] [dy]     [ r_e  ]   B_+ = B_k(v), B_- = B_k(-v), c = 1/(b_k(v)+b_k(-v))
// Eliminating every dv would give K = Q + G'WG with W = B_+/B_- = z/s, whose
// entries grow like 1/kappa on active rows; FP32 Cholesky of it fails once
// kappa is near the tolerance.  Instead the rows are split by W:
//   inactive I = {W <= tau}: dv_I = (G_I dx + rho2_I) / B_-   (B_- >= 1/2 there),
//   active   A = {W >  tau}: keep lambda = dv_A - G_A dx, scaled by 1/B_+ (>= 1/2),
// which leaves the bounded saddle-point system (tau = 1 unless more than amax
// rows are active)
//   [ K_I   F'] [dx]   [ rhs1 ]     K_I = Q + G_I' W_I G_I  (W_I <= tau)
//   [ F    -D ] [mu] = [ rhs2 ]     F = [G_A; A],  D = diag(1/W_A, 0)  (1/W_A < 1/tau)
// with rhs1 = -rho1 - G_I' (rho2_I / B_-),  rhs2 = (-rho2_A / B_+, -r_e),  mu = (lambda, dy).
// K_I = L L' (Cholesky); Y = F L^-T and C = D + Y Y' come out of the same
// blocked bordered elimination; C = L_C L_C' (Cholesky, with a 1e-7 relative
// diagonal shift that keeps FP32 Cholesky defined when F is rank-deficient,
// i.e. on degenerate problems; Newton corrects the step, and the backward
// pass refines its solve against the unshifted system).
// Solve:  u = L^-1 rhs1,  C mu = Y u - rhs2,  dx = L^-T (u - Y' mu).
// Recovery (eq. 13 rows 4-5): dv_I as above, dv_A = lambda + G_A dx,
//   dz = -r_z + B_+ dv - c r_kappa,  ds = -r_s - B_- dv - c r_kappa,  dkappa = -r_kappa.
// In exact arithmetic this is eq. 14's solution; no W-sized number is formed.
//
// The right-hand sides are affine in r_kappa = kappa - kappa_target, so one
// pass over the factors solves the two columns (r_kappa = 0, d/dr_kappa):
// the predictor (kappa_target = 0 -> alpha_aff, mu_aff, Mehrotra sigma) and
// the corrector (kappa_target = max(sigma kappa, kappa_min)) then cost only
// vector work.  Step: alpha from eq. 7, x += a dx, y += a dy, v += a dv,
// kappa += a dkappa, z = b_k(v), s = b_k(-v) (retraction, eq. 11, App. C).
//
// Alg. 2 (relax) repeats the step with kappa_target = kappa_relax, then the
// system is factored once more at the relaxed point and the factors, W, the
// active-row map and the relaxed (x, y, z) go to the gradient cache (Alg. 3).
//
// The explicit-complementarity ablation (eq. 6 / eq. 8) uses W = z ./ s, a
// Mehrotra predictor-corrector (second solve for the corrector) and
// fraction-to-boundary 0.99, either through the same two-level factorisation
// (QP_STANDARD) or with eq. 8's Q + G' diag(z/s) G factored as it stands
// (QP_STANDARD_SCHUR: every row eliminated, no shift, no retry).
//
// Register budget: the layout lives in shared memory and each method forms
// only the addresses it uses, so that no pointer stays live across phases.
#pragma once
#include <mutex>

#include "qp_device.cuh"
#include "qp_internal.h"
#include "qp_tc.cuh"

namespace qpgpu {

namespace fwd {

constexpr int ST_SOLVED = 0, ST_MAX_ITER = 1, ST_STALLED = 2, ST_NUMERICAL = 3, ST_BAD_INPUT = 4;
constexpr float kCReg = 1e-7f;  // relative diagonal shift of C
constexpr float kStallMeasure = 1e-4f;  // Alg. 1 may end STALLED only below this measure
// Alg. 2 chord steps reuse a factorisation while each step cuts the relax
// measure at least this much (4x); a slower step means the frozen Newton
// matrix (W moves like z^2 / kappa on active rows) has drifted too far
constexpr float kChordRate = 0.25f;
constexpr int kStaticSmem = 1152;  // upper bound of the kernel's static shared memory (state + params)

struct FLayout {
  int n, m, p, amax, fmax;
  int ldk, ldg, ldx, ldc, nv, mv, pv, fv;
  int split;      // K, G, Y, C in a global workspace (large problems)
  int big_total;  // floats of K, G, Y, C
  int o_K, o_qd, o_G, o_Y, o_C, o_R, o_col, o_red, o_Pb;
  int o_q, o_x, o_rt, o_dinv, o_tn;
  int o_b, o_y, o_re;
  int o_cdinv, o_D, o_ua, o_ub, o_act;
  int o_h, o_z, o_s, o_ri, o_bz, o_bs, o_ea, o_eb, o_ta, o_tb, o_pos, o_ina;
  int o_rf;   // refinement of the folded solves (large variant): the saved
              // right-hand sides of both columns (2 nv + 2 fv floats)
  int o_rfs;  // its per-sweep scratch in the union region (4 nv + 2 fv floats)
  int o_wp;   // (large variant) per-warp column sums of the row sweeps over K,
              // G, A, in the union region (3 (NT / 32) nv floats)
  int total;
};

// The panel buffer Pb of the blocked factorisation is only live inside
// factor_once(), so it shares one region with col, ta, tb, eb and tn, which
// are dead there.
// Y and C carry two extra rows: the right-hand sides folded into the
// factorisation of an implicit step.
// Panel width of the blocked factorisation: 32 for the large variant (its
// trailing updates read and write global memory, so fewer passes pay: 16-wide
// +14-18 % over 8-wide at n = 256, 32-wide another 7 %), 8 on chip, where the
// wide diagonal-block factor (one warp, shuffles) lengthens the critical path
// more than the wider update saves (16-wide measured 40 % slower at n = 50).
__host__ __device__ constexpr int panel_width(int nthreads, bool split) {
  return (split || nthreads < 0) ? 32 : 8;
}

__host__ __device__ inline FLayout make_fwd_layout(int n, int m, int p, int amax, int nthreads,
                                                   bool split = false) {
  FLayout L;
  L.n = n; L.m = m; L.p = p; L.amax = amax; L.fmax = amax + p;
  // odd strides keep shared-memory rows and columns free of bank conflicts;
  // the large variant's K, Y, C live in global memory, where 16-byte aligned
  // rows (a multiple of 4 floats, odd in quarters) allow vector accesses
  L.ldk = split ? ld_vec(n) : ld_odd(n);
  L.ldg = ld_vec(n);
  L.ldx = round4(n);
  L.ldc = split ? ld_vec(L.fmax + 2) : ld_odd(L.fmax + 2);
  L.nv = round4(n); L.mv = round4(m > 0 ? m : 1); L.pv = round4(p > 0 ? p : 1);
  L.fv = round4(L.fmax > 0 ? L.fmax : 1);
  int o = 0;
  auto take = [&](int cnt) -> int { int r = o; o += round4(cnt); return r; };
  // the four matrices: first in shared memory, or (split) at the start of
  // the instance's global workspace, with the rest in shared memory from 0.
  // A (p x n) is read where the caller keeps it (L1 / L2), row stride n.
  L.o_K = take(n * L.ldk);
  L.o_G = take(m * L.ldg);
  L.o_Y = take((L.fmax + 2) * L.ldk);
  L.o_C = take((L.fmax + 2) * L.ldc);
  L.split = split ? 1 : 0;
  L.big_total = o;
  if (split) o = 0;
  L.o_qd = take(L.nv);
  L.o_R = take(2 * L.ldx);
  L.o_red = take(2 * (nthreads / 32) * kRedK);
  {
    // union: Pb | (col, ta, tb, eb, tn) | (large variant) the two tensor-core
    // staging buffers of G'WG, 128-byte aligned
    if (split) o = (o + 31) & ~31;
    const int base = o;
    const int pw = panel_width(nthreads, split);
    int pb = pw > 8 ? pbw_floats(pbw_rows(n, L.fmax + 2, pw), pw) + fb_floats(pw)
                    : pb_floats(n + L.fmax + 2 + 4);
    pb = round4(pb);
    if (split && pb < 2 * tc::stage_bytes(n, 4) / 4) pb = 2 * tc::stage_bytes(n, 4) / 4;
    // (large variant) the two 32-row buffers of the staged back substitutions
    if (split && pb < 64 * round4(n > L.fmax ? n : L.fmax)) pb = 64 * round4(n > L.fmax ? n : L.fmax);
    L.o_Pb = base;
    L.o_col = take(2 * nthreads);
    L.o_ta = take(L.mv); L.o_tb = take(L.mv); L.o_eb = take(L.mv);
    L.o_tn = take(L.nv);
    // (large variant) the refinement sweep's dx, mu and G't of both columns,
    // live only within a sweep, after the factorisation
    L.o_rfs = take(split ? 4 * L.nv + 2 * L.fv : 0);
    L.o_wp = take(split ? 3 * (nthreads / 32) * L.nv : 0);
    if (o < base + pb) o = base + pb;
  }
  L.o_q = take(L.nv); L.o_x = take(L.nv); L.o_rt = take(L.nv); L.o_dinv = take(L.nv);
  L.o_b = take(L.pv); L.o_y = take(L.pv); L.o_re = take(L.pv);
  L.o_cdinv = take(L.fv); L.o_D = take(L.fv); L.o_ua = take(L.fv); L.o_ub = take(L.fv);
  L.o_act = take(L.fv);
  L.o_h = take(L.mv); L.o_z = take(L.mv); L.o_s = take(L.mv); L.o_ri = take(L.mv);
  L.o_bz = take(L.mv); L.o_bs = take(L.mv);
  L.o_ea = take(L.mv);
  L.o_pos = take(L.mv);
  L.o_ina = take(L.mv);
  L.o_rf = take(split ? 2 * L.nv + 2 * L.fv : 0);
  L.total = o;
  return L;
}

// Per-CTA scalars kept in shared memory (static; the dynamic allocation must
// leave kStaticSmem bytes of the 227 KB per-CTA limit for it).
struct SharedState {
  FLayout L;
  long long t_mark;                // phase timers only
  unsigned long long* timers;      // phase timers only
  int a, nf;         // active rows, rows of F = a + p (set by partition())
  int ni;            // inactive rows (listed in ina)
  float* gbase;      // base of K, G, Y, C: the dynamic shared memory or the workspace
  const float* gA;   // this instance's A in the caller's memory (row stride n)
  uint64_t mbar[2];  // tensor-core G'WG: completion of the two staging buffers
  uint64_t mbar_g[2];  // FP32 G'WG (large variant): bulk copies of the two row buffers
  uint32_t tc_chunks, g_chunks;  // chunks committed through mbar / mbar_g (phase parity)
  uint32_t tmem;     // its TMEM base (large variant with gwg != 0)
  int tc_flag;       // a bounded wait ran out in the current G'WG
  int tc_bad;        // sticky: G'WG falls back to FP32 for the rest of the solve
  int async_lost;    // bulk copies may still be in flight after a bounded wait
  int diag;          // diagnostic bits of this instance (QP_DIAG_*)
  int nan_stage;     // first stage with a non-finite value (QP_STAGE_*), 0: none
  int in_relax;      // Alg. 2 (or the factorisation cached for Alg. 3) is running
  int all_inactive;  // eq. 8 as it stands: every row in K (QP_STANDARD_SCHUR)
  int refine;        // refinement sweeps of each folded solve (large variant)
  int gwg;           // 0 FP32, 1 TF32, 2 BF16 (tensor-core products, large variant)
  float chord_kappa;  // kappa of the factorisation that Alg. 2's chord steps reuse
  float qn, bn, hn;  // |q|, |b|, |h| (infinity norms)
};

// Phase timers (tracing facility, compiled only with -DQP_PHASE_TIMERS): thread
// 0 of each CTA adds the cycles between consecutive marks, taken at barrier
// boundaries, to the caller's counter array (qp_debug_set_phase_counters()).
enum Phase { PH_LOAD, PH_RESID, PH_PART, PH_RHS, PH_SYRK, PH_BORDER, PH_CCHOL, PH_SOLVE, PH_GDX,
             PH_STEP, PH_CACHE, PH_COUNT };
#ifdef QP_PHASE_TIMERS
#define QP_MARK(ph)                                                                    \
  do {                                                                                 \
    if (threadIdx.x == 0 && fwd_state.timers) {                                              \
      const long long now_ = clock64();                                                \
      atomicAdd(&fwd_state.timers[ph], (unsigned long long)(now_ - fwd_state.t_mark));             \
      fwd_state.t_mark = now_;                                                               \
    }                                                                                  \
  } while (0)
#else
#define QP_MARK(ph) do {} while (0)
#endif

// Per-CTA state at namespace scope.  The phases are noinline functions; they
// reach the layout, the scalars and the dynamic shared memory through fixed
// shared addresses, so nothing of the solver's state lives in local memory
// (which would miss in the small L1 left beside the shared-memory carve-out).
extern __shared__ __align__(16) float fwd_dyn[];   // the per-instance layout
static __shared__ SharedState fwd_state;
static __shared__ unsigned char fwd_parity[512];   // block_reduce buffer parity, per thread

// address of array `name` in the per-instance shared-memory layout; QP_BIG for
// the five matrices, which the large-problem variant keeps in global memory
#define QP_ARR(name) float* const name = fwd_dyn + fwd_state.L.o_##name
#define QP_BIG(name) float* const name = (kBig ? fwd_state.gbase : fwd_dyn) + fwd_state.L.o_##name
#define QP_IARR(name) int* const name = reinterpret_cast<int*>(fwd_dyn + fwd_state.L.o_##name)

// kCoh: the instance's data may sit in memory that other requests used
// earlier in the same kernel's lifetime (a persistent serving loop), which the
// read-only cache path does not see as changed: read it through L2 instead.
template <int NT, bool kBig, bool kCoh = false>
struct Solver {
  static constexpr int kPW = panel_width(NT, kBig);

  static __device__ __forceinline__ float ld_ro(const float* ptr) {
    if constexpr (kCoh) return __ldcg(ptr);
    else return __ldg(ptr);
  }

  // The bulk-copy and tensor-core barriers and their chunk counters, once per
  // CTA (their phases follow from the counts); ends with a barrier.
  static __device__ void init_async() {
    if (threadIdx.x == 0) {
      fwd_state.tc_chunks = 0;
      fwd_state.g_chunks = 0;
      fwd_state.tmem = 0;
      tc::mbar_init(&fwd_state.mbar[0], 1);
      tc::mbar_init(&fwd_state.mbar[1], 1);
      tc::mbar_init(&fwd_state.mbar_g[0], 1);
      tc::mbar_init(&fwd_state.mbar_g[1], 1);
      tc::fence_mbar_init();
    }
    __syncthreads();
  }

  // keep_async: a CTA that solves several instances in turn keeps the
  // barriers, chunk counters and TMEM of init_async (never re-initialised
  // while valid).
  static __device__ void init(int n, int m, int p, int amax, float* ws, int gwg, int refine,
                              bool keep_async = false) {
    if (threadIdx.x == 0) {
      fwd_state.L = make_fwd_layout(n, m, p, amax, NT, kBig);
      fwd_state.gbase = kBig ? ws : fwd_dyn;
      fwd_state.gwg = kBig ? gwg : 0;
      fwd_state.tc_flag = 0;
      fwd_state.tc_bad = 0;
      fwd_state.async_lost = 0;
      fwd_state.diag = 0;
      fwd_state.nan_stage = 0;
      fwd_state.in_relax = 0;
      fwd_state.all_inactive = 0;
      fwd_state.refine = kBig ? refine : 0;
      if (!keep_async) {
        fwd_state.tc_chunks = 0;
        fwd_state.g_chunks = 0;
        fwd_state.tmem = 0;
        if (kBig) {
          // the bulk-copy and tensor-core barriers, once per CTA (their phases
          // follow from the chunk counts above)
          tc::mbar_init(&fwd_state.mbar[0], 1);
          tc::mbar_init(&fwd_state.mbar[1], 1);
          tc::mbar_init(&fwd_state.mbar_g[0], 1);
          tc::mbar_init(&fwd_state.mbar_g[1], 1);
          tc::fence_mbar_init();
        }
      }
      fwd_state.a = 0;
      fwd_state.nf = p;
      fwd_state.chord_kappa = 0.f;
      fwd_state.t_mark = clock64();
      fwd_state.timers = nullptr;
    }
    fwd_parity[threadIdx.x] = 0;
    __syncthreads();
  }

  // block reduction with this thread's buffer parity kept in shared memory
  template <int K, class Op>
  static __device__ __forceinline__ void reduce(float (&v)[K], float* red, Op op) {
    int parity = fwd_parity[threadIdx.x];
    block_reduce<NT, K>(v, red, parity, op);
    fwd_parity[threadIdx.x] = (unsigned char)parity;
  }

  // diagnostics: if any thread saw a non-finite value (`bad`), record `stage`
  // as the instance's first such stage (Alg. 2 as a whole counts as the relax
  // stage).  A block-wide vote, made only when the caller registered a
  // diagnostics array (uniform over the CTA).
  static __device__ void trace(const FwdParams& P, int stage, bool bad) {
    if (!P.diag) return;
    if (__syncthreads_or(bad ? 1 : 0) && threadIdx.x == 0 && fwd_state.nan_stage == 0)
      fwd_state.nan_stage = fwd_state.in_relax ? QP_STAGE_RELAX : stage;
  }

  // bad = some entry of v[0 .. len) is not finite
  static __device__ __forceinline__ bool any_nonfinite(const float* v, int len) {
    bool bad = false;
    for (int i = threadIdx.x; i < len; i += NT) bad |= !isfinite(v[i]);
    return bad;
  }

  // trace the Newton matrix's diagonal (W of the inactive rows, 1/W of the
  // active ones) right after partition().  The checks are out of line so that
  // the solve's hot loop (instruction-cache bound on chip) only carries a
  // branch and a call.
  static __device__ __noinline__ void trace_scaling_nl(const FwdParams& P) {
    QP_ARR(ea); QP_ARR(D); QP_IARR(pos);
    bool bad = false;
    for (int r = threadIdx.x; r < fwd_state.L.m; r += NT) {
      const float wv = pos[r] < 0 ? ea[r] : D[pos[r]];
      bad |= !(isfinite(wv) && wv >= 0.f);
    }
    trace(P, QP_STAGE_SCALING, bad);
  }
  static __device__ __forceinline__ void trace_scaling(const FwdParams& P) {
    if (P.diag) trace_scaling_nl(P);
  }

  // a factorisation failed: the predictor stage (its first use), flagged
  static __device__ void trace_factor_failed(const FwdParams& P) {
    if (threadIdx.x == 0) fwd_state.diag |= QP_DIAG_FACTOR_FAILED;
    trace(P, QP_STAGE_PREDICTOR, true);
  }

  // the iterate after a step
  static __device__ __noinline__ void trace_iterate_nl(const FwdParams& P, int stage) {
    QP_ARR(x); QP_ARR(z); QP_ARR(s); QP_ARR(y);
    const bool bad = any_nonfinite(x, fwd_state.L.n) || any_nonfinite(z, fwd_state.L.m) ||
                     any_nonfinite(s, fwd_state.L.m) || any_nonfinite(y, fwd_state.L.p);
    trace(P, stage, bad);
  }
  static __device__ __forceinline__ void trace_iterate(const FwdParams& P, int stage) {
    if (P.diag) trace_iterate_nl(P, stage);
  }

  // the implicit step's two solved columns (predictor stage)
  static __device__ __noinline__ void trace_folded_solve(const FwdParams& P) {
    QP_ARR(R); QP_ARR(ua); QP_ARR(ub); QP_ARR(ea); QP_ARR(eb);
    const FLayout& L = fwd_state.L;
    const bool bad = any_nonfinite(R, L.n) || any_nonfinite(R + L.ldx, L.n) ||
                     any_nonfinite(ua, fwd_state.nf) || any_nonfinite(ub, fwd_state.nf) ||
                     any_nonfinite(ea, L.m) || any_nonfinite(eb, L.m);
    trace(P, QP_STAGE_PREDICTOR, bad);
  }

  // the implicit step's corrector direction (ds, dz, dv on every row, dx)
  static __device__ __noinline__ void trace_corrector(const FwdParams& P, float rk) {
    QP_ARR(R);
    const FLayout& L = fwd_state.L;
    bool bad = false;
    for (int r = threadIdx.x; r < L.m; r += NT) {
      float dsr, dzr, dvr;
      implicit_dir<false>(r, rk, dsr, dzr, dvr);
      bad |= !isfinite(dsr) || !isfinite(dzr) || !isfinite(dvr);
    }
    for (int i = threadIdx.x; i < L.n; i += NT) bad |= !isfinite(fmaf(rk, R[L.ldx + i], R[i]));
    trace(P, QP_STAGE_CORRECTOR, bad);
  }

  // ---- load one instance; Q's strict upper triangle goes to K's upper part ----
  // Returns false if some datum is not finite.
  static __device__ __noinline__ bool load(const FwdParams& P, int bi) {
    const FLayout& L = fwd_state.L;
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    QP_BIG(K); QP_ARR(qd); QP_BIG(G); QP_ARR(q); QP_ARR(b); QP_ARR(h); QP_ARR(red);
    for (int i = t; i < L.total; i += NT) fwd_dyn[i] = 0.0f;
    if (kBig)
      for (int i = t; i < L.big_total; i += NT) fwd_state.gbase[i] = 0.0f;
    __syncthreads();
    const float* gQ = P.Q + (size_t)bi * n * n;
    const float* gG = P.G + (size_t)bi * m * n;
    const float* gA = P.A + (size_t)bi * p * n;
    float chk = 0.f;
    for (int e = t; e < n * n; e += NT) {
      const int r = e / n, c = e - r * n;
      if (c < r) continue;  // the solver reads the upper triangle of the symmetric Q
      const float v = gQ[e];
      chk = isfinite(v) ? chk : 1.0f;
      if (c == r) qd[r] = v; else K[r * L.ldk + c] = v;
    }
    for (int e = t; e < m * n; e += NT) {
      const int r = e / n, c = e - r * n;
      const float v = gG[e];
      chk = isfinite(v) ? chk : 1.0f;
      G[r * L.ldg + c] = v;
    }
    // the workspace copy of G is read by bulk copies (async proxy) later
    if (kBig) tc::fence_async_global();
    for (int e = t; e < p * n; e += NT) chk = isfinite(gA[e]) ? chk : 1.0f;
    if (t == 0) fwd_state.gA = gA;  // A stays in the caller's memory
    float lq = 0.f, lb = 0.f, lh = 0.f;
    for (int i = t; i < n; i += NT) {
      const float v = P.q[(size_t)bi * n + i];
      q[i] = v; lq = fmaxf(lq, fabsf(v)); chk = isfinite(v) ? chk : 1.0f;
    }
    for (int i = t; i < p; i += NT) {
      const float v = P.b[(size_t)bi * p + i];
      b[i] = v; lb = fmaxf(lb, fabsf(v)); chk = isfinite(v) ? chk : 1.0f;
    }
    for (int i = t; i < m; i += NT) {
      const float v = P.h[(size_t)bi * m + i];
      h[i] = v; lh = fmaxf(lh, fabsf(v)); chk = isfinite(v) ? chk : 1.0f;
    }
    float v[4] = {chk, lq, lb, lh};
    reduce<4>(v, red, OpMax());
    if (t == 0) { fwd_state.qn = v[1]; fwd_state.bn = v[2]; fwd_state.hn = v[3]; }
    __syncthreads();
    QP_MARK(PH_LOAD);
    return v[0] == 0.0f;
  }

  // ---- split rows by W = bz/bs; build F = [G_A; A], D, C = diag(D) and the
  // SYRK weights (W on inactive rows, 0 on active rows, in ea) ----
  static __device__ __noinline__ void partition() {
    const FLayout& L = fwd_state.L;
    const int m = L.m, p = L.p, n = L.n, t = threadIdx.x, w = t >> 5, lane = t & 31;
    QP_ARR(bz); QP_ARR(bs); QP_ARR(red); QP_BIG(G); QP_BIG(Y);
    const float* const A = fwd_state.gA;
    QP_BIG(C); QP_ARR(D); QP_ARR(ea); QP_IARR(act); QP_IARR(pos); QP_IARR(ina);
    (void)red;
    // one warp: tau = 1 unless more than amax rows have W > tau (then tau
    // grows tenfold until they fit), and the ordered compaction of the rows
    if (w == 0) {
      float tau = fwd_state.all_inactive ? INFINITY : 1.0f;
      for (int round = 0; round < 40 && tau < INFINITY; ++round) {
        int cnt = 0;
        for (int r0 = 0; r0 < m; r0 += 32) {
          const int r = r0 + lane;
          cnt += __popc(__ballot_sync(kFull, r < m && bz[r] > tau * bs[r]));
        }
        if (cnt <= L.amax) break;
        tau *= 10.0f;
      }
      int base = 0, ibase = 0;
      for (int r0 = 0; r0 < m; r0 += 32) {
        const int r = r0 + lane;
        const bool on = r < m && bz[r] > tau * bs[r];
        const unsigned mask = __ballot_sync(kFull, on);
        const int k = base + __popc(mask & ((1u << lane) - 1u));
        const bool keep = on && k < L.amax;  // always true after the tau loop; keeps act[] in bounds
        const bool off = r < m && !keep;
        const unsigned imask = __ballot_sync(kFull, off);
        if (r < m) pos[r] = keep ? k : -1;
        if (keep) act[k] = r;
        if (off) ina[ibase + __popc(imask & ((1u << lane) - 1u))] = r;
        base += __popc(mask);
        ibase += __popc(imask);
      }
      if (lane == 0) {
        fwd_state.a = min(base, L.amax);
        fwd_state.nf = fwd_state.a + p;
        fwd_state.ni = ibase;
      }
    }
    __syncthreads();
    const int a = fwd_state.a, nf = fwd_state.nf;
    for (int k = w; k < nf; k += NT / 32) {
      const float* src = k < a ? G + act[k] * L.ldg : A + (k - a) * n;
      const float dk = k < a ? bs[act[k]] / bz[act[k]] : 0.f;
      if constexpr (kBig) {
        // the whole row is loaded before it is stored (src may alias Y as
        // far as the compiler knows, which would serialise the round trips)
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = lane + 32 * j < n ? src[lane + 32 * j] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (lane + 32 * j < n) Y[k * L.ldk + lane + 32 * j] = v[j];
      } else {
        // likewise on chip (n <= 128): an equality row comes from the caller's
        // A in global memory, whose round trips would otherwise be serialised
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = lane + 32 * j < n ? src[lane + 32 * j] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (lane + 32 * j < n) Y[k * L.ldk + lane + 32 * j] = v[j];
      }
      for (int c = lane; c <= k; c += 32) C[k * L.ldc + c] = c == k ? dk : 0.f;
      if (lane == 0) D[k] = dk;
    }
    for (int r = t; r < m; r += NT) ea[r] = pos[r] < 0 ? bz[r] / bs[r] : 0.f;
    __syncthreads();
    QP_MARK(PH_PART);
  }

  // ---- fold the two right-hand sides of an implicit step into the border:
  // Y rows nf, nf+1 <- r1 (columns A, B) and C rows nf, nf+1 <- -rhs2, so that
  // the factorisation leaves u = L^-1 r1 in Y and w = L_C^-1 (Y u - rhs2) in C.
  static __device__ void fold_rhs() {
    const FLayout& L = fwd_state.L;
    QP_ARR(R); QP_BIG(Y); QP_BIG(C); QP_ARR(ua); QP_ARR(ub);
    const int n = L.n, nf = fwd_state.nf, t = threadIdx.x;
    if (kBig && fwd_state.refine > 0) {
      // keep both columns' right-hand sides for the refinement sweeps
      QP_ARR(rf);
      float* const r1s = rf;
      float* const r2s = rf + 2 * L.nv;
      for (int e = t; e < 2 * n; e += NT) {
        const int c = e / n, i = e - c * n;
        r1s[c * L.nv + i] = R[c * L.ldx + i];
      }
      for (int e = t; e < 2 * nf; e += NT) {
        const int c = e / nf, k = e - c * nf;
        r2s[c * L.fv + k] = (c == 0 ? ua : ub)[k];
      }
    }
    for (int e = t; e < 2 * n; e += NT) {
      const int c = e / n, i = e - c * n;
      Y[(nf + c) * L.ldk + i] = R[c * L.ldx + i];
    }
    for (int e = t; e < 2 * (nf + 2); e += NT) {
      const int c = e / (nf + 2), k = e - c * (nf + 2);
      C[(nf + c) * L.ldc + k] = k < nf ? -(c == 0 ? ua : ub)[k] : 0.f;
    }
    __syncthreads();
  }

  // ---- factor K_I and the bordered block.  F, D and C = D must have just
  // been set by partition() (and the right-hand sides by fold_rhs() when
  // nfold = 2): the elimination overwrites them. ----
  static __device__ __noinline__ bool factor_once(float creg, int nfold) {
    const FLayout& L = fwd_state.L;
    QP_BIG(K); QP_ARR(qd); QP_BIG(G); QP_ARR(ea); QP_BIG(Y); QP_BIG(C); QP_ARR(dinv);
    QP_ARR(cdinv); QP_ARR(Pb); QP_ARR(red); QP_IARR(ina);
    const int nf = fwd_state.nf;
    bool tc_done = false;
    if constexpr (kBig) {
      if (fwd_state.gwg != 0 && !fwd_state.tc_bad) {
        char* stage = reinterpret_cast<char*>(fwd_dyn + L.o_Pb);  // dead during the factorisation
        const int ni = fwd_state.ni;
        const uint32_t tm = fwd_state.tmem;
        tc_done = fwd_state.gwg == 2
                      ? tc::syrk_gwg_tc<NT, true>(K, L.ldk, qd, G, L.ldg, ea, ina, ni, L.n, stage,
                                                  fwd_state.mbar, &fwd_state.tc_chunks, tm,
                                                  &fwd_state.tc_flag)
                      : tc::syrk_gwg_tc<NT, false>(K, L.ldk, qd, G, L.ldg, ea, ina, ni, L.n,
                                                   stage, fwd_state.mbar, &fwd_state.tc_chunks,
                                                   tm, &fwd_state.tc_flag);
        if (!tc_done && threadIdx.x == 0) {
          fwd_state.tc_bad = 1;
          fwd_state.diag |= QP_DIAG_TC_FALLBACK;
        }
      }
      if (!tc_done && !fwd_state.async_lost) {
        // FP32 products from rows staged in shared memory by bulk copies
        float* stage = fwd_dyn + L.o_Pb;  // dead during the factorisation
#ifdef QP_PHASE_TIMERS
        unsigned long long* const ssub = fwd_state.timers ? fwd_state.timers + PH_COUNT + 8 : nullptr;
#else
        unsigned long long* const ssub = nullptr;
#endif
        if constexpr (NT == 512)
          tc_done = tc::syrk_gwg_staged_blocks<NT>(K, L.ldk, qd, G, L.ldg, ea, ina, fwd_state.ni,
                                                   L.n, stage, fwd_state.mbar_g,
                                                   &fwd_state.g_chunks, &fwd_state.tc_flag,
                                                   &fwd_state.async_lost, ssub);
        else
          tc_done = tc::syrk_gwg_staged<NT>(K, L.ldk, qd, G, L.ldg, ea, ina, fwd_state.ni, L.n,
                                            stage, fwd_state.mbar_g, &fwd_state.g_chunks,
                                            &fwd_state.tc_flag, &fwd_state.async_lost, ssub);
        if (!tc_done && threadIdx.x == 0) fwd_state.diag |= QP_DIAG_STAGE_FALLBACK;
        __syncthreads();
      }
    }
    if (!tc_done) syrk_gwg<NT>(K, L.ldk, qd, G, L.ldg, ea, ina, fwd_state.ni, L.n);
    QP_MARK(PH_SYRK);
#ifdef QP_PHASE_TIMERS
    unsigned long long* const sub = fwd_state.timers ? fwd_state.timers + PH_COUNT : nullptr;
#else
    unsigned long long* const sub = nullptr;
#endif
    // tracing builds: counters 11-14 (K, C: panel / trailing), 24-27 and
    // 40-43 (K, C: inside the wide panel), 32-34 and 48-50 (K, C: the panel
    // solve's own row / store / wait), 28-31 and 44-47 (K, C: the
    // look-ahead), 19-23 (staged G'WG); 64 counters
    bool ok = blocked_cholesky_bordered<NT, kPW>(K, L.ldk, L.n, Y, L.ldk, nf + nfold, C, L.ldc, dinv,
                                            Pb, sub, sub ? sub + 13 : nullptr);
    QP_MARK(PH_BORDER);
    if (nf > 0) {
      float dm[1] = {1.0f};
      for (int k = threadIdx.x; k < nf; k += NT) dm[0] = fmaxf(dm[0], C[k * L.ldc + k]);
      reduce<1>(dm, red, OpMax());
      const float shift = creg * dm[0];
      for (int k = threadIdx.x; k < nf; k += NT) C[k * L.ldc + k] += shift;
      __syncthreads();
      ok = blocked_cholesky_bordered<NT, kPW>(C, L.ldc, nf, C + nf * L.ldc, L.ldc, nfold, nullptr, 0,
                                         cdinv, Pb, sub ? sub + 2 : nullptr,
                                         sub ? sub + 29 : nullptr) && ok;
      QP_MARK(PH_CCHOL);
    }
    return ok;
  }

  // factor; if FP32 Cholesky of C meets a non-positive pivot (rank-deficient
  // F), redo the partition and factorisation with a 100x, then 10^4x larger shift.
  static __device__ bool factor(int nfold = 0) {
    // eq. 8 as it stands: one attempt, no shift of the equality block
    if (fwd_state.all_inactive) return factor_once(0.0f, nfold);
    float creg = kCReg;
    for (int attempt = 0; attempt < 3; ++attempt, creg *= 100.0f) {
      if (attempt > 0) {
        partition();
        if (nfold) fold_rhs();
      }
      if (factor_once(creg, nfold)) return true;
    }
    return false;
  }

  // ---- finish a folded solve: mu = L_C^-T w, dx = L^-T (u - Y' mu) for both
  // columns; dx returned in R rows 0, 1 and mu in ua / ub ----
  static __device__ void solve_folded() {
    const FLayout& L = fwd_state.L;
    QP_BIG(K); QP_ARR(dinv); QP_ARR(R); QP_BIG(Y); QP_BIG(C); QP_ARR(ua); QP_ARR(ub);
    const int n = L.n, t = threadIdx.x, w = t >> 5, nf = fwd_state.nf;
    if (nf > 0) {
      if constexpr (kBig) {
        // L_C in global memory: blocked solve with every warp
        QP_ARR(cdinv);
        for (int e = t; e < 2 * nf; e += NT) {
          const int c = e / nf, k = e - c * nf;
          (c == 0 ? ua : ub)[k] = C[(nf + c) * L.ldc + k];
        }
        __syncthreads();
        upper_solve_big(C, L.ldc, cdinv, nf, ua, ub);
      } else {
        // one warp per column (both columns in turn with a single warp)
        for (int c = w; c < 2; c += NT / 32) {
          float* u = c == 0 ? ua : ub;
          const float* wrow = C + (nf + c) * L.ldc;
          for (int k = t & 31; k < nf; k += 32) u[k] = wrow[k];
          __syncwarp();
          c_solve_n(u, nf, true);
        }
        __syncthreads();
      }
    }
    if constexpr (kBig) {
      // Y in global memory: Y'u for both columns in one coalesced sweep over
      // Y's rows (per-warp column sums, added in warp order)
      QP_ARR(wp);
      constexpr int nw = NT / 32;
      const float* cw[2] = {ua, ub};
      warp_rows_n<NT, 4, 0, 2, false, false>(Y, L.ldk, nf, n, nullptr, nullptr, cw, wp, L.nv);
      __syncthreads();
      for (int e = t; e < 2 * n; e += NT) {
        const int c = e / n, i = e - c * n;
        const float* pk = wp + c * nw * L.nv;
        float acc = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) acc += pk[w2 * L.nv + i];
        R[c * L.ldx + i] = Y[(nf + c) * L.ldk + i] - acc;
      }
    } else {
      for (int e = t; e < 2 * n; e += NT) {
        const int c = e / n, i = e - c * n;
        const float* u = c == 0 ? ua : ub;
        float acc = Y[(nf + c) * L.ldk + i];
        for (int k = 0; k < nf; ++k) acc = fmaf(-Y[k * L.ldk + i], u[k], acc);
        R[c * L.ldx + i] = acc;
      }
    }
    __syncthreads();
    if constexpr (kBig)
      upper_solve_big(K, L.ldk, dinv, n, R, R + L.ldx);
    else
      solve_rows<NT, true, 4>(K, L.ldk, dinv, n, R, L.ldx, 0, 2);
    QP_MARK(PH_SOLVE);
  }

  // (large variant) back substitution with a factor in the workspace: its
  // 32-row blocks staged in shared memory by bulk copies (the union region is
  // dead here), or read in place once bulk copies are no longer trusted
  static __device__ void upper_solve_big(const float* Lf, int ld, const float* di, int nn,
                                         float* x0, float* x1) {
    if (!fwd_state.async_lost) {
      float* const stage = fwd_dyn + fwd_state.L.o_Pb;
      const bool all = tc::block_trsv_upper_staged<NT>(Lf, ld, di, nn, x0, x1, stage, round4(nn),
                                                       fwd_state.mbar_g, &fwd_state.g_chunks,
                                                       &fwd_state.tc_flag, &fwd_state.async_lost);
      if (!all && threadIdx.x == 0) fwd_state.diag |= QP_DIAG_STAGE_FALLBACK;
    } else {
      block_trsv<NT, true>(Lf, ld, di, nn, x0, x1);
    }
  }

  // warp solve with C for nf rows (up to 128, on chip)
  // (on chip only; the large variant solves with L_C by block_trsv)
  static __device__ void c_solve_n(float* u, int nf, bool upper_only) {
    if (nf <= 32) c_solve<1>(u, nf, upper_only);
    else if (nf <= 64) c_solve<2>(u, nf, upper_only);
    else if (nf <= 96) c_solve<3>(u, nf, upper_only);
    else c_solve<4>(u, nf, upper_only);
  }

  template <int SP>
  static __device__ void c_solve(float* v, int nf, bool upper_only = false) {
    const FLayout& L = fwd_state.L;
    QP_BIG(C); QP_ARR(cdinv);
    const int lane = threadIdx.x & 31;
    float r[1][SP];
#pragma unroll
    for (int s2 = 0; s2 < SP; ++s2) {
      const int i = lane + 32 * s2;
      r[0][s2] = i < nf ? v[i] : 0.f;
    }
    if (!upper_only) warp_lower_solve<SP, 1>(C, L.ldc, cdinv, nf, r);
    warp_upper_solve<SP, 1>(C, L.ldc, cdinv, nf, r);
#pragma unroll
    for (int s2 = 0; s2 < SP; ++s2) {
      const int i = lane + 32 * s2;
      if (i < nf) v[i] = r[0][s2];
    }
  }

  // ---- solve [K_I F'; F -D] (dx, mu) = (rhs1, rhs2) for columns slot0..slot0+nrhs-1 ----
  // rhs1 in R rows, rhs2 in ua (column 0) / ub (column 1); dx returned in R, mu in ua / ub.
  static __device__ __noinline__ void solve(int slot0, int nrhs) {
    const FLayout& L = fwd_state.L;
    QP_BIG(K); QP_ARR(dinv); QP_ARR(R); QP_BIG(Y); QP_ARR(ua); QP_ARR(ub);
    const int n = L.n, t = threadIdx.x, w = t >> 5, nf = fwd_state.nf;
    float* const r0 = R + slot0 * L.ldx;
    float* const r1 = nrhs == 2 ? R + (slot0 + 1) * L.ldx : nullptr;
    if constexpr (kBig)
      block_trsv<NT, false>(K, L.ldk, dinv, n, r0, r1);
    else
      solve_rows<NT, false, 4>(K, L.ldk, dinv, n, R, L.ldx, slot0, nrhs);
    if (nf > 0) {
      for (int e = t; e < nf * nrhs; e += NT) {
        const int k = e % nf, cc = slot0 + e / nf;
        float* u = cc == 0 ? ua : ub;
        const float* yk = Y + k * L.ldk;
        const float* rr = R + cc * L.ldx;
        float acc = 0.f;
        if constexpr (kBig) {
#pragma unroll 8
          for (int i = 0; i < n; ++i) acc = fmaf(yk[i], rr[i], acc);
        } else {
          for (int i = 0; i < n; ++i) acc = fmaf(yk[i], rr[i], acc);
        }
        u[k] = acc - u[k];
      }
      __syncthreads();
      if constexpr (kBig) {
        QP_ARR(cdinv); QP_BIG(C);
        float* const u0 = slot0 == 0 ? ua : ub;
        float* const u1 = nrhs == 2 ? ub : nullptr;
        block_trsv<NT, false>(C, L.ldc, cdinv, nf, u0, u1);
        block_trsv<NT, true>(C, L.ldc, cdinv, nf, u0, u1);
      } else {
        for (int c = w; c < nrhs; c += NT / 32) {
          float* u = (slot0 + c) == 0 ? ua : ub;
          c_solve_n(u, nf, false);
        }
        __syncthreads();
      }
      for (int e = t; e < n * nrhs; e += NT) {
        const int i = e % n, cc = slot0 + e / n;
        const float* u = cc == 0 ? ua : ub;
        float acc = R[cc * L.ldx + i];
        if constexpr (kBig) {
#pragma unroll 8
          for (int k = 0; k < nf; ++k) acc = fmaf(-Y[k * L.ldk + i], u[k], acc);
        } else {
          for (int k = 0; k < nf; ++k) acc = fmaf(-Y[k * L.ldk + i], u[k], acc);
        }
        R[cc * L.ldx + i] = acc;
      }
      __syncthreads();
    }
    if constexpr (kBig)
      block_trsv<NT, true>(K, L.ldk, dinv, n, r0, r1);
    else
      solve_rows<NT, true, 4>(K, L.ldk, dinv, n, R, L.ldx, slot0, nrhs);
    QP_MARK(PH_SOLVE);
  }

  // e = G dx for the solved columns (ea for column 0, eb for column 1)
  static __device__ __noinline__ void g_times_dx(int slot0, int nrhs) {
    const FLayout& L = fwd_state.L;
    QP_BIG(G); QP_ARR(R); QP_ARR(ea); QP_ARR(eb);
    if constexpr (kBig) {
      // G in global memory: coalesced row sweep, a warp per four rows
      if (nrhs == 2) {
        const float* xv[2] = {R, R + L.ldx};
        float* dv[2] = {ea, eb};
        warp_rows_n<NT, 4, 2, 0, false, false>(G, L.ldg, L.m, L.n, xv, dv, nullptr, nullptr, 0);
      } else {
        const float* xv[1] = {R + slot0 * L.ldx};
        float* dv[1] = {slot0 == 0 ? ea : eb};
        warp_rows_n<NT, 4, 1, 0, false, false>(G, L.ldg, L.m, L.n, xv, dv, nullptr, nullptr, 0);
      }
    } else {
      for (int r = threadIdx.x; r < L.m; r += NT) {
        if (nrhs == 2) {
          float u, v;
          row_dot2(G, L.ldg, r, R, R + L.ldx, L.nv, u, v);
          ea[r] = u;
          eb[r] = v;
        } else {
          (slot0 == 0 ? ea : eb)[r] = row_dot(G, L.ldg, r, R + slot0 * L.ldx, L.nv);
        }
      }
    }
    __syncthreads();
    QP_MARK(PH_GDX);
  }

  // ---- one iterative-refinement sweep of a folded solve (large variant):
  // the residual of the bounded system
  //   r1 = rhs1 - (K_I dx + F' mu),  r2 = rhs2 - (F dx - D mu),
  // K_I dx = Q dx + G_I' W_I (G_I dx) and F' mu = G_A' mu_A + A' mu_eq formed in
  // FP32 from Q, G, A (not from the factorised matrix, whose G'WG may carry
  // TF32 / BF16 products and whose C carries the small diagonal shift), then
  // the correction from the same factors; both columns.  Needs e = G dx of
  // the current solution in ea / eb, and leaves them updated. ----
  static __device__ __noinline__ void refine_folded() {
    const FLayout& L = fwd_state.L;
    QP_BIG(K); QP_ARR(qd); QP_BIG(G); QP_ARR(R); QP_ARR(ua); QP_ARR(ub); QP_ARR(ea);
    QP_ARR(eb); QP_ARR(bz); QP_ARR(bs); QP_ARR(D); QP_ARR(ta); QP_ARR(tb); QP_ARR(col);
    QP_ARR(rf); QP_ARR(rfs); QP_IARR(pos); QP_IARR(act);
    const float* const A = fwd_state.gA;
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x, a = fwd_state.a, nf = fwd_state.nf;
    float* const dx = rfs;                  // 2 nv: the solution's dx, both columns
    float* const mu = rfs + 2 * L.nv;       // 2 fv: its mu
    float* const u = mu + 2 * L.fv;         // 2 nv: G't
    const float* const r1s = rf;            // 2 nv: rhs1 (fold_rhs)
    const float* const r2s = rf + 2 * L.nv; // 2 fv: rhs2
    for (int e = t; e < 2 * n; e += NT) {
      const int c = e / n, i = e - c * n;
      dx[c * L.nv + i] = R[c * L.ldx + i];
    }
    for (int e = t; e < 2 * nf; e += NT) {
      const int c = e / nf, k = e - c * nf;
      mu[c * L.fv + k] = (c == 0 ? ua : ub)[k];
    }
    // the G' coefficients: W e on inactive rows (K_I), mu on active rows (F')
    for (int r = t; r < m; r += NT) {
      const int k = pos[r];
      if (k < 0) {
        const float w = bz[r] / bs[r];
        ta[r] = w * ea[r];
        tb[r] = w * eb[r];
      } else {
        ta[r] = ua[k];
        tb[r] = ub[k];
      }
    }
    __syncthreads();
    {
      const float* vv[2] = {ta, tb};
      float* oo[2] = {u, u + L.nv};
      col_dot<NT, 2>(G, L.ldg, m, n, vv, oo, col);
    }
    for (int e = t; e < 2 * n; e += NT) {
      const int c = e / n, i = e - c * n;
      const float* x = dx + c * L.nv;
      float qx = qd[i] * x[i];
#pragma unroll 8
      for (int j = 0; j < i; ++j) qx = fmaf(K[j * L.ldk + i], x[j], qx);
#pragma unroll 8
      for (int j = i + 1; j < n; ++j) qx = fmaf(K[i * L.ldk + j], x[j], qx);
      float aty = 0.f;
      for (int k = 0; k < p; ++k) aty = fmaf(ld_ro(A + k * n + i), mu[c * L.fv + a + k], aty);
      R[c * L.ldx + i] = r1s[c * L.nv + i] - qx - u[c * L.nv + i] - aty;
    }
    for (int e = t; e < 2 * nf; e += NT) {
      const int c = e / nf, k = e - c * nf;
      float fdx;
      if (k < a) {
        fdx = fmaf(-D[k], mu[c * L.fv + k], (c == 0 ? ea : eb)[act[k]]);
      } else {
        const float* x = dx + c * L.nv;
        fdx = 0.f;
        for (int j = 0; j < n; ++j) fdx = fmaf(ld_ro(A + (k - a) * n + j), x[j], fdx);
      }
      (c == 0 ? ua : ub)[k] = r2s[c * L.fv + k] - fdx;
    }
    __syncthreads();
    solve(0, 2);  // the correction
    for (int e = t; e < 2 * n; e += NT) {
      const int c = e / n, i = e - c * n;
      R[c * L.ldx + i] += dx[c * L.nv + i];
    }
    for (int e = t; e < 2 * nf; e += NT) {
      const int c = e / nf, k = e - c * nf;
      (c == 0 ? ua : ub)[k] += mu[c * L.fv + k];
    }
    __syncthreads();
    g_times_dx(0, 2);
  }

  // ---- residuals (eq. 4, eq. 10) and the measure ----
  // implicit: bz = b_k(v), bs = b_k(-v) with kappa = s'z/m; standard: bz = z, bs = s.
  // mode 0: complementarity term max z.*s; mode 1 (relax): |kappa - kr| / kr.
  static __device__ __noinline__ float2 residuals(const FwdParams& P, bool implicit, int mode) {
    const FLayout& L = fwd_state.L;
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    QP_BIG(K); QP_ARR(qd); QP_BIG(G); QP_ARR(q); QP_ARR(b); QP_ARR(h); QP_ARR(x);
    const float* const A = fwd_state.gA;
    QP_ARR(y); QP_ARR(z); QP_ARR(s); QP_ARR(rt); QP_ARR(re); QP_ARR(ri);
    QP_ARR(bz); QP_ARR(bs); QP_ARR(tn); QP_ARR(red); QP_ARR(col);
    float ks[1] = {0.f};
    for (int r = t; r < m; r += NT) ks[0] = fmaf(z[r], s[r], ks[0]);
    reduce<1>(ks, red, OpSum());
    const float kappa = m > 0 ? ks[0] / (float)m : 0.f;
    // the large variant: one coalesced sweep over the rows of K's upper
    // triangle (Q), G and A gives Q x (row dots into rt, column sums), G x
    // (into ri), G'z, A x (into re) and A'y; qcol / acol hold the Q and A
    // column sums afterwards
    float* qcol = nullptr;
    float* acol = nullptr;
    if constexpr (kBig) {
      QP_ARR(wp);
      constexpr int nw = NT / 32;
      const float* xq[1] = {x};
      float* dq[1] = {rt};
      warp_rows_n<NT, 4, 1, 1, true, false>(K, L.ldk, n, n, xq, dq, xq, wp, L.nv);
      float* dg[1] = {ri};
      const float* cz[1] = {z};
      warp_rows_n<NT, 4, 1, 1, false, false>(G, L.ldg, m, n, xq, dg, cz, wp + nw * L.nv, L.nv);
      float* da[1] = {re};
      const float* cy[1] = {y};
      warp_rows_n<NT, 4, 1, 1, false, kCoh>(A, n, p, n, xq, da, cy, wp + 2 * nw * L.nv, L.nv);
      __syncthreads();
      // column sums over the warps, in warp order, into each matrix's first
      // partial row (column c is summed and written by one thread)
      for (int e = t; e < 3 * n; e += NT) {
        const int k = e / n, c = e - k * n;
        float* pk = wp + k * nw * L.nv;
        float acc = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) acc += pk[w2 * L.nv + c];
        if (k == 1) tn[c] = acc;
        else pk[c] = acc;
      }
      __syncthreads();
      qcol = wp;
      acol = wp + 2 * nw * L.nv;
    } else {
      const float* vv[1] = {z};
      float* oo[1] = {tn};
      col_dot<NT, 1>(G, L.ldg, m, n, vv, oo, col);
      // A x: A is the caller's, in global memory: a warp per row (coalesced,
      // the row's loads in flight together) instead of a thread walking it
      if (p > 0) {
        const float* xq[1] = {x};
        float* da[1] = {re};
        warp_rows_n<NT, 2, 1, 0, false, kCoh>(A, n, p, n, xq, da, nullptr, nullptr, 0);
        __syncthreads();
      }
    }
    // 0 |rt| 1 |Qx| 2 |A'y| 3 |G'z| 4 |re| 5 |Ax| 6 |ri| 7 |Gx| 8 |s| 9 zs 10 |rz,rs| 11 |z| 12 nonfinite
    float mx[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) mx[k] = 0.f;
    for (int u = t; u < n + m + p; u += NT) {
      if (u < n) {
        const int i = u;
        // (Q x)_i from K's strict upper triangle and the diagonal qd
        float qx = qd[i] * x[i];
        float aty = 0.f;
        if constexpr (kBig) {
          // the sweep's parts: row i's upper entries (rt), column i above it
          qx += rt[i] + qcol[i];
          aty = acol[i];
        } else {
          for (int j = 0; j < i; ++j) qx = fmaf(K[j * L.ldk + i], x[j], qx);
          for (int j = i + 1; j < n; ++j) qx = fmaf(K[i * L.ldk + j], x[j], qx);
          for (int k = 0; k < p; ++k) aty = fmaf(ld_ro(A + k * n + i), y[k], aty);
        }
        const float r = qx + q[i] + tn[i] + aty;
        rt[i] = r;
        mx[12] += isfinite(r) ? 0.f : 1.f;
        mx[0] = fmaxf(mx[0], fabsf(r)); mx[1] = fmaxf(mx[1], fabsf(qx));
        mx[2] = fmaxf(mx[2], fabsf(aty)); mx[3] = fmaxf(mx[3], fabsf(tn[i]));
      } else if (u < n + m) {
        const int r = u - n;
        const float gx = kBig ? ri[r] : row_dot(G, L.ldg, r, x, L.nv);
        const float rii = gx + s[r] - h[r];
        ri[r] = rii;
        mx[12] += (isfinite(rii) && isfinite(z[r]) && isfinite(s[r])) ? 0.f : 1.f;
        mx[6] = fmaxf(mx[6], fabsf(rii)); mx[7] = fmaxf(mx[7], fabsf(gx));
        mx[8] = fmaxf(mx[8], fabsf(s[r])); mx[9] = fmaxf(mx[9], z[r] * s[r]);
        mx[11] = fmaxf(mx[11], fabsf(z[r]));
        if (implicit) {
          float pz, ps;
          retract_pair(z[r] - s[r], kappa, pz, ps);
          const float rzz = z[r] - pz, rss = s[r] - ps;
          bz[r] = pz; bs[r] = ps;  // r_z = z - bz and r_s = s - bs are formed where used
          mx[10] = fmaxf(mx[10], fmaxf(fabsf(rzz), fabsf(rss)));
        } else {
          bz[r] = z[r]; bs[r] = s[r];
          // relax of the standard method: distance of each z_i s_i from kappa_relax
          if (mode == 1) mx[10] = fmaxf(mx[10], fabsf(fmaf(z[r], s[r], -P.kappa_relax)));
        }
      } else {
        const int k = u - n - m;
        const float ax = re[k];  // from the row sweep above
        const float r = ax - b[k];
        re[k] = r;
        mx[12] += isfinite(r) ? 0.f : 1.f;
        mx[4] = fmaxf(mx[4], fabsf(r)); mx[5] = fmaxf(mx[5], fabsf(ax));
      }
    }
    reduce<13>(mx, red, OpMax());
    QP_MARK(PH_RESID);
    if (mx[12] > 0.f) return make_float2(NAN, kappa);
    float comp = mx[9];
    if (mode == 1)
      comp = (implicit ? fabsf(kappa - P.kappa_relax) : mx[10]) / P.kappa_relax;
    if (!implicit) mx[10] = 0.f;  // (r_z, r_s) exist on the implicit manifold only
    if (P.norm_abs)
      return make_float2(fmaxf(fmaxf(fmaxf(mx[0], mx[4]), fmaxf(mx[6], comp)), mx[10]), kappa);
    const float dt = fmaxf(fmaxf(1.0f, fwd_state.qn), fmaxf(fmaxf(mx[1], mx[2]), mx[3]));
    const float de = fmaxf(fmaxf(1.0f, fwd_state.bn), mx[5]);
    const float di = fmaxf(fmaxf(1.0f, fwd_state.hn), fmaxf(mx[7], mx[8]));
    const float dz = fmaxf(1.0f, fmaxf(mx[11], mx[8]));
    return make_float2(
        fmaxf(fmaxf(fmaxf(mx[0] / dt, mx[4] / de), fmaxf(mx[6] / di, comp)), mx[10] / dz), kappa);
  }

  // b_k(v), b_k(-v) of row r in the Newton matrix: those of the current
  // point, or (kChord) those frozen with the factorisation that chord steps
  // reuse -- b_k(v) kept in `ina` (read only while factoring), b_k(-v) =
  // kappa / b_k(v) (the retraction keeps b_k(v) b_k(-v) = kappa)
  template <bool kChord>
  static __device__ __forceinline__ void newton_diag(int r, float& jz, float& js) {
    if constexpr (kChord) {
      QP_ARR(ina);
      jz = ina[r];
      js = fwd_state.chord_kappa / jz;
    } else {
      QP_ARR(bz); QP_ARR(bs);
      jz = bz[r];
      js = bs[r];
    }
  }

  // ---- implicit right-hand sides, two columns (r_kappa = 0 and d/dr_kappa) ----
  // The residuals r_z = z - bz, r_s = s - bs are the current point's; the
  // elimination's diagonals are the Newton matrix's (newton_diag).
  template <bool kChord>
  static __device__ __noinline__ void implicit_rhs() {
    const FLayout& L = fwd_state.L;
    QP_ARR(bz); QP_ARR(bs); QP_ARR(z); QP_ARR(s); QP_ARR(ri); QP_ARR(re); QP_ARR(ta);
    QP_ARR(tb); QP_ARR(ua); QP_ARR(ub); QP_ARR(R); QP_BIG(G); QP_ARR(rt); QP_ARR(col);
    QP_IARR(pos); QP_IARR(act);
    const int m = L.m, t = threadIdx.x, a = fwd_state.a, nf = fwd_state.nf;
    for (int r = t; r < m; r += NT) {
      float jz, js;
      newton_diag<kChord>(r, jz, js);
      const float rho = jz + js;
      const bool inact = pos[r] < 0;
      const float rzr = z[r] - bz[r], rsr = s[r] - bs[r];
      const float dri = ri[r] - rsr;
      ta[r] = ri[r] + rzr - rsr - (inact ? dri * rho / js : 0.f);
      tb[r] = inact ? 1.0f / js : 0.f;
    }
    for (int k = t; k < nf; k += NT) {
      if (k < a) {
        const int r = act[k];
        float jz, js;
        newton_diag<kChord>(r, jz, js);
        const float rho = jz + js;
        ua[k] = -(ri[r] - (s[r] - bs[r])) * rho / jz;
        ub[k] = 1.0f / jz;
      } else {
        ua[k] = -re[k - a];
        ub[k] = 0.f;
      }
    }
    __syncthreads();
    const float* vv[2] = {ta, tb};
    float* oo[2] = {R, R + L.ldx};
    if constexpr (kBig) {
      // G in global memory: coalesced row sweep, per-warp column sums added
      // in warp order
      QP_ARR(wp);
      constexpr int nw = NT / 32;
      warp_rows_n<NT, 4, 0, 2, false, false>(G, L.ldg, m, L.n, nullptr, nullptr, vv, wp, L.nv);
      __syncthreads();
      for (int e = t; e < 2 * L.n; e += NT) {
        const int k = e / L.n, c = e - k * L.n;
        const float* pk = wp + k * nw * L.nv;
        float acc = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) acc += pk[w2 * L.nv + c];
        oo[k][c] = k == 0 ? acc - rt[c] : acc;
      }
      __syncthreads();
    } else {
      col_dot<NT, 2>(G, L.ldg, m, L.n, vv, oo, col, rt, -1.0f);
    }
    QP_MARK(PH_RHS);
  }

  // ds, dz, dv of the implicit direction for r_kappa = rk on row r
  template <bool kChord>
  static __device__ __forceinline__ void implicit_dir(int r, float rk, float& dsr, float& dzr,
                                                      float& dvr) {
    QP_ARR(bz); QP_ARR(bs); QP_ARR(ea); QP_ARR(eb); QP_ARR(ri); QP_ARR(z); QP_ARR(s);
    QP_ARR(ua); QP_ARR(ub); QP_IARR(pos);
    float jz, js;
    newton_diag<kChord>(r, jz, js);
    const float rzr = z[r] - bz[r], rsr = s[r] - bs[r];
    const float rho = jz + js;
    const float c = 1.0f / rho;
    const float e = fmaf(rk, eb[r], ea[r]);
    const int k = pos[r];
    if (k < 0) {
      const float rho2 = ri[r] - rsr - c * rk;
      dvr = (e + rho2) * rho / js;
    } else {
      dvr = fmaf(rk, ub[k], ua[k]) + e;
    }
    dzr = -rzr + (jz * c) * dvr - c * rk;
    dsr = -rsr - (js * c) * dvr - c * rk;
  }

  template <bool kChord>
  static __device__ __noinline__ float implicit_alpha(float rk, bool store) {
    QP_ARR(s); QP_ARR(z); QP_ARR(tb); QP_ARR(red);
    float amin[1] = {1.0f};
    for (int r = threadIdx.x; r < fwd_state.L.m; r += NT) {
      float dsr, dzr, dvr;
      implicit_dir<kChord>(r, rk, dsr, dzr, dvr);
      if (dsr < 0.f) amin[0] = fminf(amin[0], -s[r] / dsr);
      if (dzr < 0.f) amin[0] = fminf(amin[0], -z[r] / dzr);
      if (store) tb[r] = dvr;
    }
    reduce<1>(amin, red, OpMin());
    return amin[0];
  }

  static __device__ __noinline__ float implicit_mu_aff(float rk, float alpha) {
    QP_ARR(s); QP_ARR(z); QP_ARR(red);
    float acc[1] = {0.f};
    for (int r = threadIdx.x; r < fwd_state.L.m; r += NT) {
      float dsr, dzr, dvr;
      implicit_dir<false>(r, rk, dsr, dzr, dvr);
      acc[0] = fmaf(fmaf(alpha, dsr, s[r]), fmaf(alpha, dzr, z[r]), acc[0]);
    }
    reduce<1>(acc, red, OpSum());
    return acc[0] / (float)fwd_state.L.m;
  }

  static __device__ __noinline__ void implicit_update(float alpha, float rk, float kappa) {
    const FLayout& L = fwd_state.L;
    QP_ARR(x); QP_ARR(y); QP_ARR(z); QP_ARR(s); QP_ARR(R); QP_ARR(ua); QP_ARR(ub); QP_ARR(tb);
    const int p = L.p, t = threadIdx.x, a = fwd_state.a;
    const float knew = kappa - alpha * rk;
    for (int i = t; i < L.n; i += NT) x[i] = fmaf(alpha, fmaf(rk, R[L.ldx + i], R[i]), x[i]);
    for (int k = t; k < p; k += NT) y[k] = fmaf(alpha, fmaf(rk, ub[a + k], ua[a + k]), y[k]);
    for (int r = t; r < L.m; r += NT) {
      const float vn = fmaf(alpha, tb[r], z[r] - s[r]);
      float pz, ps;
      retract_pair(vn, knew, pz, ps);
      z[r] = pz;
      s[r] = ps;
    }
    __syncthreads();
  }

  // One implicit Newton step (Alg. 1 with predictor-corrector, or Alg. 2 when
  // kt_fixed >= 0).  Returns false on a factorisation failure.
  static __device__ __noinline__ bool implicit_step(const FwdParams& P, float kappa, float kt_fixed) {
    partition();
    trace_scaling(P);
    implicit_rhs<false>();
    fold_rhs();
    if (!factor(2)) {
      trace_factor_failed(P);
      return false;
    }
    solve_folded();
    g_times_dx(0, 2);
    if constexpr (kBig) {
      for (int k = 0; k < fwd_state.refine; ++k) refine_folded();
    }
    if (P.diag) trace_folded_solve(P);
    float kt;
    if (kt_fixed >= 0.f) {
      kt = kt_fixed;
    } else {
      float sigma;
      if (P.sigma_mode == 1) {
        sigma = P.sigma;
      } else {
        const float aa = implicit_alpha<false>(kappa, false);
        const float mua = implicit_mu_aff(kappa, aa);
        const float ratio = mua / kappa;
        trace(P, QP_STAGE_CENTERING, !isfinite(aa) || !isfinite(ratio));
        sigma = ratio * ratio * ratio;
        if (!(sigma >= 0.f)) sigma = 0.f;
        if (sigma > 1.f) sigma = 1.f;
      }
      kt = fmaxf(sigma * kappa, P.kappa_min);
    }
    const float rk = kappa - kt;
    if (P.diag) trace_corrector(P, rk);
    const float alpha = P.step_frac * implicit_alpha<false>(rk, true);
    trace(P, QP_STAGE_LINESEARCH, !isfinite(alpha));
    implicit_update(alpha, rk, kappa);
    trace_iterate(P, QP_STAGE_LINESEARCH);
    QP_MARK(PH_STEP);
    return true;
  }

  // ---- Alg. 2 chord step: the Newton step to kt with the factorisation of an
  // earlier iterate (its partition, factors and Newton-matrix diagonals, see
  // freeze_newton_matrix) and the residuals of the current one.  Its fixed
  // point is the relaxed point itself; convergence is linear instead of
  // quadratic. ----
  static __device__ __noinline__ void chord_step(const FwdParams& P, float kappa, float kt) {
    implicit_rhs<true>();
    solve(0, 2);
    g_times_dx(0, 2);
    const float rk = kappa - kt;
    const float alpha = P.step_frac * implicit_alpha<true>(rk, true);
    implicit_update(alpha, rk, kappa);
    QP_MARK(PH_STEP);
  }

  // Right after an implicit step: keep its Newton matrix's b_k(v) (bz, not yet
  // recomputed at the new point) and kappa for the chord steps that follow.
  static __device__ void freeze_newton_matrix(float kappa) {
    QP_ARR(bz); QP_ARR(ina);
    for (int r = threadIdx.x; r < fwd_state.L.m; r += NT) ina[r] = bz[r];
    if (threadIdx.x == 0) fwd_state.chord_kappa = kappa;
    __syncthreads();
  }

  // ---- explicit complementarity (ablation): Mehrotra predictor-corrector on
  // eq. 8 in the same two-level form.  For r_c (z.*s, then the corrector term)
  // rhs1 = -r_t + G_I'(-W r_i + r_c/s), rhs2 = (-(r_i - r_c/z)_A, -r_e). ----
  static __device__ __noinline__ bool standard_step(const FwdParams& P, float mu) {
    const FLayout& L = fwd_state.L;
    const int m = L.m, p = L.p, t = threadIdx.x;
    partition();
    QP_ARR(z); QP_ARR(s); QP_ARR(ri); QP_ARR(re); QP_ARR(ta); QP_ARR(tb);
    QP_ARR(ua); QP_ARR(ub); QP_ARR(ea); QP_ARR(eb); QP_ARR(R); QP_BIG(G); QP_ARR(rt);
    QP_ARR(col); QP_ARR(red); QP_ARR(x); QP_ARR(y); QP_IARR(pos); QP_IARR(act);
    const int a = fwd_state.a, nf = fwd_state.nf;
    trace_scaling(P);
    // predictor (slot 0): r_c = z.*s
    for (int r = t; r < m; r += NT) ta[r] = pos[r] < 0 ? -(z[r] / s[r]) * ri[r] + z[r] : 0.f;
    for (int k = t; k < nf; k += NT) ua[k] = k < a ? -(ri[act[k]] - s[act[k]]) : -re[k - a];
    __syncthreads();
    {
      const float* vv[1] = {ta};
      float* oo[1] = {R};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col, rt, -1.0f);
    }
    if (!factor()) {
      trace_factor_failed(P);
      return false;
    }
    // W lives in the factors now: bz / bs serve as ds / dz scratch below
    float* const rz = fwd_dyn + fwd_state.L.o_bz;
    float* const rs = fwd_dyn + fwd_state.L.o_bs;
    solve(0, 1);
    g_times_dx(0, 1);
    float amin[1] = {1.0f};
    bool bad = false;
    for (int r = t; r < m; r += NT) {
      const float e = ea[r];
      const float dzr = pos[r] < 0 ? (z[r] / s[r]) * (e + ri[r]) - z[r] : ua[pos[r]];
      const float dsr = -ri[r] - e;
      rz[r] = dsr;  // keep ds_aff
      rs[r] = dzr;  // keep dz_aff
      bad |= !isfinite(dsr) || !isfinite(dzr);
      if (dsr < 0.f) amin[0] = fminf(amin[0], -s[r] / dsr);
      if (dzr < 0.f) amin[0] = fminf(amin[0], -z[r] / dzr);
    }
    if (P.diag) trace(P, QP_STAGE_PREDICTOR, bad || any_nonfinite(R, L.n));
    reduce<1>(amin, red, OpMin());
    const float aa = amin[0];
    float acc[1] = {0.f};
    for (int r = t; r < m; r += NT) acc[0] = fmaf(fmaf(aa, rz[r], s[r]), fmaf(aa, rs[r], z[r]), acc[0]);
    reduce<1>(acc, red, OpSum());
    const float ratio = (acc[0] / (float)m) / mu;
    trace(P, QP_STAGE_CENTERING, !isfinite(aa) || !isfinite(ratio));
    float sigma = ratio * ratio * ratio;
    if (!(sigma >= 0.f)) sigma = 0.f;
    if (sigma > 1.f) sigma = 1.f;
    if (P.sigma_mode == 1) sigma = P.sigma;
    const float smu = sigma * mu;
    // corrector increment (slot 1): r_c' = ds_a .* dz_a - sigma mu, zero base residuals
    for (int r = t; r < m; r += NT) {
      const float rc = rz[r] * rs[r] - smu;
      ta[r] = rc;  // keep r_c'
      tb[r] = pos[r] < 0 ? rc / s[r] : 0.f;
    }
    for (int k = t; k < nf; k += NT) ub[k] = k < a ? ta[act[k]] / z[act[k]] : 0.f;
    __syncthreads();
    {
      const float* vv[1] = {tb};
      float* oo[1] = {R + L.ldx};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col);
    }
    solve(1, 1);
    g_times_dx(1, 1);
    float amin2[1] = {1.0f};
    bad = false;
    for (int r = t; r < m; r += NT) {
      const float e = eb[r];
      const float dzc = pos[r] < 0 ? (z[r] / s[r]) * e - ta[r] / s[r] : ub[pos[r]];
      const float dsr = rz[r] - e;
      const float dzr = rs[r] + dzc;
      rz[r] = dsr;
      rs[r] = dzr;
      bad |= !isfinite(dsr) || !isfinite(dzr);
      if (dsr < 0.f) amin2[0] = fminf(amin2[0], -s[r] / dsr);
      if (dzr < 0.f) amin2[0] = fminf(amin2[0], -z[r] / dzr);
    }
    if (P.diag) {
      for (int i = t; i < L.n; i += NT) bad |= !isfinite(R[i] + R[L.ldx + i]);
      for (int k = t; k < p; k += NT) bad |= !isfinite(ua[a + k] + ub[a + k]);
      trace(P, QP_STAGE_CORRECTOR, bad);
    }
    reduce<1>(amin2, red, OpMin());
    const float alpha = fminf(1.0f, 0.99f * amin2[0]);
    trace(P, QP_STAGE_LINESEARCH, !isfinite(alpha));
    for (int i = t; i < L.n; i += NT) x[i] = fmaf(alpha, R[i] + R[L.ldx + i], x[i]);
    for (int k = t; k < p; k += NT) y[k] = fmaf(alpha, ua[a + k] + ub[a + k], y[k]);
    for (int r = t; r < m; r += NT) {
      z[r] = fmaf(alpha, rs[r], z[r]);
      s[r] = fmaf(alpha, rz[r], s[r]);
    }
    __syncthreads();
    trace_iterate(P, QP_STAGE_LINESEARCH);
    return true;
  }

  // ---- explicit complementarity, Alg. 2 for the standard method: one
  // Newton step on the KKT system with z .* s = target (no predictor),
  // fraction-to-boundary 0.99.  With r_c = z .* s - target:
  // rhs1 = -r_t + G_I'(-W r_i + r_c/s), rhs2 = (-(r_i - r_c/z)_A, -r_e);
  // dz = W (r_i + G dx) - r_c/s on inactive rows, ds = -r_i - G dx. ----
  static __device__ __noinline__ bool standard_fixed_step(const FwdParams& P, float target) {
    const FLayout& L = fwd_state.L;
    const int m = L.m, p = L.p, t = threadIdx.x;
    partition();
    QP_ARR(z); QP_ARR(s); QP_ARR(ri); QP_ARR(re); QP_ARR(ta); QP_ARR(ua); QP_ARR(ea);
    QP_ARR(R); QP_BIG(G); QP_ARR(rt); QP_ARR(col); QP_ARR(red); QP_ARR(x); QP_ARR(y);
    QP_IARR(pos); QP_IARR(act);
    const int a = fwd_state.a, nf = fwd_state.nf;
    trace_scaling(P);
    for (int r = t; r < m; r += NT)
      ta[r] = pos[r] < 0 ? -(z[r] / s[r]) * ri[r] + z[r] - target / s[r] : 0.f;
    for (int k = t; k < nf; k += NT)
      ua[k] = k < a ? -(ri[act[k]] - s[act[k]] + target / z[act[k]]) : -re[k - a];
    __syncthreads();
    {
      const float* vv[1] = {ta};
      float* oo[1] = {R};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col, rt, -1.0f);
    }
    if (!factor()) {
      trace_factor_failed(P);
      return false;
    }
    // W lives in the factors now: bz / bs serve as ds / dz scratch below
    float* const rz = fwd_dyn + fwd_state.L.o_bz;
    float* const rs = fwd_dyn + fwd_state.L.o_bs;
    solve(0, 1);
    g_times_dx(0, 1);
    float amin[1] = {1.0f};
    bool bad = false;
    for (int r = t; r < m; r += NT) {
      const float e = ea[r];
      const float dzr =
          pos[r] < 0 ? (z[r] / s[r]) * (e + ri[r]) - z[r] + target / s[r] : ua[pos[r]];
      const float dsr = -ri[r] - e;
      rz[r] = dsr;
      rs[r] = dzr;
      bad |= !isfinite(dsr) || !isfinite(dzr);
      if (dsr < 0.f) amin[0] = fminf(amin[0], -s[r] / dsr);
      if (dzr < 0.f) amin[0] = fminf(amin[0], -z[r] / dzr);
    }
    if (P.diag) trace(P, QP_STAGE_CORRECTOR, bad || any_nonfinite(R, L.n));
    reduce<1>(amin, red, OpMin());
    const float alpha = fminf(1.0f, 0.99f * amin[0]);
    trace(P, QP_STAGE_LINESEARCH, !isfinite(alpha));
    for (int i = t; i < L.n; i += NT) x[i] = fmaf(alpha, R[i], x[i]);
    for (int k = t; k < p; k += NT) y[k] = fmaf(alpha, ua[a + k], y[k]);
    for (int r = t; r < m; r += NT) {
      z[r] = fmaf(alpha, rs[r], z[r]);
      s[r] = fmaf(alpha, rz[r], s[r]);
    }
    __syncthreads();
    trace_iterate(P, QP_STAGE_LINESEARCH);
    return true;
  }

  // CVXOPT-style start: (Q + G'G) x + A'y = -q + G'h, A x = b; z = G x - h, s = -z, shifted.
  // With m = 0 this is the exact solution of the equality-constrained QP.
  static __device__ __noinline__ bool initialize() {
    const FLayout& L = fwd_state.L;
    const int m = L.m, p = L.p, t = threadIdx.x;
    QP_ARR(bz); QP_ARR(bs); QP_ARR(ua); QP_ARR(b); QP_ARR(h); QP_ARR(R); QP_BIG(G); QP_ARR(col);
    QP_ARR(q); QP_ARR(x); QP_ARR(y); QP_ARR(z); QP_ARR(s); QP_ARR(red);
    for (int r = t; r < m; r += NT) { bz[r] = 1.0f; bs[r] = 1.0f; }
    __syncthreads();
    partition();  // W = 1 everywhere: no active rows, F = A
    for (int k = t; k < p; k += NT) ua[k] = b[k];
    {
      const float* vv[1] = {h};
      float* oo[1] = {R};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col, q, -1.0f);
    }
    const bool ok = factor();
    solve(0, 1);
    for (int i = t; i < L.n; i += NT) x[i] = R[i];
    for (int k = t; k < p; k += NT) y[k] = ua[k];
    __syncthreads();
    if (m == 0) return ok;
    float mx[3] = {-INFINITY, -INFINITY, 0.f};
    for (int r = t; r < m; r += NT) {
      const float zr = row_dot(G, L.ldg, r, x, L.nv) - h[r];
      z[r] = zr;
      s[r] = -zr;
      mx[0] = fmaxf(mx[0], zr);   // -min(s)
      mx[1] = fmaxf(mx[1], -zr);  // -min(z)
      mx[2] = fmaxf(mx[2], fabsf(zr));
    }
    reduce<3>(mx, red, OpMax());
    const float thr = -1e-8f * fmaxf(1.0f, mx[2]);
    const bool shs = mx[0] >= thr, shz = mx[1] >= thr;
    for (int r = t; r < m; r += NT) {
      if (shs) s[r] += 1.0f + mx[0];
      if (shz) z[r] += 1.0f + mx[1];
    }
    __syncthreads();
    return ok;
  }

  // ---- gradient cache: factors, W, active map and the point (Alg. 3 input) ----
  static __device__ __noinline__ void write_cache(const FwdParams& P, int bi) {
    const FLayout& L = fwd_state.L;
    QP_BIG(K); QP_BIG(Y); QP_BIG(C); QP_ARR(ea); QP_ARR(D); QP_ARR(x); QP_ARR(y); QP_ARR(z);
    QP_IARR(pos);
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x, a = fwd_state.a, nf = fwd_state.nf;
    const CacheLayout cl = cache_layout(n, m, p, L.amax, kBig);
    float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
    if (t == 0) {
      reinterpret_cast<int*>(c + cl.oHdr)[0] = a;
      reinterpret_cast<int*>(c + cl.oHdr)[1] = nf;
      reinterpret_cast<int*>(c + cl.oHdr)[2] = P.refine_steps;
    }
    if (kBig) {
      // unpacked, with the workspace strides (cl.ldk == L.ldk, cl.ldc == L.ldc)
      for (int e = t; e < n * n; e += NT) {
        const int i = e / n, j = e - i * n;
        if (j <= i) c[cl.oL + i * cl.ldk + j] = K[i * L.ldk + j];
      }
      for (int e = t; e < nf * n; e += NT) {
        const int k = e / n, i = e - k * n;
        c[cl.oY + k * cl.ldk + i] = Y[k * L.ldk + i];
      }
      for (int e = t; e < nf * nf; e += NT) {
        const int i = e / nf, j = e - i * nf;
        if (j <= i) c[cl.oLC + i * cl.ldc + j] = C[i * L.ldc + j];
      }
    }
    const int nl = kBig ? 0 : n * (n + 1) / 2;
    for (int e = t; e < nl; e += NT) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      c[cl.oL + e] = K[i * L.ldk + (e - i * (i + 1) / 2)];
    }
    for (int e = t; e < (kBig ? 0 : nf * n); e += NT) {
      const int k = e / n, i = e - k * n;
      c[cl.oY + e] = Y[k * L.ldk + i];
    }
    const int fl = kBig ? 0 : nf * (nf + 1) / 2;
    for (int e = t; e < fl; e += NT) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      c[cl.oLC + e] = C[i * L.ldc + (e - i * (i + 1) / 2)];
    }
    for (int r = t; r < m; r += NT) {
      c[cl.oW + r] = pos[r] < 0 ? ea[r] : D[pos[r]];  // W (inactive rows) or 1/W (active rows)
      reinterpret_cast<int*>(c + cl.oPos)[r] = pos[r];
      c[cl.oz + r] = z[r];
    }
    for (int i = t; i < n; i += NT) c[cl.ox + i] = x[i];
    for (int k = t; k < p; k += NT) c[cl.oy + k] = y[k];
    __syncthreads();
  }

  // save (restore = false) or restore the iterate (x, y, z, s) in the
  // instance's gradient-cache slot (its x, y, z blocks and the s block)
  static __device__ __noinline__ void snapshot(const FwdParams& P, int bi, bool restore) {
    const FLayout& L = fwd_state.L;
    QP_ARR(x); QP_ARR(y); QP_ARR(z); QP_ARR(s);
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    const CacheLayout cl = cache_layout(n, m, p, L.amax, kBig);
    float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
    if (restore) {
      for (int i = t; i < n; i += NT) x[i] = c[cl.ox + i];
      for (int k = t; k < p; k += NT) y[k] = c[cl.oy + k];
      for (int r = t; r < m; r += NT) { z[r] = c[cl.oz + r]; s[r] = c[cl.os + r]; }
    } else {
      for (int i = t; i < n; i += NT) c[cl.ox + i] = x[i];
      for (int k = t; k < p; k += NT) c[cl.oy + k] = y[k];
      for (int r = t; r < m; r += NT) { c[cl.oz + r] = z[r]; c[cl.os + r] = s[r]; }
    }
    __syncthreads();
  }

  static __device__ __noinline__ void write_solution(const FwdParams& P, int bi, bool good) {
    const FLayout& L = fwd_state.L;
    QP_ARR(x); QP_ARR(y); QP_ARR(z); QP_ARR(s);
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    const float nanv = NAN;
    for (int i = t; i < n; i += NT) P.x[(size_t)bi * n + i] = good ? x[i] : nanv;
    for (int k = t; k < p; k += NT) P.y[(size_t)bi * p + k] = good ? y[k] : nanv;
    for (int r = t; r < m; r += NT) {
      P.z[(size_t)bi * m + r] = good ? z[r] : nanv;
      P.s[(size_t)bi * m + r] = good ? s[r] : nanv;
    }
  }

  // ---- whole instance ----
  static __device__ __noinline__ void run(const FwdParams& P, int bi) {
    const int n = fwd_state.L.n, m = fwd_state.L.m, p = fwd_state.L.p, t = threadIdx.x;
    const bool implicit = P.formulation == 0;
    if (t == 0) fwd_state.all_inactive = P.formulation == 2;  // eq. 8 as it stands
    int status = ST_SOLVED, iters = 0;
    float meas = NAN;
    bool snap = false;      // a snapshot for Alg. 2 is in the cache slot
    bool polished = false;  // the relax ended with a polishing step (its factor is current)
    const bool good = load(P, bi);
    if (!good) {
      status = ST_BAD_INPUT;
    } else {
      bool warm = false;
      if (P.warm_start && m > 0) {
        QP_ARR(x); QP_ARR(y); QP_ARR(z); QP_ARR(s); QP_ARR(red);
        float mn[1] = {INFINITY};
        for (int i = t; i < n; i += NT) x[i] = P.x[(size_t)bi * n + i];
        for (int k = t; k < p; k += NT) y[k] = P.y[(size_t)bi * p + k];
        for (int r = t; r < m; r += NT) {
          z[r] = P.z[(size_t)bi * m + r];
          s[r] = P.s[(size_t)bi * m + r];
          mn[0] = fminf(mn[0], fminf(z[r], s[r]));
        }
        reduce<1>(mn, red, OpMin());
        warm = mn[0] > 0.f;
      }
      if (!warm && !initialize()) status = ST_NUMERICAL;
      if (!warm) trace_iterate(P, QP_STAGE_INIT);
      if (m == 0) {
        // equality-only QP: the start is the exact solve; Newton steps on the
        // linear KKT system refine it with the same factorisation
        for (int it = 0; status == ST_SOLVED; ++it) {
          meas = residuals(P, implicit, 0).x;
          if (!(meas == meas)) { status = ST_NUMERICAL; break; }
          if (meas < P.tol || it >= P.max_iter) break;
          QP_ARR(R); QP_ARR(rt); QP_ARR(ua); QP_ARR(re); QP_ARR(x); QP_ARR(y);
          for (int i = t; i < n; i += NT) R[i] = -rt[i];
          for (int k = t; k < p; k += NT) ua[k] = -re[k];
          __syncthreads();
          solve(0, 1);
          for (int i = t; i < n; i += NT) x[i] += R[i];
          for (int k = t; k < p; k += NT) y[k] += ua[k];
          __syncthreads();
          iters = it + 1;
        }
      } else {
        // ---- Alg. 1 ----
        float best = INFINITY;
        int since_best = 0;
        const bool snap_on = implicit && P.cache && P.kappa_relax > 0.f;
        for (int it = 0; status == ST_SOLVED; ++it) {
          const float2 rk = residuals(P, implicit, 0);
          const float kappa = rk.y;
          meas = rk.x;
          if (!(meas == meas)) { status = ST_NUMERICAL; break; }
          // the last iterate with kappa >= kappa_relax is where Alg. 2 starts
          if (snap_on && kappa >= P.kappa_relax) {
            snapshot(P, bi, false);
            snap = true;
          }
          if (meas < P.tol) break;
          if (it >= P.max_iter) { status = ST_MAX_ITER; break; }
          // stalled: the measure has reached its FP32 floor (~1e-7 scaled)
          // without reaching tol -- below kStallMeasure and no 10 % better
          // in 10 iterations.  Above it the iteration is still far from the
          // solution (short steps) and continues to max_iter, as in Alg. 1.
          if (meas < 0.9f * best) { best = meas; since_best = 0; }
          else if (++since_best >= 10 && best < kStallMeasure) { status = ST_STALLED; break; }
          const bool ok = implicit ? implicit_step(P, kappa, -1.0f) : standard_step(P, kappa);
          if (!ok) { status = ST_NUMERICAL; break; }
          iters = it + 1;
        }
      }
    }
    write_solution(P, bi, good);
    // ---- Alg. 2 (relax) and the factor at the relaxed point ----
    if (t == 0) fwd_state.in_relax = 1;
    if (P.cache && status != ST_BAD_INPUT) {
      QP_ARR(z); QP_ARR(s); QP_ARR(bz); QP_ARR(bs);
      if (m > 0 && P.kappa_relax > 0.f && status != ST_NUMERICAL && !implicit) {
        // Alg. 2 for the standard method: Newton steps on z .* s =
        // kappa_relax from its solution (each z_i s_i, not only their mean)
        int rstatus = ST_MAX_ITER;
        float rbest = INFINITY;
        int rsince = 0;
        for (int it = 0;; ++it) {
          const float rm = residuals(P, false, 1).x;
          if (!(rm == rm)) {
            trace(P, QP_STAGE_RELAX, true);
            rstatus = ST_NUMERICAL;
            break;
          }
          if (rm < 0.9f * rbest) { rbest = rm; rsince = 0; } else { ++rsince; }
          if (rm < P.relax_tol || (rm < P.tol && rsince >= 3)) { rstatus = ST_SOLVED; break; }
          if (it >= P.relax_max_iter) break;
          if (!standard_fixed_step(P, P.kappa_relax)) { rstatus = ST_NUMERICAL; break; }
          ++iters;
        }
        if (status == ST_SOLVED) status = rstatus;
        // gradients at this point: W = z ./ s
        for (int r = t; r < m; r += NT) { bz[r] = z[r]; bs[r] = s[r]; }
        __syncthreads();
      } else if (m > 0 && P.kappa_relax > 0.f && status != ST_NUMERICAL) {
        // Alg. 2 targets the central-path point x(kappa_relax), which does
        // not depend on where the Newton iteration starts; from the solve's
        // last iterate with kappa >= kappa_relax it is a few steps away,
        // from the converged solution (kappa << kappa_relax) about twice as
        // many (eq. 7 limits how fast kappa can grow back).
        if (snap) snapshot(P, bi, true);
        int rstatus = ST_MAX_ITER;
        float rbest = INFINITY;
        int rsince = 0;
        bool chord = false;  // a factorisation of an earlier relax iterate is current
        float rprev = INFINITY;
        for (int it = 0;; ++it) {
          const float2 rr = residuals(P, true, 1);
          const float rm = rr.x, kappa = rr.y;
          // chord steps continue while each cuts the measure at least
          // kChordRate-fold and it is above tol; otherwise the next step
          // refactors (linear convergence would end the relax on its floor
          // rule, short of relax_tol)
          if (chord && !(rm <= kChordRate * rprev && rm >= P.tol)) chord = false;
          rprev = rm;
          if (!(rm == rm)) { rstatus = ST_NUMERICAL; break; }
          if (rm < 0.9f * rbest) { rbest = rm; rsince = 0; } else { ++rsince; }
          // relax_tol where FP32 reaches it; otherwise its floor, once the
          // measure is below the solve tolerance and has stopped decreasing
          if (rm < P.relax_tol || (rm < P.tol && rsince >= 3)) {
            // one more (quadratically convergent) Newton step polishes the
            // relaxed point the gradients are taken at
            rstatus = ST_SOLVED;
            if (implicit_step(P, kappa, P.kappa_relax)) {
              ++iters;
              polished = true;
            }
            break;
          }
          if (it >= P.relax_max_iter) break;
          if (chord) {
            chord_step(P, kappa, P.kappa_relax);
          } else {
            if (!implicit_step(P, kappa, P.kappa_relax)) { rstatus = ST_NUMERICAL; break; }
            if (P.chord) { freeze_newton_matrix(kappa); chord = true; }
          }
          ++iters;
        }
        if (status == ST_SOLVED) status = rstatus;
        for (int r = t; r < m; r += NT) retract_pair(z[r] - s[r], P.kappa_relax, bz[r], bs[r]);
        __syncthreads();
      } else if (m > 0) {
        // gradients at the solution itself: W = z ./ s
        for (int r = t; r < m; r += NT) { bz[r] = z[r]; bs[r] = s[r]; }
        __syncthreads();
      }
      if (polished) {
        // The polishing step factored the Newton matrix one step before the
        // final point; W moved by ~1e-6 relative since.  Cache that factor
        // with the final point's W: the backward refines its solve against
        // the system built from the cached W, Q, G, A, with this factor as
        // the preconditioner (gradient errors unchanged in the tests), and
        // one factorisation per solve is saved.
        QP_ARR(ea); QP_ARR(D); QP_IARR(pos);
        for (int r = t; r < m; r += NT) {
          if (pos[r] < 0) ea[r] = bz[r] / bs[r];
          else D[pos[r]] = bs[r] / bz[r];
        }
        __syncthreads();
      } else {
        partition();
        if (!factor()) {
          trace_factor_failed(P);
          if (status == ST_SOLVED) status = ST_NUMERICAL;
        }
      }
      write_cache(P, bi);
      QP_MARK(PH_CACHE);
    } else if (P.cache && t == 0) {
      // non-finite data: mark the slot unwritten (active count -1) so the
      // backward pass gives NaN gradients instead of reading stale contents
      int* hdr = reinterpret_cast<int*>(P.cache + (size_t)bi * (size_t)P.cache_stride +
                                        cache_layout(n, m, p, fwd_state.L.amax, kBig).oHdr);
      hdr[0] = -1;
      hdr[1] = -1;
      hdr[2] = 0;
    }
    __syncthreads();
    if (t == 0) {
      // bulk copies that may still have been in flight: nothing of this
      // instance is trusted
      if (fwd_state.async_lost) {
        status = ST_NUMERICAL;
        fwd_state.diag |= QP_DIAG_ASYNC_LOST;
      }
      if (P.status) P.status[bi] = status;
      if (P.iters) P.iters[bi] = iters;
      if (P.kkt) P.kkt[bi] = meas;
      if (P.diag) P.diag[bi] = (fwd_state.diag & ~QP_STAGE_MASK) | fwd_state.nan_stage;
    }
  }
};

#undef QP_ARR
#undef QP_IARR
#undef QP_BIG

// minimum resident CTAs per SM the register budget is sized for (128
// registers a thread in the large variant: one 512-thread or two 256-thread
// CTAs per SM)
template <int NT, bool kBig> struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<32, false> { static constexpr int value = 12; };
template <> struct MinBlocks<128, false> { static constexpr int value = 3; };
template <> struct MinBlocks<256, false> { static constexpr int value = 3; };
template <> struct MinBlocks<256, true> { static constexpr int value = 2; };

// kBig: the large-problem variant, K, G, A, Y, C in the instance's slice of
// the global workspace P.ws (L1/L2-cached) instead of shared memory.
template <int NT, bool kBig>
__global__ void __launch_bounds__(NT, (MinBlocks<NT, kBig>::value)) qp_forward_kernel(const FwdParams P) {
  // the phases take the parameters by reference: keep them in shared memory
  // rather than letting each thread copy the whole block to local memory
  __shared__ FwdParams sP;
  if (threadIdx.x == 0) {
    sP = P;
    if (P.desc) {
      // ragged launch: this CTA's request, addressed as instance 0
      const ReqDesc& d = P.desc[blockIdx.x];
      sP.batch = 1; sP.n = d.n; sP.m = d.m; sP.p = d.p; sP.amax = d.amax;
      sP.Q = d.Q; sP.q = d.q; sP.A = d.A; sP.b = d.b; sP.G = d.G; sP.h = d.h;
      sP.x = d.x; sP.y = d.y; sP.z = d.z; sP.s = d.s;
      sP.status = d.status; sP.iters = d.iters; sP.kkt = d.kkt;
      sP.cache = d.cache; sP.cache_stride = 0;
      sP.ws = d.ws; sP.ws_stride = 0;
    }
  }
  __syncthreads();
  const int bi = P.desc ? 0 : blockIdx.x;
  float* const ws = kBig ? sP.ws + (size_t)bi * (size_t)sP.ws_stride : nullptr;
  Solver<NT, kBig>::init(sP.n, sP.m, sP.p, sP.amax, ws, sP.gwg, sP.refine_fwd);  // ends with a barrier
#ifdef QP_PHASE_TIMERS
  if (threadIdx.x == 0) fwd_state.timers = P.timers;
  __syncthreads();
#endif
  if constexpr (kBig) {
    // tensor-core G'WG: this CTA's TMEM for the whole solve (one CTA per SM:
    // the variant uses the whole register file)
    if (sP.gwg != 0) {
      if (threadIdx.x < 32) {
        tc::tmem_alloc(&fwd_state.tmem, tc::kTmemCols);
        tc::tmem_relinquish();
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  Solver<NT, kBig>::run(sP, bi);
  if constexpr (kBig) {
    if (sP.gwg != 0) {
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (threadIdx.x < 32) tc::tmem_dealloc(fwd_state.tmem, tc::kTmemCols);
    }
  }
}

}  // namespace fwd

// The kernel's dynamic shared-memory limit is set once, to the largest
// request any size can make: the attribute is per function and per process,
// and setting it can wait for kernels already running on the device, so it
// must not happen on the launch path.
template <int NT, bool kBig>
cudaError_t ensure_forward_smem(size_t smem) {
  static std::mutex mu;
  static size_t configured = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (configured == 0) {
    const size_t maxdyn = 227 * 1024 - fwd::kStaticSmem;
    cudaError_t e = cudaFuncSetAttribute(
        fwd::qp_forward_kernel<NT, kBig>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxdyn);
    if (e != cudaSuccess) return e;
    if (kBig && NT == 256) {
      // two CTAs per SM need the largest shared-memory carveout; without the
      // preference the runtime may configure less and keep one CTA per SM
      e = cudaFuncSetAttribute(fwd::qp_forward_kernel<NT, kBig>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
    }
    configured = maxdyn;
  }
  return smem <= configured ? cudaSuccess : cudaErrorInvalidValue;
}

// Instantiated once per (block size, variant) in qp_forward_<NT>[w].cu.
template <int NT, bool kBig>
cudaError_t launch_forward_nt(const FwdParams& P, size_t smem, int grid, cudaStream_t st) {
  const cudaError_t e = ensure_forward_smem<NT, kBig>(smem);
  if (e != cudaSuccess) return e;
  fwd::qp_forward_kernel<NT, kBig><<<grid, NT, smem, st>>>(P);
  return cudaGetLastError();
}

template <int NT, bool kBig>
int forward_blocks_per_sm_nt(size_t smem) {
  int nb = 0;
  if (ensure_forward_smem<NT, kBig>(smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd::qp_forward_kernel<NT, kBig>, NT,
                                                    smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace qpgpu
