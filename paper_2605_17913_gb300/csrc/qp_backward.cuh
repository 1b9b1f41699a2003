// qp_backward.cuh -- the backward pass of one instance (Alg. 3), shared by the
// backward kernel and the persistent serving kernel.
//
// At the relaxed point the forward kernel cached the two-level factors of the
// Newton matrix (eq. 14 with the inactive dv eliminated):
//   K_I = Q + G_I' W_I G_I = L L',   Y = F L^-T with F = [G_A; A],
//   C = D + Y Y' (+ a 1e-7 relative shift) = L_C L_C',  D = diag(1/W_A, 0),
// with W / (1/W), the row -> position map and the relaxed (x, y, z).  eq. 14
// is symmetric, so the adjoint solve of the implicit function theorem
// (App. A) is the same solve with right-hand side (-g, 0, 0), g = dl/dx:
//   [ K_I  F' ] [dx]   [ -g ]
//   [ F   -D  ] [mu] = [  0 ],     mu = (lambda, dy)
//   u = L^-1 r1,  C mu = Y u - r2,  dx = L^-T (u - Y' mu),
// refined `refine` times against the unshifted bounded system (residuals
// from Q, G, A, W, D in FP32; every coefficient is bounded, so they are
// accurate), then
//   dz_A = lambda (= W_A G_A dx),  dz_I = W_I (G_I dx)
// (dz = B_k(v) dv is eq. 13's fourth row with zero residuals), and as printed
// in Alg. 3
//   dQ = (dx x' + x dx')/2, dq = dx, dA = dy x' + y dx', db = -dy,
//   dG = dz x' + z dx',     dh = -dz.
// One CTA per instance: the factors are staged in shared memory once (the
// large variant reads them in place); Q, G, A are read where the caller keeps
// them, through L1 / L2, so that the small shared-memory layout lets five
// CTAs share an SM at n = 50 (copying Q, G, A as well left room for three).
// Each refinement residual takes one pass over the rows of [G; Q; A] with
// several rows' loads in flight per warp; the gradient blocks go out as
// coalesced 16-byte streaming stores.
//
// Bar: the barrier of the threads that run it (the whole CTA, or the first NT
// threads of a larger one); kCoh: read the data and the cache through L2
// (memory reused within one kernel's lifetime, see Solver::ld_ro).
#pragma once

#include "qp_device.cuh"
#include "qp_internal.h"

namespace qpgpu {

namespace {

template <bool kCoh>
__device__ __forceinline__ float ld_ro(const float* ptr) {
  if constexpr (kCoh) return __ldcg(ptr);
  else return __ldg(ptr);
}
template <bool kCoh>
__device__ __forceinline__ int ld_ro(const int* ptr) {
  if constexpr (kCoh) return __ldcg(ptr);
  else return __ldg(ptr);
}

struct BLayout {
  int ldk, ldc, ldx, ldg, nv, mv, pv, fv;
  int oK, oY, oC, oR, oPart, o_dinv, o_cdinv, o_mu, o_dmu, o_g, o_x, o_y, o_z, o_W,
      o_pos, o_act, o_e, o_dz, o_qdx, o_adx, total;
};

// global: the large-problem variant, whose factors are read in place from the
// (unpacked) gradient cache, so K, Y, C take no shared memory.
__host__ __device__ inline BLayout make_blayout(int n, int m, int p, int amax, int nthreads,
                                                bool global) {
  BLayout B;
  const int f = amax + p;
  B.ldk = ld_odd(n);
  B.ldc = ld_odd(f > 0 ? f : 1);
  B.ldx = round4(n);
  B.ldg = ld_vec(n);
  B.nv = round4(n); B.mv = round4(m > 0 ? m : 1); B.pv = round4(p > 0 ? p : 1);
  B.fv = round4(f > 0 ? f : 1);
  int o = 0;
  auto take = [&](int c) -> int { int r = o; o += round4(c); return r; };
  B.oK = take(global ? 0 : n * B.ldk);
  B.oY = take(global ? 0 : f * B.ldk);
  B.oC = take(global ? 0 : f * B.ldc);
  B.oR = take(2 * B.ldx);
  B.oPart = take((nthreads / 32) * B.nv);
  B.o_dinv = take(B.nv); B.o_cdinv = take(B.fv); B.o_mu = take(B.fv); B.o_dmu = take(B.fv);
  B.o_g = take(B.nv); B.o_x = take(B.nv); B.o_y = take(B.pv); B.o_z = take(B.mv);
  B.o_W = take(B.mv); B.o_pos = take(B.mv); B.o_act = take(B.fv); B.o_e = take(B.mv);
  B.o_dz = take(B.mv); B.o_qdx = take(B.nv); B.o_adx = take(B.pv);
  B.total = o;
  return B;
}

__device__ __forceinline__ int tri_row(int e) {
  int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  while (i * (i + 1) / 2 > e) --i;
  return i;
}

// dst[i][j] = f(i, j) for a rows x cols block, coalesced; 16-byte streaming
// stores when the block is 16-byte aligned and a multiple of 4 long.
template <int NT, class F>
__device__ __forceinline__ void write_block(float* dst, int rows, int cols, F f) {
  const int total = rows * cols;
  if (total == 0 || dst == nullptr) return;
  if ((total & 3) == 0 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e4 = threadIdx.x; e4 < (total >> 2); e4 += NT) {
      const int e = e4 << 2;
      int i = e / cols, j = e - i * cols;
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[k] = f(i, j);
        if (++j == cols) { j = 0; ++i; }
      }
      __stcs(d4 + e4, make_float4(v[0], v[1], v[2], v[3]));
    }
  } else {
    for (int e = threadIdx.x; e < total; e += NT) {
      const int i = e / cols, j = e - i * cols;
      __stcs(dst + e, f(i, j));
    }
  }
}

template <int SP>
__device__ void small_chol_solve(const float* C, int ldc, const float* cdinv, int nf, float* v) {
  const int lane = threadIdx.x & 31;
  float r[1][SP];
#pragma unroll
  for (int s2 = 0; s2 < SP; ++s2) {
    const int i = lane + 32 * s2;
    r[0][s2] = i < nf ? v[i] : 0.f;
  }
  warp_lower_solve<SP, 1>(C, ldc, cdinv, nf, r);
  warp_upper_solve<SP, 1>(C, ldc, cdinv, nf, r);
#pragma unroll
  for (int s2 = 0; s2 < SP; ++s2) {
    const int i = lane + 32 * s2;
    if (i < nf) v[i] = r[0][s2];
  }
}

// One pass over the rows of [G; Q; A] (each row of the caller's arrays, row
// stride n) with v = dx held in registers (lane owns columns lane + 32 s):
//   e = G dx,  qdx = Q dx,  adx = A dx,
// and, when `accumulate`, the per-warp column sums of
//   G' t + A' mu_y,   t_r = W_r e_r (inactive rows), mu_pos(r) (active rows),
// written to part[w][0 .. n) (summed over warps by the caller, in warp order).
// Each warp takes U consecutive rows at a time, so U x S loads are in flight
// per lane; every element of G, Q, A is read once per pass.  with_qa = false:
// G rows only (e = G dx).  Ends with a barrier.
template <int NT, int S, int U, class Bar, bool kCoh>
__device__ __forceinline__ void rows_pass_S(const float* G, const float* Q, const float* A, int m,
                                            int n, int p, int a, const float* dx, const float* W,
                                            const int* pos, const float* mu, float* e, float* qdx,
                                            float* adx, float* part, int ldp, bool accumulate,
                                            bool with_qa) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nw = NT / 32;
  float xr[S], acc[S];
#pragma unroll
  for (int s2 = 0; s2 < S; ++s2) {
    const int c = lane + 32 * s2;
    xr[s2] = c < n ? dx[c] : 0.f;
    acc[s2] = 0.f;
  }
  const int nrows = with_qa ? m + n + p : m;
  for (int r0 = w * U; r0 < nrows; r0 += nw * U) {
    float v[U][S];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      const float* row = r < m ? G + (size_t)r * n
                               : (r < m + n ? Q + (size_t)(r - m) * n : A + (size_t)(r - m - n) * n);
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int c = lane + 32 * s2;
        v[u][s2] = (r < nrows && c < n) ? ld_ro<kCoh>(row + c) : 0.f;
      }
    }
    float d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      d[u] = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) d[u] = fmaf(v[u][s2], xr[s2], d[u]);
    }
    // butterfly: every lane ends with the same sum (addition commutes)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < U; ++u) d[u] += __shfl_xor_sync(kFull, d[u], o);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r >= nrows) break;
      float coef = 0.f;
      if (r < m) {
        if (lane == 0) e[r] = d[u];
        const int k = pos[r];
        coef = k < 0 ? W[r] * d[u] : mu[k];
      } else if (r < m + n) {
        if (lane == 0) qdx[r - m] = d[u];
      } else {
        if (lane == 0) adx[r - m - n] = d[u];
        coef = mu[a + (r - m - n)];
      }
      if (accumulate) {
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc[s2] = fmaf(coef, v[u][s2], acc[s2]);
      }
    }
  }
  if (accumulate) {
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int c = lane + 32 * s2;
      if (c < n) part[w * ldp + c] = acc[s2];
    }
  }
  Bar::sync();
}

template <int NT, bool kGlobal, class Bar, bool kCoh>
__device__ __forceinline__ void rows_pass(const float* G, const float* Q, const float* A, int m,
                                          int n, int p, int a, const float* dx, const float* W,
                                          const int* pos, const float* mu, float* e, float* qdx,
                                          float* adx, float* part, int ldp, bool accumulate,
                                          bool with_qa) {
  if (n <= 32)
    rows_pass_S<NT, 1, 4, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp, accumulate,
                          with_qa);
  else if (n <= 64)
    rows_pass_S<NT, 2, 4, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp, accumulate,
                          with_qa);
  else if (n <= 96)
    rows_pass_S<NT, 3, 4, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp, accumulate,
                          with_qa);
  else if (!kGlobal || n <= 128)
    rows_pass_S<NT, 4, 4, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp, accumulate,
                          with_qa);
  else if constexpr (kGlobal) {
    if (n <= 192)
      rows_pass_S<NT, 6, 2, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp,
                            accumulate, with_qa);
    else
      rows_pass_S<NT, 8, 2, Bar, kCoh>(G, Q, A, m, n, p, a, dx, W, pos, mu, e, qdx, adx, part, ldp,
                            accumulate, with_qa);
  }
}

// Solve [K_I F'; F -D] (d, t) = (r1, r2) with the cached factors: r1 in R
// (row 0), r2 in t; the solution overwrites both.  kMaxS: warp-solve length
// bound of the K part in units of 32 rows (4 on chip, 8 for the large
// variant, whose C part goes to 320 rows).
template <int NT, int kMaxS, class Bar, bool kCoh = false>
__device__ void two_level_solve(const float* K, int ldk, const float* dinv, const float* Y,
                                const float* C, int ldc, const float* cdinv, int n, int nf,
                                float* R, int ldx, float* t, float* part = nullptr) {
  const int tid = threadIdx.x;
  if constexpr (kMaxS > 4) {
    // the large variant: factors in global memory.  Blocked triangular solves
    // with every warp, and the products with Y as coalesced row sweeps
    // (per-warp column sums in part, nw x round4(n) floats, added in warp
    // order); part[0 .. nf) first holds Y R.
    constexpr int nw = NT / 32;
    const int nv = (n + 3) & ~3;
    block_trsv<NT, false, Bar>(K, ldk, dinv, n, R, nullptr);
    if (nf > 0) {
      {
        const float* xv[1] = {R};
        float* dv[1] = {part};
        warp_rows_n<NT, 4, 1, 0, false, kCoh>(Y, ldk, nf, n, xv, dv, nullptr, nullptr, 0);
      }
      Bar::sync();
      for (int k = tid; k < nf; k += NT) t[k] = part[k] - t[k];
      Bar::sync();
      block_trsv<NT, false, Bar>(C, ldc, cdinv, nf, t, nullptr);
      block_trsv<NT, true, Bar>(C, ldc, cdinv, nf, t, nullptr);
      {
        const float* cw[1] = {t};
        warp_rows_n<NT, 4, 0, 1, false, kCoh>(Y, ldk, nf, n, nullptr, nullptr, cw, part, nv);
      }
      Bar::sync();
      for (int i = tid; i < n; i += NT) {
        float acc = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) acc += part[w2 * nv + i];
        R[i] -= acc;
      }
      Bar::sync();
    }
    block_trsv<NT, true, Bar>(K, ldk, dinv, n, R, nullptr);
    return;
  }
  solve_rows<NT, false, kMaxS, Bar>(K, ldk, dinv, n, R, ldx, 0, 1);
  if (nf > 0) {
    for (int k = tid; k < nf; k += NT) {
      float acc = 0.f;
      for (int i = 0; i < n; ++i) acc = fmaf(Y[k * ldk + i], R[i], acc);
      t[k] = acc - t[k];
    }
    Bar::sync();
    if (tid < 32) {
      if (nf <= 32) small_chol_solve<1>(C, ldc, cdinv, nf, t);
      else if (nf <= 64) small_chol_solve<2>(C, ldc, cdinv, nf, t);
      else if (nf <= 96) small_chol_solve<3>(C, ldc, cdinv, nf, t);
      else if (kMaxS <= 4 || nf <= 128) small_chol_solve<4>(C, ldc, cdinv, nf, t);
      else if constexpr (kMaxS > 4) {
        if (nf <= 160) small_chol_solve<5>(C, ldc, cdinv, nf, t);
        else if (nf <= 192) small_chol_solve<6>(C, ldc, cdinv, nf, t);
        else if (nf <= 224) small_chol_solve<7>(C, ldc, cdinv, nf, t);
        else if (nf <= 256) small_chol_solve<8>(C, ldc, cdinv, nf, t);
        else if (nf <= 288) small_chol_solve<9>(C, ldc, cdinv, nf, t);
        else small_chol_solve<10>(C, ldc, cdinv, nf, t);
      }
    }
    Bar::sync();
    for (int i = tid; i < n; i += NT) {
      float acc = R[i];
      for (int k = 0; k < nf; ++k) acc = fmaf(-Y[k * ldk + i], t[k], acc);
      R[i] = acc;
    }
    Bar::sync();
  }
  solve_rows<NT, true, kMaxS, Bar>(K, ldk, dinv, n, R, ldx, 0, 1);
}

template <int NT, bool kGlobal, class Bar = CtaBar, bool kCoh = false>
__device__ __forceinline__ void backward_body(const BwdParams& P, int bi) {
  extern __shared__ __align__(16) float sm[];
  const int n = P.n, m = P.m, p = P.p, t = threadIdx.x;
  const BLayout B = make_blayout(n, m, p, P.amax, NT, kGlobal);
  const CacheLayout cl = cache_layout(n, m, p, P.amax, kGlobal);
  const float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
  // the factors: staged in shared memory, or (large variant) read in place
  float* K = kGlobal ? const_cast<float*>(c + cl.oL) : sm + B.oK;
  float* Y = kGlobal ? const_cast<float*>(c + cl.oY) : sm + B.oY;
  float* C = kGlobal ? const_cast<float*>(c + cl.oLC) : sm + B.oC;
  const int ldk = kGlobal ? cl.ldk : B.ldk;
  const int ldc = kGlobal ? cl.ldc : B.ldc;
  float* R = sm + B.oR;
  float* part = sm + B.oPart;  // per-warp column sums of the row pass
  float* dinv = sm + B.o_dinv;
  float* cdinv = sm + B.o_cdinv;
  float* mu = sm + B.o_mu;
  float* dmu = sm + B.o_dmu;
  float* gv = sm + B.o_g;
  float* xs = sm + B.o_x;
  float* ys = sm + B.o_y;
  float* zs = sm + B.o_z;
  float* Ws = sm + B.o_W;
  int* pos = reinterpret_cast<int*>(sm + B.o_pos);
  int* act = reinterpret_cast<int*>(sm + B.o_act);
  float* e = sm + B.o_e;
  float* dz = sm + B.o_dz;
  float* qdx = sm + B.o_qdx;  // Q dx (n)
  float* adx = sm + B.o_adx;  // A dx (p)
  const int a = reinterpret_cast<const int*>(c + cl.oHdr)[0];
  const int nf = reinterpret_cast<const int*>(c + cl.oHdr)[1];
  int refine = reinterpret_cast<const int*>(c + cl.oHdr)[2];
  refine = refine < 0 ? 0 : (refine > 16 ? 16 : refine);
  // a cache that was not written by a forward solve of this size cannot index
  // out of bounds: its gradients come out NaN instead
  const bool valid = a >= 0 && a <= P.amax && nf == a + p;
  // ---- stage the cached factors and the point ----
  for (int i = t; i < B.total; i += NT) sm[i] = 0.0f;
  Bar::sync();
  // the data stay in the caller's memory (row stride n)
  const float* const Qm = P.Q + (size_t)bi * n * n;
  const float* const Gm = P.G + (size_t)bi * m * n;
  const float* const Am = P.A + (size_t)bi * p * n;
  const int nfl = valid ? nf : 0;
  if (kGlobal) {
    // factors stay in the cache: only the reciprocal pivots go to shared memory
    for (int i = t; i < n; i += NT) dinv[i] = 1.0f / ld_ro<kCoh>(c + cl.oL + i * ldk + i);
    for (int i = t; i < nfl; i += NT) cdinv[i] = 1.0f / ld_ro<kCoh>(c + cl.oLC + i * ldc + i);
  } else {
    const int nl = n * (n + 1) / 2;
    for (int e2 = t; e2 < nl; e2 += NT) {
      const int i = tri_row(e2), j = e2 - i * (i + 1) / 2;
      const float v = ld_ro<kCoh>(c + cl.oL + e2);
      K[i * ldk + j] = v;
      if (i == j) dinv[i] = 1.0f / v;
    }
    for (int e2 = t; e2 < nfl * n; e2 += NT) {
      const int k = e2 / n, i = e2 - k * n;
      Y[k * ldk + i] = ld_ro<kCoh>(c + cl.oY + e2);
    }
    const int fl = nfl * (nfl + 1) / 2;
    for (int e2 = t; e2 < fl; e2 += NT) {
      const int i = tri_row(e2), j = e2 - i * (i + 1) / 2;
      const float v = ld_ro<kCoh>(c + cl.oLC + e2);
      C[i * ldc + j] = v;
      if (i == j) cdinv[i] = 1.0f / v;
    }
  }
  for (int i = t; i < n; i += NT) {
    xs[i] = ld_ro<kCoh>(c + cl.ox + i);
    gv[i] = ld_ro<kCoh>(P.g + (size_t)bi * n + i);
    R[i] = -gv[i];
  }
  for (int k = t; k < p; k += NT) ys[k] = ld_ro<kCoh>(c + cl.oy + k);
  int bad = valid ? 0 : 1;
  const int acap = valid ? a : 0;  // an unchecked header must not bound the row map
  for (int r = t; r < m; r += NT) {
    zs[r] = ld_ro<kCoh>(c + cl.oz + r);
    Ws[r] = ld_ro<kCoh>(c + cl.oW + r);
    int k = ld_ro<kCoh>(reinterpret_cast<const int*>(c + cl.oPos) + r);
    if (k >= acap || k < -1) { k = -1; bad = 1; }
    pos[r] = k;
    if (k >= 0) act[k] = r;
  }
  if (Bar::sync_or(bad)) {
    // a cache slot this call cannot use (never written, or overwritten):
    // NaN gradients, recorded as the backward stage's
    if (P.diag && t == 0) {
      int32_t* dw = P.diag + bi;
      if ((*dw & QP_STAGE_MASK) == QP_STAGE_NONE) *dw |= QP_STAGE_BACKWARD;
    }
    const float nanv = NAN;
    if (P.dQ) for (int i = t; i < n * n; i += NT) P.dQ[(size_t)bi * n * n + i] = nanv;
    if (P.dq) for (int i = t; i < n; i += NT) P.dq[(size_t)bi * n + i] = nanv;
    if (P.dA) for (int i = t; i < p * n; i += NT) P.dA[(size_t)bi * p * n + i] = nanv;
    if (P.db) for (int i = t; i < p; i += NT) P.db[(size_t)bi * p + i] = nanv;
    if (P.dG) for (int i = t; i < m * n; i += NT) P.dG[(size_t)bi * m * n + i] = nanv;
    if (P.dh) for (int i = t; i < m; i += NT) P.dh[(size_t)bi * m + i] = nanv;
    return;
  }
  // ---- adjoint solve, then refinement against the bounded system ----
  two_level_solve<NT, kGlobal ? 8 : 4, Bar, kCoh>(K, ldk, dinv, Y, C, ldc, cdinv, n, nf, R, B.ldx, mu,
                                                 part);
  float* dx = R + B.ldx;  // accumulated solution; R row 0 is the work row
  for (int i = t; i < n; i += NT) dx[i] = R[i];
  Bar::sync();
  // Sweep it < refine: one row pass gives e = G dx, Q dx, A dx and the column
  // sums of G' t + A' mu_y; r1 = -g - (K_I dx + F' mu) = -g - (Q dx + G' t +
  // A' mu_y), r2 = -(F dx - D mu).  The last pass (it == refine) only forms
  // e = G dx for dz.
  for (int it = 0;; ++it) {
    const bool last = it == refine;
    rows_pass<NT, kGlobal, Bar, kCoh>(Gm, Qm, Am, m, n, p, a, dx, Ws, pos, mu, e, qdx, adx, part, B.nv, !last,
                           !last);
    if (last) break;
    for (int i = t; i < n; i += NT) {
      float acc = qdx[i];
      for (int w2 = 0; w2 < NT / 32; ++w2) acc += part[w2 * B.nv + i];
      R[i] = -gv[i] - acc;
    }
    for (int k = t; k < nf; k += NT) {
      if (k < a) {
        const int r = act[k];
        dmu[k] = -(e[r] - Ws[r] * mu[k]);  // r2 = -(F dx - D mu), D = 1/W on active rows
      } else {
        dmu[k] = -adx[k - a];
      }
    }
    Bar::sync();
    two_level_solve<NT, kGlobal ? 8 : 4, Bar, kCoh>(K, ldk, dinv, Y, C, ldc, cdinv, n, nf, R, B.ldx,
                                                   dmu, part);
    for (int i = t; i < n; i += NT) dx[i] += R[i];
    for (int k = t; k < nf; k += NT) mu[k] += dmu[k];
    Bar::sync();
  }
  const float* dy = mu + a;
  // ---- dz: active rows from the multipliers, inactive rows W (G dx) ----
  for (int r = t; r < m; r += NT) {
    const int k = pos[r];
    dz[r] = k >= 0 ? mu[k] : Ws[r] * e[r];
  }
  Bar::sync();
  if (P.diag) {
    // diagnostics: a non-finite adjoint solution is the backward stage's,
    // unless the solve already recorded an earlier stage
    bool bad = false;
    for (int i = t; i < n; i += NT) bad |= !isfinite(dx[i]);
    for (int k = t; k < p; k += NT) bad |= !isfinite(dy[k]);
    for (int r = t; r < m; r += NT) bad |= !isfinite(dz[r]);
    if (Bar::sync_or(bad ? 1 : 0) && t == 0) {
      int32_t* dw = P.diag + bi;
      if ((*dw & QP_STAGE_MASK) == QP_STAGE_NONE) *dw |= QP_STAGE_BACKWARD;
    }
  }
  // ---- gradient blocks (Alg. 3) ----
  if (P.dQ)
    write_block<NT>(P.dQ + (size_t)bi * n * n, n, n, [&](int i, int j) {
      return 0.5f * fmaf(dx[i], xs[j], xs[i] * dx[j]);
    });
  if (P.dG)
    write_block<NT>(P.dG + (size_t)bi * m * n, m, n, [&](int i, int j) {
      return fmaf(dz[i], xs[j], zs[i] * dx[j]);
    });
  if (P.dA)
    write_block<NT>(P.dA + (size_t)bi * p * n, p, n, [&](int i, int j) {
      return fmaf(dy[i], xs[j], ys[i] * dx[j]);
    });
  if (P.dq)
    for (int i = t; i < n; i += NT) __stcs(P.dq + (size_t)bi * n + i, dx[i]);
  if (P.db)
    for (int k = t; k < p; k += NT) __stcs(P.db + (size_t)bi * p + k, -dy[k]);
  if (P.dh)
    for (int r = t; r < m; r += NT) __stcs(P.dh + (size_t)bi * m + r, -dz[r]);
}

}  // namespace

}  // namespace qpgpu
