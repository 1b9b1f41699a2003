// qp_forward.cuh -- batched implicit-complementarity IPM (Alg. 1, Alg. 2) for
// QPs whose data fit in one SM's shared memory.  One CTA solves one QP.
//
// Per Newton iteration (Alg. 1):
//   v = z - s, kappa = s'z / m_ineq                       (manifold coordinates)
//   r_t = Qx + q + G'z + A'y, r_e = Ax - b, r_i = Gx + s - h,
//   r_z = z - b_k(v), r_s = s - b_k(-v)                  (eq. 4, eq. 10)
//   stop if the residual measure < tol
//   W = B_k(v) / B_k(-v) = b_k(v) / b_k(-v)              (eq. 12 with b'(v) = b(v)/rho)
//   K = Q + G' W G;  K = L L';  U = L^-1 A';  S = U'U = L_S L_S'
//   eq. 14 with dv eliminated:  K dx + A'dy = -r_t + G't,  A dx = -r_e,
//     t = r_z - W (r_i - r_s) + r_kappa / b_k(-v)
//   The solution is affine in r_kappa = kappa - kappa_target, so one pass over
//   the factor solves for the two right-hand sides t_A = r_z - W(r_i - r_s) and
//   t_B = 1/b_k(-v); any kappa_target then costs only vector work:
//     dx = dx_A + r_kappa dx_B (same for dy and e = G dx),
//     ds = -e - r_i,   dz = -r_z + W (e + r_i - r_s) - r_kappa / b_k(-v),
//     dv = dz - ds + r_z - r_s,  dkappa = -r_kappa       (eq. 13 rows 3-6)
//   predictor kappa_target = 0 -> alpha_aff (eq. 7), mu_aff, sigma = (mu_aff/kappa)^3;
//   corrector kappa_target = max(sigma kappa, kappa_min);
//   alpha from eq. 7;  x += a dx, y += a dy, v += a dv, kappa += a dkappa;
//   z = b_k(v), s = b_k(-v)                               (retraction, eq. 11, App. C)
//
// Alg. 2 (relax) repeats the step with kappa_target = kappa_relax from the
// solution, then the Newton matrix is factored once more at the relaxed point
// and cached with W and the relaxed (x, y, z) for the backward pass (Alg. 3).
//
// The explicit-complementarity ablation (eq. 6 / eq. 8, Mehrotra predictor-
// corrector, fraction-to-boundary 0.99) uses the same factorisation with
// W = z ./ s and a second solve for the corrector.
#pragma once
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qpgpu {

namespace fwd {

constexpr int ST_SOLVED = 0, ST_MAX_ITER = 1, ST_STALLED = 2, ST_NUMERICAL = 3, ST_BAD_INPUT = 4;

template <int NT>
struct Solver {
  Layout L;
  float *Q, *G, *A, *K, *X, *S, *col, *red;
  float *q, *x, *rt, *dinv, *tn, *sdinv;
  float *b, *y, *re, *r3a, *r3b, *dya, *dyb;
  float *h, *z, *s, *ri, *rz, *rs, *W, *ibs, *ea, *eb, *ta, *tb;
  int parity;
  float qn, bn, hn;  // |q|_inf, |b|_inf, |h|_inf

  __device__ void bind(float* sm, int n, int m, int p) {
    L = make_layout(n, m, p, NT);
    Q = sm + L.oQ; G = sm + L.oG; A = sm + L.oA; K = sm + L.oK; X = sm + L.oX; S = sm + L.oS;
    col = sm + L.oCol; red = sm + L.oRed;
    q = sm + L.o_q; x = sm + L.o_x; rt = sm + L.o_rt; dinv = sm + L.o_dinv; tn = sm + L.o_tn;
    sdinv = sm + L.o_sdinv;
    b = sm + L.o_b; y = sm + L.o_y; re = sm + L.o_re; r3a = sm + L.o_r3a; r3b = sm + L.o_r3b;
    dya = sm + L.o_dya; dyb = sm + L.o_dyb;
    h = sm + L.o_h; z = sm + L.o_z; s = sm + L.o_s; ri = sm + L.o_ri; rz = sm + L.o_rz;
    rs = sm + L.o_rs; W = sm + L.o_W; ibs = sm + L.o_ibs; ea = sm + L.o_ea; eb = sm + L.o_eb;
    ta = sm + L.o_ta; tb = sm + L.o_tb;
    parity = 0;
  }

  // ---- load one instance into shared memory (pads stay zero) ----
  // Returns false if any datum is not finite.
  __device__ bool load(const FwdParams& P, int bi, float* sm) {
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    for (int i = t; i < L.total; i += NT) sm[i] = 0.0f;
    __syncthreads();
    const float* gQ = P.Q + (size_t)bi * n * n;
    const float* gG = P.G + (size_t)bi * m * n;
    const float* gA = P.A + (size_t)bi * p * n;
    float chk = 0.f;  // 1 if some datum is NaN or infinite
    for (int e = t; e < n * n; e += NT) {
      const int r = e / n, c = e - r * n;
      const float v = gQ[e];
      chk = isfinite(v) ? chk : 1.0f;
      Q[r * L.ldg + c] = v;
    }
    for (int e = t; e < m * n; e += NT) {
      const int r = e / n, c = e - r * n;
      const float v = gG[e];
      chk = isfinite(v) ? chk : 1.0f;
      G[r * L.ldg + c] = v;
    }
    for (int e = t; e < p * n; e += NT) {
      const int r = e / n, c = e - r * n;
      const float v = gA[e];
      chk = isfinite(v) ? chk : 1.0f;
      A[r * L.ldg + c] = v;
    }
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
    block_reduce<NT, 4>(v, red, parity, OpMax());
    qn = v[1]; bn = v[2]; hn = v[3];
    return v[0] == 0.0f;
  }

  // ---- factorisation of the reduced Newton matrix for the current W ----
  __device__ bool factor() {
    const int n = L.n, p = L.p, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    syrk_gwg<NT>(Q, L.ldg, G, W, L.m, n, K, L.ldk);
    bool ok = cholesky<NT>(K, L.ldk, n, dinv);
    if (p > 0) {
      for (int k = w; k < p; k += NT / 32)
        for (int i = l; i < n; i += 32) X[k * L.ldx + i] = A[k * L.ldg + i];
      __syncthreads();
      solve_rows<NT, false>(K, L.ldk, dinv, n, X, L.ldx, 0, p);  // U' rows = L^-1 a_k
      const int np = p * (p + 1) / 2;
      for (int e = threadIdx.x; e < np; e += NT) {
        int a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        while (a * (a + 1) / 2 > e) --a;
        const int c = e - a * (a + 1) / 2;
        S[a * L.lds + c] = row_dot(X, L.ldx, a, X + c * L.ldx, L.nv);
      }
      __syncthreads();
      ok = cholesky<NT>(S, L.lds, p, sdinv) && ok;
    }
    return ok;
  }

  // Small p x p solves L_S L_S' y = r for one right-hand side held by a warp.
  template <int SP>
  __device__ void small_solve(float* v) {
    const int lane = threadIdx.x & 31;
    float r[1][SP];
#pragma unroll
    for (int s2 = 0; s2 < SP; ++s2) {
      const int i = lane + 32 * s2;
      r[0][s2] = i < L.p ? v[i] : 0.f;
    }
    warp_lower_solve<SP, 1>(S, L.lds, sdinv, L.p, r);
    warp_upper_solve<SP, 1>(S, L.lds, sdinv, L.p, r);
#pragma unroll
    for (int s2 = 0; s2 < SP; ++s2) {
      const int i = lane + 32 * s2;
      if (i < L.p) v[i] = r[0][s2];
    }
  }

  // ---- solve K dx + A'dy = r1_k, A dx = r3_k for nrhs (1 or 2) systems ----
  // r1_k in X row p+k, r3 in r3a/r3b; dx_k returned in X row p+k, dy in dya/dyb.
  __device__ void solve(int nrhs) {
    const int n = L.n, p = L.p, t = threadIdx.x, w = t >> 5;
    solve_rows<NT, false>(K, L.ldk, dinv, n, X, L.ldx, p, nrhs);
    if (p > 0) {
      for (int e = t; e < p * nrhs; e += NT) {
        const int k = e / p, a = e - k * p;
        float* dy = k == 0 ? dya : dyb;
        const float* r3 = k == 0 ? r3a : r3b;
        dy[a] = row_dot(X, L.ldx, a, X + (p + k) * L.ldx, L.nv) - r3[a];
      }
      __syncthreads();
      if (w < nrhs) {
        float* dy = w == 0 ? dya : dyb;
        if (p <= 32) small_solve<1>(dy);
        else if (p <= 64) small_solve<2>(dy);
        else if (p <= 96) small_solve<3>(dy);
        else small_solve<4>(dy);
      }
      __syncthreads();
      for (int e = t; e < n * nrhs; e += NT) {
        const int k = e / n, i = e - k * n;
        const float* dy = k == 0 ? dya : dyb;
        float acc = X[(p + k) * L.ldx + i];
        for (int a = 0; a < p; ++a) acc = fmaf(-X[a * L.ldx + i], dy[a], acc);
        X[(p + k) * L.ldx + i] = acc;
      }
      __syncthreads();
    }
    solve_rows<NT, true>(K, L.ldk, dinv, n, X, L.ldx, p, nrhs);
  }

  // ---- residuals (eq. 4) and the measure; for the implicit method also the
  // retraction residuals (eq. 10), W, 1/b_k(-v) and t_A.  kappa is s'z/m.
  // mode: 0 solve (complementarity term max z.*s), 1 relax (|kappa-kr|/kr).
  __device__ float residuals(const FwdParams& P, bool implicit, int mode, float& kappa) {
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    float ks[1] = {0.f};
    for (int r = t; r < m; r += NT) ks[0] = fmaf(z[r], s[r], ks[0]);
    block_reduce<NT, 1>(ks, red, parity, OpSum());
    kappa = m > 0 ? ks[0] / (float)m : 0.f;
    {
      const float* vv[1] = {z};
      float* oo[1] = {tn};
      col_dot<NT, 1>(G, L.ldg, m, n, vv, oo, col);
    }
    // maxima: 0 |rt| 1 |Qx| 2 |A'y| 3 |G'z| 4 |re| 5 |Ax| 6 |ri| 7 |Gx| 8 |s| 9 zs 10 |rz,rs| 11 |z|
    float mx[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) mx[k] = 0.f;
    float nanflag = 0.f;  // fmaxf drops NaN, so count non-finite values separately
    const int tot = n + m + p;
    for (int u = t; u < tot; u += NT) {
      if (u < n) {
        const int i = u;
        const float qx = row_dot(Q, L.ldg, i, x, L.nv);
        float aty = 0.f;
        for (int k = 0; k < p; ++k) aty = fmaf(A[k * L.ldg + i], y[k], aty);
        const float r = qx + q[i] + tn[i] + aty;
        rt[i] = r;
        nanflag += isfinite(r) ? 0.f : 1.f;
        mx[0] = fmaxf(mx[0], fabsf(r)); mx[1] = fmaxf(mx[1], fabsf(qx));
        mx[2] = fmaxf(mx[2], fabsf(aty)); mx[3] = fmaxf(mx[3], fabsf(tn[i]));
      } else if (u < n + m) {
        const int r = u - n;
        const float gx = row_dot(G, L.ldg, r, x, L.nv);
        const float rii = gx + s[r] - h[r];
        ri[r] = rii;
        nanflag += (isfinite(rii) && isfinite(z[r]) && isfinite(s[r])) ? 0.f : 1.f;
        mx[6] = fmaxf(mx[6], fabsf(rii)); mx[7] = fmaxf(mx[7], fabsf(gx));
        mx[8] = fmaxf(mx[8], fabsf(s[r])); mx[9] = fmaxf(mx[9], z[r] * s[r]);
        mx[11] = fmaxf(mx[11], fabsf(z[r]));
        if (implicit) {
          float bz, bs;
          retract_pair(z[r] - s[r], kappa, bz, bs);
          const float rzz = z[r] - bz, rss = s[r] - bs;
          rz[r] = rzz; rs[r] = rss;
          const float Wr = bz / bs;
          W[r] = Wr;
          ibs[r] = 1.0f / bs;
          ta[r] = rzz - Wr * (rii - rss);
          mx[10] = fmaxf(mx[10], fmaxf(fabsf(rzz), fabsf(rss)));
        } else {
          const float Wr = z[r] / s[r];
          W[r] = Wr;
          ibs[r] = 1.0f / s[r];
        }
      } else {
        const int k = u - n - m;
        const float ax = row_dot(A, L.ldg, k, x, L.nv);
        const float r = ax - b[k];
        re[k] = r;
        mx[4] = fmaxf(mx[4], fabsf(r)); mx[5] = fmaxf(mx[5], fabsf(ax));
      }
    }
    float v[13];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = mx[k];
    v[12] = nanflag;
    block_reduce<NT, 13>(v, red, parity, OpMax());
    if (v[12] > 0.f) return NAN;
    float comp = v[9];
    if (mode == 1) comp = fabsf(kappa - P.kappa_relax) / P.kappa_relax;
    if (P.norm_abs) {
      return fmaxf(fmaxf(fmaxf(v[0], v[4]), fmaxf(v[6], comp)), v[10]);
    }
    const float dt = fmaxf(fmaxf(1.0f, qn), fmaxf(fmaxf(v[1], v[2]), v[3]));
    const float de = fmaxf(fmaxf(1.0f, bn), v[5]);
    const float di = fmaxf(fmaxf(1.0f, hn), fmaxf(v[7], v[8]));
    const float dz = fmaxf(1.0f, fmaxf(v[11], v[8]));
    return fmaxf(fmaxf(fmaxf(v[0] / dt, v[4] / de), fmaxf(v[6] / di, comp)), v[10] / dz);
  }

  // Right-hand sides of the two implicit systems: r1_A = -r_t + G't_A, r1_B = G'(1/b(-v)).
  __device__ void implicit_rhs() {
    const int p = L.p;
    const float* vv[2] = {ta, ibs};
    float* oo[2] = {X + p * L.ldx, X + (p + 1) * L.ldx};
    col_dot<NT, 2>(G, L.ldg, L.m, L.n, vv, oo, col, rt, -1.0f);
    for (int k = threadIdx.x; k < p; k += NT) { r3a[k] = -re[k]; r3b[k] = 0.f; }
  }

  // e_A = G dx_A, e_B = G dx_B
  __device__ void g_times_dx(int nrhs) {
    const int p = L.p;
    for (int r = threadIdx.x; r < L.m; r += NT) {
      if (nrhs == 2) {
        float a, c;
        row_dot2(G, L.ldg, r, X + p * L.ldx, X + (p + 1) * L.ldx, L.nv, a, c);
        ea[r] = a; eb[r] = c;
      } else {
        ea[r] = row_dot(G, L.ldg, r, X + p * L.ldx, L.nv);
      }
    }
    __syncthreads();
  }

  // Step length (eq. 7) of the implicit direction for a given r_kappa; stores dv in tb.
  __device__ float implicit_alpha(float rk, bool store) {
    float amin[1] = {1.0f};
    for (int r = threadIdx.x; r < L.m; r += NT) {
      const float e = fmaf(rk, eb[r], ea[r]);
      const float dsr = -e - ri[r];
      const float dzr = -rz[r] + W[r] * (e + ri[r] - rs[r]) - rk * ibs[r];
      if (dsr < 0.f) amin[0] = fminf(amin[0], -s[r] / dsr);
      if (dzr < 0.f) amin[0] = fminf(amin[0], -z[r] / dzr);
      if (store) tb[r] = dzr - dsr + rz[r] - rs[r];
    }
    block_reduce<NT, 1>(amin, red, parity, OpMin());
    return amin[0];
  }

  __device__ float implicit_mu_aff(float rk, float alpha) {
    float acc[1] = {0.f};
    for (int r = threadIdx.x; r < L.m; r += NT) {
      const float e = fmaf(rk, eb[r], ea[r]);
      const float dsr = -e - ri[r];
      const float dzr = -rz[r] + W[r] * (e + ri[r] - rs[r]) - rk * ibs[r];
      acc[0] = fmaf(fmaf(alpha, dsr, s[r]), fmaf(alpha, dzr, z[r]), acc[0]);
    }
    block_reduce<NT, 1>(acc, red, parity, OpSum());
    return acc[0] / (float)L.m;
  }

  // x += a (dx_A + rk dx_B), y likewise, v += a dv, kappa' = kappa - a rk, retract.
  __device__ void implicit_update(float alpha, float rk, float kappa) {
    const int p = L.p, t = threadIdx.x;
    const float knew = kappa - alpha * rk;
    for (int i = t; i < L.n; i += NT)
      x[i] = fmaf(alpha, fmaf(rk, X[(p + 1) * L.ldx + i], X[p * L.ldx + i]), x[i]);
    for (int k = t; k < p; k += NT) y[k] = fmaf(alpha, fmaf(rk, dyb[k], dya[k]), y[k]);
    for (int r = t; r < L.m; r += NT) {
      const float vn = fmaf(alpha, tb[r], z[r] - s[r]);
      float bz, bs;
      retract_pair(vn, knew, bz, bs);
      z[r] = bz;
      s[r] = bs;
    }
    __syncthreads();
  }

  // CVXOPT-style start: (Q + G'G) x + A'y = -q + G'h, Ax = b; z = Gx - h, s = -z, shifted.
  __device__ bool initialize() {
    const int p = L.p, m = L.m, t = threadIdx.x;
    for (int r = t; r < m; r += NT) W[r] = 1.0f;
    __syncthreads();
    {
      const float* vv[1] = {h};
      float* oo[1] = {X + p * L.ldx};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col, q, -1.0f);
    }
    for (int k = t; k < p; k += NT) r3a[k] = b[k];
    __syncthreads();
    bool ok = factor();
    solve(1);
    for (int i = t; i < L.n; i += NT) x[i] = X[p * L.ldx + i];
    for (int k = t; k < p; k += NT) y[k] = dya[k];
    __syncthreads();
    float mx[4] = {-INFINITY, -INFINITY, 0.f, 0.f};
    for (int r = t; r < m; r += NT) {
      const float zr = row_dot(G, L.ldg, r, x, L.nv) - h[r];
      z[r] = zr;
      s[r] = -zr;
      mx[0] = fmaxf(mx[0], zr);   // -min(s)
      mx[1] = fmaxf(mx[1], -zr);  // -min(z)
      mx[2] = fmaxf(mx[2], fabsf(zr));
    }
    block_reduce<NT, 4>(mx, red, parity, OpMax());
    const float thr = -1e-8f * fmaxf(1.0f, mx[2]);
    const bool shs = mx[0] >= thr, shz = mx[1] >= thr;
    for (int r = t; r < m; r += NT) {
      if (shs) s[r] += 1.0f + mx[0];
      if (shz) z[r] += 1.0f + mx[1];
    }
    __syncthreads();
    return ok;
  }

  // Equality-only problem: one solve of [Q A'; A 0] is exact.
  __device__ bool solve_eq_only() {
    const int p = L.p, t = threadIdx.x;
    for (int i = t; i < L.n; i += NT) X[p * L.ldx + i] = -q[i];
    for (int k = t; k < p; k += NT) r3a[k] = b[k];
    __syncthreads();
    bool ok = factor();
    solve(1);
    for (int i = t; i < L.n; i += NT) x[i] = X[p * L.ldx + i];
    for (int k = t; k < p; k += NT) y[k] = dya[k];
    __syncthreads();
    return ok;
  }

  // ---- explicit complementarity (ablation): Mehrotra predictor-corrector ----
  // rhs t = -W r_i + r_c ./ s with r_c = z.*s (predictor) or the corrector term.
  __device__ float standard_step(float mu, float sigma_const) {
    const int p = L.p, m = L.m, t = threadIdx.x;
    // predictor system A: t_A = -W r_i + z
    for (int r = t; r < m; r += NT) ta[r] = -W[r] * ri[r] + z[r];
    __syncthreads();
    {
      const float* vv[1] = {ta};
      float* oo[1] = {X + p * L.ldx};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col, rt, -1.0f);
    }
    for (int k = t; k < p; k += NT) r3a[k] = -re[k];
    __syncthreads();
    bool ok = factor();
    solve(1);
    g_times_dx(1);
    // predictor ds, dz; alpha_aff
    float amin[1] = {1.0f};
    for (int r = t; r < m; r += NT) {
      const float dzr = W[r] * (ea[r] + ri[r]) - z[r];
      const float dsr = -ea[r] - ri[r];
      eb[r] = dzr;  // keep dz_aff
      tb[r] = dsr;  // keep ds_aff
      if (dsr < 0.f) amin[0] = fminf(amin[0], -s[r] / dsr);
      if (dzr < 0.f) amin[0] = fminf(amin[0], -z[r] / dzr);
    }
    block_reduce<NT, 1>(amin, red, parity, OpMin());
    const float aa = amin[0];
    float acc[1] = {0.f};
    for (int r = t; r < m; r += NT) acc[0] = fmaf(fmaf(aa, tb[r], s[r]), fmaf(aa, eb[r], z[r]), acc[0]);
    block_reduce<NT, 1>(acc, red, parity, OpSum());
    const float mua = acc[0] / (float)m;
    const float ratio = mua / mu;
    float sigma = ratio * ratio * ratio;  // Mehrotra
    if (!(sigma >= 0.f)) sigma = 0.f;
    if (sigma > 1.f) sigma = 1.f;
    if (sigma_const >= 0.f) sigma = sigma_const;
    const float smu = sigma * mu;
    // keep predictor dx, dy
    for (int i = t; i < L.n; i += NT) tn[i] = X[p * L.ldx + i];
    for (int k = t; k < p; k += NT) dyb[k] = dya[k];
    // corrector system C: r_c = ds_a.*dz_a - sigma mu  ->  t_C = r_c ./ s, r1 = G't_C
    for (int r = t; r < m; r += NT) ta[r] = (tb[r] * eb[r] - smu) * ibs[r];
    __syncthreads();
    {
      const float* vv[1] = {ta};
      float* oo[1] = {X + p * L.ldx};
      col_dot<NT, 1>(G, L.ldg, m, L.n, vv, oo, col);
    }
    for (int k = t; k < p; k += NT) r3a[k] = 0.f;
    __syncthreads();
    solve(1);
    g_times_dx(1);
    // total direction = predictor + corrector
    float amin2[1] = {1.0f};
    for (int r = t; r < m; r += NT) {
      const float e = ea[r];
      // ds = ds_a - e_C ; dz = dz_a + W e_C - t_C
      const float dsr = tb[r] - e;
      const float dzr = eb[r] + W[r] * e - ta[r];
      eb[r] = dzr;
      tb[r] = dsr;
      if (dsr < 0.f) amin2[0] = fminf(amin2[0], -s[r] / dsr);
      if (dzr < 0.f) amin2[0] = fminf(amin2[0], -z[r] / dzr);
    }
    block_reduce<NT, 1>(amin2, red, parity, OpMin());
    const float alpha = fminf(1.0f, 0.99f * amin2[0]);
    for (int i = t; i < L.n; i += NT) x[i] = fmaf(alpha, tn[i] + X[p * L.ldx + i], x[i]);
    for (int k = t; k < p; k += NT) y[k] = fmaf(alpha, dyb[k] + dya[k], y[k]);
    for (int r = t; r < m; r += NT) {
      z[r] = fmaf(alpha, eb[r], z[r]);
      s[r] = fmaf(alpha, tb[r], s[r]);
    }
    __syncthreads();
    return ok ? alpha : NAN;
  }

  // ---- whole instance ----
  __device__ void run(const FwdParams& P, int bi, float* sm) {
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    const bool implicit = P.formulation == 0;
    int status = ST_SOLVED, iters = 0;
    float meas = 0.f;
    const bool good = load(P, bi, sm);
    if (!good) {
      status = ST_BAD_INPUT;
      meas = NAN;
    } else if (m == 0) {
      if (!solve_eq_only()) status = ST_NUMERICAL;
      iters = 1;
      float kap;
      meas = residuals(P, implicit, 0, kap);
    } else {
      bool warm = false;
      if (P.warm_start) {
        float mn[1] = {INFINITY};
        for (int i = t; i < n; i += NT) x[i] = P.x[(size_t)bi * n + i];
        for (int k = t; k < p; k += NT) y[k] = P.y[(size_t)bi * p + k];
        for (int r = t; r < m; r += NT) {
          z[r] = P.z[(size_t)bi * m + r];
          s[r] = P.s[(size_t)bi * m + r];
          mn[0] = fminf(mn[0], fminf(z[r], s[r]));
        }
        block_reduce<NT, 1>(mn, red, parity, OpMin());
        warm = mn[0] > 0.f;
      }
      if (!warm && !initialize()) status = ST_NUMERICAL;
      // ---- Alg. 1 ----
      float best = INFINITY;
      int since_best = 0;
      for (int it = 0; status == ST_SOLVED; ++it) {
        float kappa;
        meas = residuals(P, implicit, 0, kappa);
        if (!(meas == meas)) { status = ST_NUMERICAL; break; }
        if (meas < P.tol) break;
        if (it >= P.max_iter) { status = ST_MAX_ITER; break; }
        if (meas < 0.9f * best) { best = meas; since_best = 0; }
        else if (++since_best >= 10) { status = ST_STALLED; break; }
        if (implicit) {
          implicit_rhs();
          if (!factor()) { status = ST_NUMERICAL; break; }
          solve(2);
          g_times_dx(2);
          float sigma;
          if (P.sigma_mode == 1) {
            sigma = P.sigma;
          } else {
            const float aa = implicit_alpha(kappa, false);
            const float mua = implicit_mu_aff(kappa, aa);
            const float ratio = mua / kappa;
            sigma = ratio * ratio * ratio;
            if (!(sigma >= 0.f)) sigma = 0.f;
            if (sigma > 1.f) sigma = 1.f;
          }
          const float kt = fmaxf(sigma * kappa, P.kappa_min);
          const float rk = kappa - kt;
          const float alpha = P.step_frac * implicit_alpha(rk, true);
          implicit_update(alpha, rk, kappa);
        } else {
          const float a = standard_step(kappa, P.sigma_mode == 1 ? P.sigma : -1.0f);
          if (!(a == a)) { status = ST_NUMERICAL; break; }
        }
        iters = it + 1;
      }
      // ---- Alg. 2 (relax) and the cached factor at the relaxed point ----
      if (P.cache && P.kappa_relax > 0.f && (status == ST_SOLVED || status == ST_MAX_ITER ||
                                             status == ST_STALLED)) {
        // write the solution of Alg. 1 now; the relaxed point only goes to the cache
        for (int i = t; i < n; i += NT) P.x[(size_t)bi * n + i] = x[i];
        for (int k = t; k < p; k += NT) P.y[(size_t)bi * p + k] = y[k];
        for (int r = t; r < m; r += NT) { P.z[(size_t)bi * m + r] = z[r]; P.s[(size_t)bi * m + r] = s[r]; }
        int rstatus = ST_MAX_ITER;
        const int rmax = P.relax_max_iter;
        for (int it = 0;; ++it) {
          float kappa;
          const float rm = residuals(P, true, 1, kappa);
          if (!(rm == rm)) { rstatus = ST_NUMERICAL; break; }
          if (rm < P.relax_tol) { rstatus = ST_SOLVED; break; }
          if (it >= rmax) break;
          implicit_rhs();
          if (!factor()) { rstatus = ST_NUMERICAL; break; }
          solve(2);
          g_times_dx(2);
          const float rk = kappa - P.kappa_relax;
          const float alpha = P.step_frac * implicit_alpha(rk, true);
          implicit_update(alpha, rk, kappa);
          ++iters;
        }
        if (status == ST_SOLVED) status = rstatus;
        // factor at the relaxed point: W = b_k(v)/b_k(-v) with kappa = kappa_relax
        for (int r = t; r < m; r += NT) {
          float bz, bs;
          retract_pair(z[r] - s[r], P.kappa_relax, bz, bs);
          W[r] = bz / bs;
        }
        __syncthreads();
        if (!factor() && status == ST_SOLVED) status = ST_NUMERICAL;
        write_cache(P, bi);
        if (t == 0) {
          if (P.status) P.status[bi] = status;
          if (P.iters) P.iters[bi] = iters;
          if (P.kkt) P.kkt[bi] = meas;
        }
        __syncthreads();
        return;
      }
    }
    if (P.cache && status != ST_BAD_INPUT) {
      // gradients at the solution itself (kappa_relax = 0) or the equality-only case
      if (m > 0) {
        for (int r = t; r < m; r += NT) W[r] = z[r] / s[r];
        __syncthreads();
        factor();
      }
      write_cache(P, bi);
    }
    // outputs
    const float nanv = NAN;
    for (int i = t; i < n; i += NT) P.x[(size_t)bi * n + i] = good ? x[i] : nanv;
    for (int k = t; k < p; k += NT) P.y[(size_t)bi * p + k] = good ? y[k] : nanv;
    for (int r = t; r < m; r += NT) {
      P.z[(size_t)bi * m + r] = good ? z[r] : nanv;
      P.s[(size_t)bi * m + r] = good ? s[r] : nanv;
    }
    if (t == 0) {
      if (P.status) P.status[bi] = status;
      if (P.iters) P.iters[bi] = iters;
      if (P.kkt) P.kkt[bi] = meas;
    }
    __syncthreads();
  }

  __device__ void write_cache(const FwdParams& P, int bi) {
    const int n = L.n, m = L.m, p = L.p, t = threadIdx.x;
    const CacheLayout cl = cache_layout(n, m, p);
    float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
    const int nl = n * (n + 1) / 2;
    for (int e = t; e < nl; e += NT) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      const int j = e - i * (i + 1) / 2;
      c[cl.oL + e] = K[i * L.ldk + j];
    }
    for (int e = t; e < p * n; e += NT) {
      const int k = e / n, i = e - k * n;
      c[cl.oU + e] = X[k * L.ldx + i];
    }
    const int pl = p * (p + 1) / 2;
    for (int e = t; e < pl; e += NT) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      const int j = e - i * (i + 1) / 2;
      c[cl.oLs + e] = S[i * L.lds + j];
    }
    for (int r = t; r < m; r += NT) { c[cl.oW + r] = W[r]; c[cl.oz + r] = z[r]; }
    for (int i = t; i < n; i += NT) c[cl.ox + i] = x[i];
    for (int k = t; k < p; k += NT) c[cl.oy + k] = y[k];
    __syncthreads();
  }
};

template <int NT>
__global__ void __launch_bounds__(NT) qp_forward_kernel(const FwdParams P) {
  extern __shared__ __align__(16) float sm[];
  Solver<NT> slv;
  slv.bind(sm, P.n, P.m, P.p);
  slv.run(P, blockIdx.x, sm);
}

}  // namespace fwd

// Instantiated once per block size in qp_forward_<NT>.cu.
template <int NT>
cudaError_t launch_forward_nt(const FwdParams& P, size_t smem, int grid, cudaStream_t st) {
  static bool configured = false;  // the attribute is per function and per process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fwd::qp_forward_kernel<NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fwd::qp_forward_kernel<NT><<<grid, NT, smem, st>>>(P);
  return cudaGetLastError();
}

template <int NT>
int forward_blocks_per_sm_nt(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(fwd::qp_forward_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd::qp_forward_kernel<NT>, NT, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace qpgpu
