// qp_device.cuh -- building blocks of the batched IPM kernels: retraction,
// reductions, G'WG, the blocked bordered Cholesky and triangular solves, and
// (for matrices in global memory) warp row sweeps and blocked solves.
//
// One CTA owns one QP at a time.  On chip every per-instance array lives in
// shared memory with strides chosen for the two access patterns used:
//   * "vector" strides (ldg): a multiple of 4 floats whose quarter is odd, so
//     thread-per-row float4 dot products and column reads are both free of
//     bank conflicts; pad columns are zero, so float4 reads past n add 0;
//   * "odd" strides (ldk) for the Cholesky factor, so that both a column
//     (forward substitution) and a row (back substitution) of L are read by a
//     warp without bank conflicts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qpgpu {

// Barrier policies of code that a whole CTA or a subset of a larger CTA runs.
// CtaBar: every thread of the CTA.
struct CtaBar {
  static __device__ __forceinline__ void sync() { __syncthreads(); }
  static __device__ __forceinline__ int sync_or(int v) { return __syncthreads_or(v); }
};
// GroupBar<N>: the CTA's first N threads (whole warps) on named barrier 2,
// while the CTA's other threads wait elsewhere (barrier 0 is the CTA's own,
// barrier 1 the factorisation's look-ahead).
template <int N>
struct GroupBar {
  static_assert(N % 32 == 0, "a group is whole warps");
  static __device__ __forceinline__ void sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(N) : "memory");
  }
  static __device__ __forceinline__ int sync_or(int v) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 2, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v), "n"(N)
        : "memory");
    return r;
  }
};

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRedK = 16;  // maximum quantities reduced by one block_reduce call

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }
__host__ __device__ inline int ld_vec(int n) {
  int l = round4(n < 1 ? 1 : n);
  if (((l >> 2) & 1) == 0) l += 4;
  return l;
}
__host__ __device__ inline int ld_odd(int n) { return n | 1; }

// ---------------------------------------------------------------------------
// Retraction (eq. 11) in the cancellation-free form of App. C, evaluated for
// both signs at once: bz = b_k(v), bs = b_k(-v).  bz*bs = kappa, bz - bs = v,
// bz + bs = sqrt(v^2 + 4 kappa).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void retract_pair(float v, float kappa, float& bz, float& bs) {
  float rho = sqrtf(fmaf(v, v, 4.0f * kappa));
  if (v >= 0.0f) {
    bz = 0.5f * (v + rho);
    bs = (2.0f * kappa) / (rho + v);
  } else {
    bz = (2.0f * kappa) / (rho - v);
    bs = 0.5f * (rho - v);
  }
}

// ---------------------------------------------------------------------------
// Block-wide reductions of K values at once; every thread gets the results.
// Two alternating buffers make back-to-back calls safe with one barrier each.
// ---------------------------------------------------------------------------
struct OpMax { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };
struct OpMin { __device__ float operator()(float a, float b) const { return fminf(a, b); } };
struct OpSum { __device__ float operator()(float a, float b) const { return a + b; } };

template <int NT, int K, class Op>
__device__ __forceinline__ void block_reduce(float (&v)[K], float* red, int& parity, Op op) {
  static_assert(K <= kRedK, "too many reduced values");
  static_assert(NT % 32 == 0 && NT <= 512, "whole warps, at most 16");
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = op(v[k], __shfl_xor_sync(kFull, v[k], o));
  // two buffers of (NT / 32) * kRedK floats: red holds 2 * (NT / 32) * kRedK
  float* buf = red + parity * ((NT / 32) * kRedK);
  parity ^= 1;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) buf[w * K + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float r = buf[k];
    for (int j = 1; j < NT / 32; ++j) r = op(r, buf[j * K + k]);
    v[k] = r;
  }
}

// ---------------------------------------------------------------------------
// Dot products with shared-memory matrices (row-major, stride ld, zero pads).
// ---------------------------------------------------------------------------
// Row r of M times vector x (length rounded up to 4, zero-padded).
__device__ __forceinline__ float row_dot(const float* M, int ld, int r, const float* x, int nv) {
  const float4* a = reinterpret_cast<const float4*>(M + r * ld);
  const float4* b = reinterpret_cast<const float4*>(x);
  float s0 = 0.f, s1 = 0.f;
  int k = 0;
  for (; k + 1 < (nv >> 2); k += 2) {
    float4 u = a[k], v = b[k], u2 = a[k + 1], v2 = b[k + 1];
    s0 = fmaf(u.x, v.x, s0); s0 = fmaf(u.y, v.y, s0); s0 = fmaf(u.z, v.z, s0); s0 = fmaf(u.w, v.w, s0);
    s1 = fmaf(u2.x, v2.x, s1); s1 = fmaf(u2.y, v2.y, s1); s1 = fmaf(u2.z, v2.z, s1); s1 = fmaf(u2.w, v2.w, s1);
  }
  if (k < (nv >> 2)) {
    float4 u = a[k], v = b[k];
    s0 = fmaf(u.x, v.x, s0); s0 = fmaf(u.y, v.y, s0); s0 = fmaf(u.z, v.z, s0); s0 = fmaf(u.w, v.w, s0);
  }
  return s0 + s1;
}

// One sweep over the rows of M (rows x n, row stride ld) in global memory,
// for matrices too large to stage: a warp takes U rows at a time with lanes
// over the columns (lane owns columns lane + 32 s, s < S), so every load is
// a coalesced segment of a row and U x S loads are in flight per lane.  For
// each row r it forms, in the same pass,
//   the ND row dots  dout[k][r] = M[r] . xv[k]          (butterfly sums), and
//   the NC column sums of cw[k][r] M[r][.]   into this warp's partials
//     part[(k * nw + w) * ldp + c]                        (nw = NT / 32),
// which the caller adds over the warps in a fixed order.  kUpper: row r
// counts only its columns c > r (a symmetric matrix kept as its strict upper
// triangle).  kL2: read through L2 (memory that a persistent CTA may have
// seen hold other data).  No barrier.
template <int NT, int S, int U, int ND, int NC, bool kUpper, bool kL2>
__device__ __forceinline__ void warp_rows(const float* M, int ld, int rows, int n,
                                          const float* const* xv, float* const* dout,
                                          const float* const* cw, float* part, int ldp) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nw = NT / 32;
  float xr[ND > 0 ? ND : 1][S], acc[NC > 0 ? NC : 1][S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int c = lane + 32 * s;
#pragma unroll
    for (int k = 0; k < ND; ++k) xr[k][s] = c < n ? xv[k][c] : 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k][s] = 0.f;
  }
  for (int r0 = w * U; r0 < rows; r0 += nw * U) {
    float v[U][S];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      const float* row = M + (size_t)r * ld;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int c = lane + 32 * s;
        const bool in = r < rows && c < n && (!kUpper || c > r);
        v[u][s] = in ? (kL2 ? __ldcg(row + c) : row[c]) : 0.f;
      }
    }
    if constexpr (ND > 0) {
      float d[U][ND];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < ND; ++k) {
          d[u][k] = 0.f;
#pragma unroll
          for (int s = 0; s < S; ++s) d[u][k] = fmaf(v[u][s], xr[k][s], d[u][k]);
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int k = 0; k < ND; ++k) d[u][k] += __shfl_xor_sync(kFull, d[u][k], o);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (r0 + u < rows) {
#pragma unroll
            for (int k = 0; k < ND; ++k) dout[k][r0 + u] = d[u][k];
          }
      }
    }
    if constexpr (NC > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u;
        if (r < rows) {
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const float wr = cw[k][r];
#pragma unroll
            for (int s = 0; s < S; ++s) acc[k][s] = fmaf(wr, v[u][s], acc[k][s]);
          }
        }
      }
    }
  }
  if constexpr (NC > 0) {
#pragma unroll
    for (int k = 0; k < NC; ++k)
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int c = lane + 32 * s;
        if (c < n) part[(k * nw + w) * ldp + c] = acc[k][s];
      }
  }
}

// warp_rows for the column count n: S = ceil(n / 32) register slots per lane
// (n <= 256).
template <int NT, int U, int ND, int NC, bool kUpper, bool kL2>
__device__ __forceinline__ void warp_rows_n(const float* M, int ld, int rows, int n,
                                            const float* const* xv, float* const* dout,
                                            const float* const* cw, float* part, int ldp) {
  if (n <= 32)
    warp_rows<NT, 1, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 64)
    warp_rows<NT, 2, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 96)
    warp_rows<NT, 3, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 128)
    warp_rows<NT, 4, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 160)
    warp_rows<NT, 5, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 192)
    warp_rows<NT, 6, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else if (n <= 224)
    warp_rows<NT, 7, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
  else
    warp_rows<NT, 8, U, ND, NC, kUpper, kL2>(M, ld, rows, n, xv, dout, cw, part, ldp);
}

// Two vectors at once.
__device__ __forceinline__ void row_dot2(const float* M, int ld, int r, const float* x,
                                         const float* y, int nv, float& ox, float& oy) {
  const float4* a = reinterpret_cast<const float4*>(M + r * ld);
  const float4* bx = reinterpret_cast<const float4*>(x);
  const float4* by = reinterpret_cast<const float4*>(y);
  float sx = 0.f, sy = 0.f;
  for (int k = 0; k < (nv >> 2); ++k) {
    float4 u = a[k], v = bx[k], w = by[k];
    sx = fmaf(u.x, v.x, sx); sx = fmaf(u.y, v.y, sx); sx = fmaf(u.z, v.z, sx); sx = fmaf(u.w, v.w, sx);
    sy = fmaf(u.x, w.x, sy); sy = fmaf(u.y, w.y, sy); sy = fmaf(u.z, w.z, sy); sy = fmaf(u.w, w.w, sy);
  }
  ox = sx;
  oy = sy;
}

// out_k[c] = sum_r M[r][c] * v_k[r] for c < cols, K = 1 or 2 vectors; the
// row range is split over thread groups and reduced in a fixed order
// (deterministic).  Uses col scratch of 2*NT floats; ends with a barrier.
template <int NT, int K>
__device__ void col_dot(const float* M, int ld, int rows, int cols, const float* const (&v)[K],
                        float* const (&out)[K], float* col, const float* add0 = nullptr,
                        float scale0 = 1.0f) {
  const int t = threadIdx.x;
  int ns = NT / (cols > 0 ? cols : 1);
  if (ns < 1) ns = 1;
  if (ns > 16) ns = 16;
  if (ns == 1) {
    for (int c = t; c < cols; c += NT) {
      float acc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = 0.f;
      for (int r = 0; r < rows; ++r) {
        float g = M[r * ld + c];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = fmaf(g, v[k][r], acc[k]);
      }
      out[0][c] = add0 ? fmaf(scale0, add0[c], acc[0]) : acc[0];
#pragma unroll
      for (int k = 1; k < K; ++k) out[k][c] = acc[k];
    }
    __syncthreads();
    return;
  }
  const int c = t % cols, sp = t / cols;
  if (sp < ns) {
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.f;
    for (int r = sp; r < rows; r += ns) {
      float g = M[r * ld + c];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fmaf(g, v[k][r], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) col[k * NT + sp * cols + c] = acc[k];
  }
  __syncthreads();
  for (int cc = t; cc < cols; cc += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float s = col[k * NT + cc];
      for (int j = 1; j < ns; ++j) s += col[k * NT + j * cols + cc];
      if (k == 0 && add0) s = fmaf(scale0, add0[cc], s);
      out[k][cc] = s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Lower triangle of K = Q + G' diag(W) G with 4x4 register tiles, summing
// only over the rows listed in rows[0 .. nrows) (rows with W = 0 add
// nothing and are left out).  Q is read from K's strict upper triangle
// (Q[i][j] = K[j][i] for j < i, never written here) and its diagonal from
// qd.  Tiles are split over the contraction when there are fewer tiles than
// threads; the partial sums are added in a fixed order (deterministic).
// ---------------------------------------------------------------------------
template <int NT>
__device__ void syrk_gwg(float* K, int ldk, const float* qd, const float* G, int ldg,
                         const float* W, const int* rows, int nrows, int n) {
  const int nt = (n + 3) >> 2;
  const int T = nt * (nt + 1) / 2;
  int ns = NT / T;
  if (ns < 1) ns = 1;
  if (ns > 4) ns = 4;
  const int chunk = (nrows + ns - 1) / ns;
  for (int item0 = 0; item0 < T * ns; item0 += NT) {
    const int item = item0 + (int)threadIdx.x;
    const bool active = item < T * ns;
    const int t = active ? item % T : 0;
    const int sp = active ? item / T : 0;
    const float x8 = 8.0f * (float)t + 1.0f;
    int I = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    if (active) {
      const int i0 = sp * chunk, i1 = min(nrows, i0 + chunk);
#pragma unroll 2
      for (int ii = i0; ii < i1; ++ii) {
        const int r = rows[ii];
        const float w = W[r];
        const float4 a = *reinterpret_cast<const float4*>(G + r * ldg + 4 * I);
        const float4 c = *reinterpret_cast<const float4*>(G + r * ldg + 4 * J);
        const float aw[4] = {a.x * w, a.y * w, a.z * w, a.w * w};
        const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[q][jj] = fmaf(aw[q], cv[jj], acc[q][jj]);
      }
    }
    for (int phase = 0; phase < ns; ++phase) {
      if (active && sp == phase) {
        // every base value is read before the first store (a store to K may
        // alias a later load from K, which would serialise the round trips)
        float base[4][4];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int i = 4 * I + ii, j = 4 * J + jj;
            base[ii][jj] = (i < n && j <= i)
                               ? (phase != 0 ? K[i * ldk + j] : (j == i ? qd[i] : K[j * ldk + i]))
                               : 0.f;
          }
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int i = 4 * I + ii, j = 4 * J + jj;
            if (i < n && j <= i) K[i * ldk + j] = base[ii][jj] + acc[ii][jj];
          }
      }
      __syncthreads();
    }
  }
}



// ---------------------------------------------------------------------------
// Blocked (panel width 8) right-looking Cholesky of a bordered system.
//
// Eliminates the n leading pivots of  [ K  F' ; F  C0 ]  a panel of 8 columns
// at a time:
//   (1) every thread that owns a row below the diagonal block -- K rows and
//       border (F) rows alike -- factors the 8x8 diagonal block itself, in
//       registers (rsqrtf pivots), and solves its row against it; threads
//       0..7 write the block's factor back (no serial one-warp phase);
//   (2) the panel rows, copied to Pb, update the trailing part of the
//       combined lower triangle with one register-tiled (4x4) product: K rows
//       subtract, F rows subtract, and the C block (if any) accumulates Y Y'.
// Outputs: K lower = L, Y = F L^-T, C (+)= Y Y', dinv = 1 / diag(L).
// Border rows may include right-hand sides: their rows become L^-1 r (as
// rows), and their C entries Y L^-1 r -- forward substitution for free.
// Pb holds panel rows in groups of 4 (8 values each) padded to 36 floats, so
// a warp's float4 loads of 4-row groups hit distinct banks; it needs
// pb_floats(n + nB + 4) floats (B rows start at a multiple of 4).  Two
// barriers per panel.
// ---------------------------------------------------------------------------
__host__ __device__ inline int pb_floats(int rows) { return ((rows + 3) / 4 + 1) * 36; }
__device__ __forceinline__ int pb_off(int r) { return (r >> 2) * 36 + (r & 3) * 8; }

template <int NT>
__device__ bool panel_factor_trsm(float* M, int ld, int j0, int jb, float* dinv, float* A,
                                  int lda, int rowA0, int nA, float* B, int ldb, int nB,
                                  float* Pb) {
  // Pb index of a row: A rows at 0 .. nA-1, B rows from the next multiple of
  // 4, so that every 4-row tile of the trailing update lies in one block.
  const int nA4 = (nA + 3) & ~3;
  const int N = nA + nB;
  bool ok = true;
  const int tid = threadIdx.x;
  float lmine[8];  // this thread's row of the block factor (threads 0..jb-1)
  float imine = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) lmine[j] = 0.f;
  for (int rr = tid; rr < (N > 8 ? N : 8); rr += NT) {
    // the diagonal block, padded to 8x8 with the identity
    float l[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j)
        l[i][j] = (i < jb && j < jb) ? M[(j0 + i) * ld + j0 + j] : (i == j ? 1.0f : 0.0f);
    float inv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float d = l[j][j];
      if (!(d > 0.0f) || !(d < INFINITY)) ok = false;
      inv[j] = rsqrtf(d);
      l[j][j] = d * inv[j];
#pragma unroll
      for (int i = j + 1; i < 8; ++i) l[i][j] *= inv[j];
#pragma unroll
      for (int i = j + 1; i < 8; ++i)
#pragma unroll
        for (int k = j + 1; k <= i; ++k) l[i][k] = fmaf(-l[i][j], l[k][j], l[i][k]);
    }
    if (rr < N) {
      const bool inA = rr < nA;
      float* row = inA ? A + (rowA0 + rr) * lda + j0 : B + (rr - nA) * ldb + j0;
      float v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = t < jb ? row[t] : 0.0f;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float acc = v[t];
#pragma unroll
        for (int u = 0; u < t; ++u) acc = fmaf(-v[u], l[t][u], acc);
        v[t] = acc * inv[t];
      }
      float* pr = Pb + pb_off(inA ? rr : nA4 + (rr - nA));
      reinterpret_cast<float4*>(pr)[0] = make_float4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<float4*>(pr)[1] = make_float4(v[4], v[5], v[6], v[7]);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < jb) row[t] = v[t];
    }
    if (rr == tid) {
      // keep row `tid` of the block factor (selected without dynamic indexing)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i == tid) {
#pragma unroll
          for (int j = 0; j < 8; ++j) lmine[j] = l[i][j];
          imine = inv[i];
        }
    }
  }
  // zero the pad rows: nA .. nA4-1 and after the last B row up to the group end
  for (int e = tid; e < 64; e += NT) {
    const int k = e >> 3, c = e & 7;
    const int r = k < 4 ? nA + k : nA4 + nB + (k - 4);
    const bool pad = k < 4 ? r < nA4 : (r & 3) != 0 && (r >> 2) == ((nA4 + nB) >> 2);
    if (pad) Pb[pb_off(r) + c] = 0.0f;
  }
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  // every thread has read the block: threads 0..jb-1 now store its factor
  // (nothing reads it before the next barrier)
  if (tid < jb) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j <= tid) M[(j0 + tid) * ld + j0 + j] = lmine[j];
    dinv[j0 + tid] = imine;
  }
  return all_ok;
}

// Trailing update with the panel in Pb over the combined row set
// [A rows rowA0 .. rowA0+nA-1 ; B rows 0 .. nB-1] (lower triangle):
//   (A, A): A[rowA0+r][rowA0+c] -= P_r . P_c
//   (B, A): B[k][rowA0+c]        -= P_k . P_c
//   (B, B): C[k][l]              += P_k . P_l     (when C != nullptr)
// B rows start at a multiple of 4 in Pb, so each 4x4 tile is in one block:
// one base pointer and stride per tile, predicated only at the edges.
template <int NT>
__device__ void panel_syrk(const float* Pb, float* A, int lda, int rowA0, int nA, float* B,
                           int ldb, int nB, float* C, int ldc) {
  const int nA4 = (nA + 3) & ~3;
  const int ntA = nA4 >> 2;
  const int nt = ntA + ((nB + 3) >> 2);
  const int T = nt * (nt + 1) / 2;
  for (int t = threadIdx.x; t < T; t += NT) {
    // tile index -> (I, J), J <= I (square root estimate, then exact correction)
    const float x8 = 8.0f * (float)t + 1.0f;
    int I = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;
    const bool rowA = I < ntA, colA = J < ntA;
    if (!rowA && !colA && C == nullptr) continue;
    float* dst;
    int ld, rmax, cmax;
    float sgn = -1.0f;
    if (rowA) {  // then colA too
      dst = A + (rowA0 + 4 * I) * lda + rowA0 + 4 * J;
      ld = lda;
      rmax = nA - 4 * I;
      cmax = nA - 4 * J;
    } else if (colA) {
      dst = B + (4 * I - nA4) * ldb + rowA0 + 4 * J;
      ld = ldb;
      rmax = nB - (4 * I - nA4);
      cmax = nA - 4 * J;
    } else {
      dst = C + (4 * I - nA4) * ldc + (4 * J - nA4);
      ld = ldc;
      rmax = nB - (4 * I - nA4);
      cmax = nB - (4 * J - nA4);
      sgn = 1.0f;
    }
    const bool diag = I == J;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    // not unrolled: the kernel's hot code already exceeds the instruction
    // cache (72 % hit rate measured); a smaller loop body is 2 % faster
#pragma unroll 1
    for (int h2 = 0; h2 < 2; ++h2) {
      float4 ra[4], cb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        ra[a] = reinterpret_cast<const float4*>(Pb + I * 36 + a * 8)[h2];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        cb[b] = reinterpret_cast<const float4*>(Pb + J * 36 + b * 8)[h2];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b] = fmaf(ra[a].x, cb[b].x, acc[a][b]);
          acc[a][b] = fmaf(ra[a].y, cb[b].y, acc[a][b]);
          acc[a][b] = fmaf(ra[a].z, cb[b].z, acc[a][b]);
          acc[a][b] = fmaf(ra[a].w, cb[b].w, acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (a < rmax && b < cmax && (!diag || b <= a))
          dst[a * ld + b] = fmaf(sgn, acc[a][b], dst[a * ld + b]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Wide panels (PW = 16 or 32).  Pbw holds panel rows in groups of 4 (PW
// values each) padded to 4 PW + 4 floats (conflict-free float4 loads across
// row groups); fb is a PW x PW scratch for the diagonal block's factor.  Per
// panel: warp 0 factors the diagonal block with shuffles (lane i holds row
// i) while, with PW = 32 (the large variant, matrices in global memory), the
// other warps copy the panel's rows into Pbw one row per warp (coalesced);
// barrier; every row below (and every border row) is solved against the
// block by one thread, in shared memory; barrier; the solved rows go back to
// global memory one row per warp, and the rank-PW trailing update follows
// (barrier) -- three barriers per PW columns, the block factor computed once
// instead of by every thread.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pbw_group(int pw) { return 4 * pw + 4; }
__host__ __device__ inline int pbw_floats(int rows, int pw) {
  return ((rows + 3) / 4 + 1) * pbw_group(pw);
}
// rows of Pbw that a factorisation of n pivots bordered by nB rows stores: the
// rows below the first diagonal block, rounded to a 4-row group, the border
// rows and the pad rows zeroed after them
__host__ __device__ inline int pbw_rows(int n, int nB, int pw) {
  return (n > pw ? n - pw : 0) + nB + 8;
}
template <int PW>
__device__ __forceinline__ int pbw_off(int r) {
  return (r >> 2) * pbw_group(PW) + (r & 3) * PW;
}

// Row stride of the diagonal block's factor fb (PW x fb_ld floats): padded so
// that one row per lane is stored without bank conflicts.  After fb: the
// 32 x 8 exchange buffer of factor_diag_block, then the factor's transpose
// below the diagonal (fbt: row k holds L[t][k] for t > k, zeros elsewhere;
// 16-byte aligned rows of fbt_ld floats) for the column-ordered panel solve.
__host__ __device__ constexpr int fb_ld(int pw) { return pw + 1; }
__host__ __device__ constexpr int fbt_ld(int pw) { return pw + 4; }
__host__ __device__ constexpr int fbt_off(int pw) { return pw * fb_ld(pw) + 32 * 8; }
__host__ __device__ constexpr int fb_floats(int pw) { return fbt_off(pw) + pw * fbt_ld(pw); }

// Cholesky of the jb x jb diagonal block at (j0, j0) of M by one warp, lane i
// holding row i, in PW / 8 sub-blocks of 8 columns: every lane factors the
// 8 x 8 diagonal sub-block itself, in registers (no communication within its
// 8 pivots), solves its own row against it, and takes the other rows' solved
// 8 values from shared memory (sbuf, 32 x 8 floats) for its trailing update.
// Four exchange rounds per 32 columns instead of a shuffle chain through
// every pivot.  Writes the factor to fb (stride fb_ld(PW)), to M and
// 1 / diag to dinv.  Returns 0 if a pivot is not positive and finite.
// Warp 0 only; sbuf must not be in use by other warps.
template <int PW>
__device__ __noinline__ int factor_diag_block(float* M, int ld, int j0, int jb, float* dinv,
                                             float* fb, float* sbuf,
                                             unsigned long long* ft = nullptr) {
  static_assert(PW % 8 == 0 && PW <= 32, "rows are lanes; 8-column sub-blocks");
  const int lane = threadIdx.x & 31;
  const long long tf0 = ft ? clock64() : 0;
  int okw = 1;
  float a[PW];
  {
    // the block, one row per warp instruction (coalesced, all loads in
    // flight), transposed through fb (padded rows: no bank conflicts) so
    // that lane i holds row i
    float col[PW];
#pragma unroll
    for (int r = 0; r < PW; ++r)
      col[r] = (r < jb && lane <= r) ? M[(j0 + r) * ld + j0 + lane] : 0.0f;
#pragma unroll
    for (int r = 0; r < PW; ++r) fb[r * fb_ld(PW) + lane] = col[r];
    __syncwarp();
#pragma unroll
    for (int c = 0; c < PW; ++c) a[c] = (lane < jb && c <= lane) ? fb[lane * fb_ld(PW) + c] : 0.0f;
    __syncwarp();
  }
  long long tf1 = 0;
  if (ft) {
    // tracing builds: the clock is read after every load has returned
    float sum = 0.0f;
#pragma unroll
    for (int c = 0; c < PW; ++c) sum += a[c];
    tf1 = clock64() + (long long)(sum * 0.0f);
  }
  float rinv = 0.0f;
#pragma unroll
  for (int b = 0; b < PW / 8; ++b) {
    const int c0 = 8 * b;
    if (c0 >= jb) break;
    // the sub-block's rows, raw, for every lane
    if (lane >= c0 && lane < c0 + 8) {
      float4* dst = reinterpret_cast<float4*>(sbuf + 8 * lane);
      dst[0] = make_float4(a[c0], a[c0 + 1], a[c0 + 2], a[c0 + 3]);
      dst[1] = make_float4(a[c0 + 4], a[c0 + 5], a[c0 + 6], a[c0 + 7]);
    }
    __syncwarp();
    // factor it in registers (rows beyond jb: identity)
    float l[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 u = reinterpret_cast<const float4*>(sbuf + 8 * (c0 + i))[0];
      const float4 v = reinterpret_cast<const float4*>(sbuf + 8 * (c0 + i))[1];
      const float row[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        l[i][j] = (c0 + i < jb) ? (j <= i ? row[j] : 0.0f) : (i == j ? 1.0f : 0.0f);
    }
    float inv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float d = l[j][j];
      if (!(d > 0.0f) || !(d < INFINITY)) okw = 0;
      inv[j] = rsqrtf(d);
      l[j][j] = d * inv[j];
#pragma unroll
      for (int i = j + 1; i < 8; ++i) l[i][j] *= inv[j];
#pragma unroll
      for (int i = j + 1; i < 8; ++i)
#pragma unroll
        for (int k = j + 1; k <= i; ++k) l[i][k] = fmaf(-l[i][j], l[k][j], l[i][k]);
    }
    // this lane's row in the sub-block's columns: its row of the factor, or
    // (rows below) the solve against it
    float v[8];
    if (lane < c0 + 8) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (lane == c0 + i) {
#pragma unroll
          for (int t = 0; t < 8; ++t) v[t] = l[i][t];
          rinv = inv[i];
        }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float acc = a[c0 + t];
#pragma unroll
        for (int u = 0; u < t; ++u) acc = fmaf(-v[u], l[t][u], acc);
        v[t] = acc * inv[t];
      }
    }
    if (lane >= c0) {
#pragma unroll
      for (int t = 0; t < 8; ++t) a[c0 + t] = v[t];
    }
    __syncwarp();  // every lane has read the raw sub-block
    if (lane >= c0) {
      float4* dst = reinterpret_cast<float4*>(sbuf + 8 * lane);
      dst[0] = make_float4(v[0], v[1], v[2], v[3]);
      dst[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    __syncwarp();
    // trailing columns of this lane's row: a[c] -= v_lane . v_c, c in
    // (c0 + 7, lane]
    if (lane >= c0 + 8) {
#pragma unroll
      for (int c = c0 + 8; c < PW; ++c) {
        if (c <= lane) {
          const float4 p = reinterpret_cast<const float4*>(sbuf + 8 * c)[0];
          const float4 q = reinterpret_cast<const float4*>(sbuf + 8 * c)[1];
          float acc = a[c];
          acc = fmaf(-v[0], p.x, acc); acc = fmaf(-v[1], p.y, acc);
          acc = fmaf(-v[2], p.z, acc); acc = fmaf(-v[3], p.w, acc);
          acc = fmaf(-v[4], q.x, acc); acc = fmaf(-v[5], q.y, acc);
          acc = fmaf(-v[6], q.z, acc); acc = fmaf(-v[7], q.w, acc);
          a[c] = acc;
        }
      }
    }
    __syncwarp();  // sbuf is rewritten by the next sub-block
  }
  const long long tf2 = ft ? clock64() : 0;
  if (lane < jb) {
#pragma unroll
    for (int c = 0; c < PW; ++c) fb[lane * fb_ld(PW) + c] = c <= lane ? a[c] : 0.0f;
    dinv[j0 + lane] = rinv;
  }
  {
    // the transpose below the diagonal: lane t writes column t of fbt
    float* const fbt = fb + fbt_off(PW);
#pragma unroll
    for (int c = 0; c < PW; ++c) fbt[c * fbt_ld(PW) + lane] = (c < lane && lane < jb) ? a[c] : 0.0f;
  }
  __syncwarp();
  // the block's factor back to M, one row per step of the warp (coalesced)
  for (int r = 0; r < jb; ++r)
    if (lane <= r) M[(j0 + r) * ld + j0 + lane] = fb[r * fb_ld(PW) + lane];
  if (ft && lane == 0) {
    atomicAdd(&ft[0], (unsigned long long)(tf1 - tf0));
    atomicAdd(&ft[1], (unsigned long long)(tf2 - tf1));
    atomicAdd(&ft[2], (unsigned long long)(clock64() - tf2));
  }
  return okw;
}

// diag_done: the diagonal block was factored ahead, during the previous
// panel's trailing update (look-ahead): fb, dinv and M already hold it.
template <int NT, int PW>
__device__ bool panel_factor_wide(float* M, int ld, int j0, int jb, float* dinv, float* A,
                                  int lda, int rowA0, int nA, float* B, int ldb, int nB,
                                  float* Pb, float* fb, unsigned long long* sub = nullptr,
                                  bool diag_done = false) {
  const long long tp0 = sub ? clock64() : 0;
  static_assert(PW != 32 || NT >= 64, "the staged panel needs warps beside warp 0");
  const int nA4 = (nA + 3) & ~3;
  const int N = nA + nB;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int okw = 1;
  if (tid < 32) {
    if (!diag_done) okw = factor_diag_block<PW>(M, ld, j0, jb, dinv, fb, fb + PW * fb_ld(PW));
    if (sub && tid == 0) atomicAdd(&sub[2], (unsigned long long)(clock64() - tp0));
  } else if (PW == 32) {
    // meanwhile the other warps stage the panel's rows in Pb, one row per
    // warp instruction and lane = column: coalesced 128-byte reads of global
    // memory (one row per thread would touch 32 rows per warp load); eight
    // rows' loads are in flight before their stores
    constexpr int kRows = 8;
    for (int r0 = (w - 1) * kRows; r0 < N; r0 += (NT / 32 - 1) * kRows) {
      float v[kRows];
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int rr = r0 + k;
        v[k] = 0.0f;
        if (rr < N && lane < jb)
          v[k] = rr < nA ? A[(rowA0 + rr) * lda + j0 + lane] : B[(rr - nA) * ldb + j0 + lane];
      }
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int rr = r0 + k;
        if (rr < N) Pb[pbw_off<PW>(rr < nA ? rr : nA4 + (rr - nA)) + lane] = v[k];
      }
    }
    if (sub && tid == 32) atomicAdd(&sub[3], (unsigned long long)(clock64() - tp0));
  }
  const bool all_ok = __syncthreads_and(okw) != 0;
  const long long tp1 = sub ? clock64() : 0;
  // one row per thread; within each warp's 32 rows, lane l takes row
  // 4 (l % 8) + l / 8, so that the 8 lanes of a shared-memory phase read rows
  // of 8 different 4-row groups of Pb (bank-conflict-free float4 accesses)
  long long tq1 = 0, tq2 = 0;  // tracing builds: thread 0's row solved / stored
  for (int r0 = w * 32; r0 < N; r0 += NT) {
    const int rr = r0 + ((lane & 7) << 2) + (lane >> 3);
    if (rr >= N) continue;
    const bool inA = rr < nA;
    float* row = inA ? A + (rowA0 + rr) * lda + j0 : B + (rr - nA) * ldb + j0;
    float4* pr = reinterpret_cast<float4*>(Pb + pbw_off<PW>(inA ? rr : nA4 + (rr - nA)));
    float v[PW];
    if (PW == 32) {
#pragma unroll
      for (int q = 0; q < PW / 4; ++q) {
        const float4 u = pr[q];
        v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < PW; ++t) v[t] = t < jb ? row[t] : 0.0f;
    }
    if (PW == 32) {
      // column order: step k finishes v[k] and takes its multiple off every
      // later entry, with column k of the factor read as 16-byte rows of fbt
      // (the same operations in the same order as the row-ordered solve)
      // the next step's column and pivot reciprocal are loaded while this
      // step computes, so the shared-memory round trips overlap the FMAs
      // instead of forming a chain of one per 16-byte word
      const float* const fbt = fb + fbt_off(PW);
      float4 lc[PW / 4];
      float dc = jb > 0 ? dinv[j0] : 0.0f;
#pragma unroll
      for (int g = 0; g < PW / 4; ++g) lc[g] = reinterpret_cast<const float4*>(fbt)[g];
#pragma unroll
      for (int k = 0; k < PW; ++k) {
        float4 ln[PW / 4];
        float dn = 0.0f;
        if (k + 1 < PW) {
          const float4* lt = reinterpret_cast<const float4*>(fbt + (k + 1) * fbt_ld(PW));
#pragma unroll
          for (int g = (k + 2) >> 2; g < PW / 4; ++g) ln[g] = lt[g];
          if (k + 1 < jb) dn = dinv[j0 + k + 1];
        }
        if (k < jb) {
          v[k] *= dc;
#pragma unroll
          for (int g = (k + 1) >> 2; g < PW / 4; ++g) {
            const float lv[4] = {lc[g].x, lc[g].y, lc[g].z, lc[g].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int t = 4 * g + q;
              if (t > k && t < jb) v[t] = fmaf(-v[k], lv[q], v[t]);
            }
          }
        }
        if (k + 1 < PW) {
#pragma unroll
          for (int g = (k + 2) >> 2; g < PW / 4; ++g) lc[g] = ln[g];
          dc = dn;
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < PW; ++t) {
        if (t < jb) {
          float acc = v[t];
#pragma unroll
          for (int u = 0; u < t; ++u) acc = fmaf(-v[u], fb[t * fb_ld(PW) + u], acc);
          v[t] = acc * dinv[j0 + t];
        }
      }
    }
    if (sub && tid == 0) {
      float sum = 0.0f;
#pragma unroll
      for (int q = 0; q < PW; ++q) sum += v[q];
      tq1 = clock64() + (long long)(sum * 0.0f);
    }
#pragma unroll
    for (int q = 0; q < PW / 4; ++q)
      pr[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    if (sub && tid == 0) tq2 = clock64();
    if (PW != 32) {
#pragma unroll
      for (int t = 0; t < PW; ++t)
        if (t < jb) row[t] = v[t];
    }
  }
  // zero the pad rows: nA .. nA4-1 and after the last B row up to its group's end
  for (int e = tid; e < 8 * PW; e += NT) {
    const int k = e / PW, c = e - k * PW;
    const int r = k < 4 ? nA + k : nA4 + nB + (k - 4);
    const bool pad = k < 4 ? r < nA4 : (r & 3) != 0 && (r >> 2) == ((nA4 + nB) >> 2);
    if (pad) Pb[pbw_off<PW>(r) + c] = 0.0f;
  }
  __syncthreads();
  if (sub && threadIdx.x == 0) {
    // tracing builds: (diagonal block || row staging), then the row solves;
    // within them thread 0's own row (solved, stored) and the wait for the
    // other rows
    const long long tq3 = clock64();
    atomicAdd(&sub[0], (unsigned long long)(tp1 - tp0));
    atomicAdd(&sub[1], (unsigned long long)(tq3 - tp1));
    if (tq1) {
      atomicAdd(&sub[8], (unsigned long long)(tq1 - tp1));
      atomicAdd(&sub[9], (unsigned long long)(tq2 - tq1));
      atomicAdd(&sub[10], (unsigned long long)(tq3 - tq2));
    }
  }
  if (PW == 32) {
    // write the solved rows back, one row per warp (coalesced); the trailing
    // update that follows reads Pb only and writes other columns, so no
    // barrier is needed before it
    for (int rr = w; rr < N; rr += NT / 32) {
      const bool inA = rr < nA;
      float* row = inA ? A + (rowA0 + rr) * lda + j0 : B + (rr - nA) * ldb + j0;
      if (lane < jb) row[lane] = Pb[pbw_off<PW>(inA ? rr : nA4 + (rr - nA)) + lane];
    }
  }
  return all_ok;
}

// Rank-PW trailing update with the panel in Pbw (same row sets and rules as
// panel_syrk).
// One 4 x 4 tile t (row-major lower-triangular numbering over the combined
// row set) of the rank-PW trailing update with the panel in Pbw.
template <int PW>
__device__ __forceinline__ void trailing_tile(int t, const float* Pb, float* A, int lda, int rowA0,
                                              int nA, float* B, int ldb, int nB, float* C,
                                              int ldc) {
  constexpr int GS = pbw_group(PW);
  const int nA4 = (nA + 3) & ~3;
  const int ntA = nA4 >> 2;
  const float x8 = 8.0f * (float)t + 1.0f;
  int I = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  const bool rowA = I < ntA, colA = J < ntA;
  if (!rowA && !colA && C == nullptr) return;
  float* dst;
  int ld, rmax, cmax;
  float sgn = -1.0f;
  if (rowA) {
    dst = A + (rowA0 + 4 * I) * lda + rowA0 + 4 * J;
    ld = lda;
    rmax = nA - 4 * I;
    cmax = nA - 4 * J;
  } else if (colA) {
    dst = B + (4 * I - nA4) * ldb + rowA0 + 4 * J;
    ld = ldb;
    rmax = nB - (4 * I - nA4);
    cmax = nA - 4 * J;
  } else {
    dst = C + (4 * I - nA4) * ldc + (4 * J - nA4);
    ld = ldc;
    rmax = nB - (4 * I - nA4);
    cmax = nB - (4 * J - nA4);
    sgn = 1.0f;
  }
  const bool diag = I == J;
  // whole off-diagonal tiles of 16-byte aligned rows move as float4 rows
  const bool vec = !diag && rmax >= 4 && cmax >= 4 && (ld & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  // the tile's current values, read before the product and before any
  // store: a store through dst may alias a later load of dst, so loads
  // interleaved with the stores would each wait for the one before (16
  // serial round trips per tile to L2)
  float old[4][4];
  if (vec) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float4 o4 = *reinterpret_cast<const float4*>(dst + a * ld);
      old[a][0] = o4.x; old[a][1] = o4.y; old[a][2] = o4.z; old[a][3] = o4.w;
    }
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        old[a][b] = (a < rmax && b < cmax && (!diag || b <= a)) ? dst[a * ld + b] : 0.f;
  }
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll
  for (int h = 0; h < PW / 4; ++h) {
    float4 ra[4], cb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ra[a] = reinterpret_cast<const float4*>(Pb + I * GS + a * PW)[h];
#pragma unroll
    for (int b = 0; b < 4; ++b) cb[b] = reinterpret_cast<const float4*>(Pb + J * GS + b * PW)[h];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        acc[a][b] = fmaf(ra[a].x, cb[b].x, acc[a][b]);
        acc[a][b] = fmaf(ra[a].y, cb[b].y, acc[a][b]);
        acc[a][b] = fmaf(ra[a].z, cb[b].z, acc[a][b]);
        acc[a][b] = fmaf(ra[a].w, cb[b].w, acc[a][b]);
      }
  }
  if (vec) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
      *reinterpret_cast<float4*>(dst + a * ld) =
          make_float4(fmaf(sgn, acc[a][0], old[a][0]), fmaf(sgn, acc[a][1], old[a][1]),
                      fmaf(sgn, acc[a][2], old[a][2]), fmaf(sgn, acc[a][3], old[a][3]));
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (a < rmax && b < cmax && (!diag || b <= a))
          dst[a * ld + b] = fmaf(sgn, acc[a][b], old[a][b]);
  }
}

// Rank-PW trailing update with the panel in Pbw (same row sets and rules as
// panel_syrk).  Look-ahead (jb2 > 0, PW = 32 only): the next panel's
// diagonal block -- the first jb2 rows and columns of the trailing matrix,
// tiles 0 .. T2-1 in this numbering -- is updated by warps 0-3, then warp 0
// factors it (factor_diag_block: into fb, dinv and M at pivot column
// rowA0) while the other warps update the remaining tiles; the next
// panel_factor_wide is then called with diag_done.  Needs NT >= 128 and
// uses named barrier 1.  Returns the
// factorisation's pivot check (1 without look-ahead).  Ends with a barrier.
template <int NT, int PW>
__device__ int panel_syrk_wide(const float* Pb, float* A, int lda, int rowA0, int nA, float* B,
                               int ldb, int nB, float* C, int ldc, int jb2 = 0,
                               float* dinv = nullptr, float* fb = nullptr,
                               unsigned long long* ft = nullptr) {
  static_assert(NT >= 128, "the look-ahead uses warps 0-3");
  const int nA4 = (nA + 3) & ~3;
  const int ntA = nA4 >> 2;
  const int nt = ntA + ((nB + 3) >> 2);
  const int T = nt * (nt + 1) / 2;
  int okw = 1;
  if (jb2 > 0) {
    const int nt2 = (jb2 + 3) >> 2;
    const int T2 = nt2 * (nt2 + 1) / 2;
    const long long tlt = ft ? clock64() : 0;
    if (threadIdx.x < 128) {
      // warps 0-3, one per scheduler: the block's tiles, then (named
      // barrier 1, these 128 threads only: the updated values visible to warp 0)
      for (int t = threadIdx.x; t < T2; t += 128)
        trailing_tile<PW>(t, Pb, A, lda, rowA0, nA, B, ldb, nB, C, ldc);
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    if (threadIdx.x < 32) {
      const long long tl0 = ft ? clock64() : 0;
      okw = factor_diag_block<PW>(A, lda, rowA0, jb2, dinv, fb, fb + PW * fb_ld(PW), ft);
      // tracing builds: the look-ahead's tile updates, before the factorisation
      if (ft && threadIdx.x == 0) atomicAdd(&ft[3], (unsigned long long)(tl0 - tlt));
    } else {
      for (int t = T2 + (int)threadIdx.x - 32; t < T; t += NT - 32)
        trailing_tile<PW>(t, Pb, A, lda, rowA0, nA, B, ldb, nB, C, ldc);
    }
  } else {
    for (int t = threadIdx.x; t < T; t += NT)
      trailing_tile<PW>(t, Pb, A, lda, rowA0, nA, B, ldb, nB, C, ldc);
  }
  return __syncthreads_and(okw);
}

// Eliminate the n pivots of K (n x n lower, stride ldk) bordered by nB rows
// in Y (stride ldy); C (nB x nB lower, stride ldc, may be null) accumulates
// Y Y'.  With C == nullptr this is a plain blocked Cholesky of K (nB = 0) or
// a Cholesky plus triangular solve of the border rows.
// sub (tracing builds only, may be null): cycles of the factor+TRSM stage and
// of the trailing updates are added to sub[0] and sub[1] by thread 0.
// PW: panel width, 8 (Pb of pb_floats rows) or 16 / 32 (Pb of pbw_floats
// rows followed by the diagonal block's factor, PW x fb_ld(PW) floats, and
// a 32 x 8 exchange buffer: fb_floats(PW)).
// Not inlined: the forward factors K_I and C with it, and one shared copy
// of the unrolled panel code keeps the hot loop within the instruction cache
// (two inlined copies made the forward 11 % slower).
template <int NT, int PW = 8>
__device__ __noinline__ bool blocked_cholesky_bordered(float* K, int ldk, int n, float* Y, int ldy, int nB,
                                          float* C, int ldc, float* dinv, float* Pb,
                                          unsigned long long* sub = nullptr,
                                          unsigned long long* psub = nullptr) {
  bool ok = true;
  float* const fb = PW > 8 ? Pb + pbw_floats(pbw_rows(n, nB, PW), PW) : nullptr;
  bool ahead = false;  // this panel's diagonal block was factored ahead
  for (int j0 = 0; j0 < n; j0 += PW) {
    const int jb = min(PW, n - j0);
    const int nK = n - j0 - jb;
    const long long c0 = sub ? clock64() : 0;
    if constexpr (PW > 8)
      ok = panel_factor_wide<NT, PW>(K, ldk, j0, jb, dinv, K, ldk, j0 + jb, nK, Y, ldy, nB, Pb,
                                     fb, psub, ahead) &&
           ok;
    else
      ok = panel_factor_trsm<NT>(K, ldk, j0, jb, dinv, K, ldk, j0 + jb, nK, Y, ldy, nB, Pb) &&
           ok;
    const long long c1 = sub ? clock64() : 0;
    ahead = false;
    if (nK + nB > 0) {
      if constexpr (PW == 32) {
        // look-ahead: warp 0 updates and factors the next diagonal block
        // while the other warps finish the trailing update
        const int jb2 = min(PW, nK);
        ok = panel_syrk_wide<NT, PW>(Pb, K, ldk, j0 + jb, nK, Y, ldy, nB, C, ldc, jb2, dinv, fb,
                                     psub ? psub + 4 : nullptr) &&
             ok;
        ahead = jb2 > 0;
      } else if constexpr (PW > 8) {
        panel_syrk_wide<NT, PW>(Pb, K, ldk, j0 + jb, nK, Y, ldy, nB, C, ldc);
      } else {
        panel_syrk<NT>(Pb, K, ldk, j0 + jb, nK, Y, ldy, nB, C, ldc);
      }
    }
    if (sub && threadIdx.x == 0) {
      const long long c2 = clock64();
      atomicAdd(&sub[0], (unsigned long long)(c1 - c0));
      atomicAdd(&sub[1], (unsigned long long)(c2 - c1));
    }
  }
  __syncthreads();  // the last diagonal block is written after the panel's barrier
  return ok;
}

// ---------------------------------------------------------------------------
// Warp-level triangular solves for R right-hand sides held in registers
// (lane owns rows lane + 32 s, s < S).  L stride ldk (odd => conflict-free).
// ---------------------------------------------------------------------------
template <int S, int R>
__device__ __forceinline__ void warp_lower_solve(const float* L, int ldk, const float* dinv, int n,
                                                 float (&x)[R][S]) {
  const int lane = threadIdx.x & 31;
  // column j of L for this lane's rows, loaded one step ahead (the loads do
  // not depend on the solve, so their latency overlaps the previous step)
  float lc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    lc[s] = (i > 0 && i < n) ? L[i * ldk] : 0.f;
  }
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    const int jend = min(32, n - 32 * sl);
    for (int jj = 0; jj < jend; ++jj) {
      const int j = 32 * sl + jj;
      float cur[S];
#pragma unroll
      for (int s = 0; s < S; ++s) cur[s] = lc[s];
      if (j + 1 < n) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int i = lane + 32 * s;
          lc[s] = (i > j + 1 && i < n) ? L[i * ldk + j + 1] : 0.f;
        }
      }
      const float dj = dinv[j];
      float xj[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        xj[r] = __shfl_sync(kFull, x[r][sl] * dj, jj);
        if (lane == jj) x[r][sl] = xj[r];
      }
#pragma unroll
      for (int s = sl; s < S; ++s) {
        const int i = lane + 32 * s;
        if (i > j && i < n) {
#pragma unroll
          for (int r = 0; r < R; ++r) x[r][s] = fmaf(-cur[s], xj[r], x[r][s]);
        }
      }
    }
  }
}

// Solve L' x = b (back substitution using rows of L).
template <int S, int R>
__device__ __forceinline__ void warp_upper_solve(const float* L, int ldk, const float* dinv, int n,
                                                 float (&x)[R][S]) {
  const int lane = threadIdx.x & 31;
  // row j of L for this lane's columns, loaded one step ahead
  float lr[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    lr[s] = (n > 0 && i < n - 1) ? L[(n - 1) * ldk + i] : 0.f;
  }
#pragma unroll
  for (int sl = S - 1; sl >= 0; --sl) {
    const int jend = min(32, n - 32 * sl);
    for (int jj = jend - 1; jj >= 0; --jj) {
      const int j = 32 * sl + jj;
      float cur[S];
#pragma unroll
      for (int s = 0; s < S; ++s) cur[s] = lr[s];
      if (j >= 1) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int i = lane + 32 * s;
          lr[s] = (i < j - 1) ? L[(j - 1) * ldk + i] : 0.f;
        }
      }
      const float dj = dinv[j];
      float xj[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        xj[r] = __shfl_sync(kFull, x[r][sl] * dj, jj);
        if (lane == jj) x[r][sl] = xj[r];
      }
#pragma unroll
      for (int s = 0; s <= sl; ++s) {
        const int i = lane + 32 * s;
        if (i < j) {
#pragma unroll
          for (int r = 0; r < R; ++r) x[r][s] = fmaf(-cur[s], xj[r], x[r][s]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Blocked triangular solves for factors in global memory (large variant):
// x_v <- L^-1 x_v (lower) or L^-T x_v (upper) for one or two vectors x0, x1
// (x1 may be null) of length n in shared memory; L lower, stride ld;
// dinv = 1 / diag(L).  32 indices per block: warp 0 holds the block's 32x32
// diagonal part in registers and solves it with shuffles; threads 32 .. NT-1
// then apply the block to the remaining entries, one row each (32
// independent loads).  The loads never wait on the solve: the rows' entries
// of a block are loaded before the barrier, while warp 0 solves its
// diagonal part, and warp 0 loads the next diagonal part while the others
// apply the current block.  Two barriers per block.
// ---------------------------------------------------------------------------
template <int NT, bool kUpper, class Bar = CtaBar>
__device__ __noinline__ void block_trsv(const float* L, int ld, const float* dinv, int n,
                                        float* x0, float* x1) {
  static_assert(NT >= 64, "warp 0 solves, the other warps apply");
  constexpr int NR = NT - 32;
  const int t = threadIdx.x, lane = t & 31;
  const int nblk = (n + 31) >> 5;
  // r: in warp 0 the block's diagonal part -- lower: lane l holds row l,
  // r[k] = L[j0+l][j0+k] (k <= l); upper: lane l holds column l,
  // r[k] = L[j0+k][j0+l] (k >= l) --, in the other threads the entries of
  // the row they apply the block to
  float r[32];
  auto load_diag = [&](int bk) {
    const int j0 = 32 * (kUpper ? nblk - 1 - bk : bk);
    const int jb = min(32, n - j0);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const bool in = lane < jb && k < jb && (kUpper ? k >= lane : k <= lane);
      r[k] = in ? (kUpper ? L[(j0 + k) * ld + j0 + lane] : L[(j0 + lane) * ld + j0 + k]) : 0.f;
    }
  };
  auto load_row = [&](int i, int j0, int jb) {
#pragma unroll
    for (int k = 0; k < 32; ++k)
      r[k] = k < jb ? (kUpper ? L[(j0 + k) * ld + i] : L[i * ld + j0 + k]) : 0.f;
  };
  if (t < 32 && nblk > 0) load_diag(0);
  for (int bk = 0; bk < nblk; ++bk) {
    const int j0 = 32 * (kUpper ? nblk - 1 - bk : bk);
    const int jb = min(32, n - j0);
    // the rest: lower -> entries i >= j0 + jb, upper -> entries i < j0
    const int r0 = kUpper ? 0 : j0 + jb, r1 = kUpper ? j0 : n;
    const int i0 = r0 + t - 32;
    if (t < 32) {
      float v0 = lane < jb ? x0[j0 + lane] : 0.f;
      float v1 = (x1 && lane < jb) ? x1[j0 + lane] : 0.f;
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) {
        const int k = kUpper ? 31 - kk : kk;
        if (k < jb) {
          const float dk = dinv[j0 + k];
          const float s0 = __shfl_sync(kFull, v0 * dk, k);
          const float s1 = __shfl_sync(kFull, v1 * dk, k);
          if (lane == k) { v0 = s0; v1 = s1; }
          if (kUpper ? lane < k : lane > k) {
            v0 = fmaf(-r[k], s0, v0);
            v1 = fmaf(-r[k], s1, v1);
          }
        }
      }
      if (lane < jb) {
        x0[j0 + lane] = v0;
        if (x1) x1[j0 + lane] = v1;
      }
      if (bk + 1 < nblk) load_diag(bk + 1);
    } else if (i0 < r1) {
      load_row(i0, j0, jb);
    }
    Bar::sync();
    if (t >= 32) {
      for (int i = i0; i < r1; i += NR) {
        if (i != i0) load_row(i, j0, jb);
        float acc0 = x0[i], acc1 = x1 ? x1[i] : 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (k < jb) {
            acc0 = fmaf(-r[k], x0[j0 + k], acc0);
            if (x1) acc1 = fmaf(-r[k], x1[j0 + k], acc1);
          }
        }
        x0[i] = acc0;
        if (x1) x1[i] = acc1;
      }
    }
    Bar::sync();
  }
}

// Solve rows of X in place (stride ldx): forward (lower) or backward (upper).
// Rows are dealt to warps; each warp solves two rows at a time.
template <int NT, int S, bool kUpper>
__device__ void solve_rows_S(const float* L, int ldk, const float* dinv, int n, float* X, int ldx,
                             int row0, int nrows) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nw = NT / 32;
  for (int base = 2 * w; base < nrows; base += 2 * nw) {
    const int ra = row0 + base;
    const bool two = base + 1 < nrows;
    const int rb = two ? ra + 1 : ra;
    float x[2][S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int i = lane + 32 * s;
      x[0][s] = i < n ? X[ra * ldx + i] : 0.f;
      x[1][s] = i < n ? X[rb * ldx + i] : 0.f;
    }
    if (kUpper)
      warp_upper_solve<S, 2>(L, ldk, dinv, n, x);
    else
      warp_lower_solve<S, 2>(L, ldk, dinv, n, x);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int i = lane + 32 * s;
      if (i < n) {
        X[ra * ldx + i] = x[0][s];
        if (two) X[rb * ldx + i] = x[1][s];
      }
    }
  }
}

// kMaxS: 4 (n <= 128) or 8 (n <= 256; only the large-problem variant
// instantiates the longer register arrays).  Bar: the barrier it ends with.
template <int NT, bool kUpper, int kMaxS = 4, class Bar = CtaBar>
__device__ void solve_rows(const float* L, int ldk, const float* dinv, int n, float* X, int ldx,
                           int row0, int nrows) {
  if (n <= 32)
    solve_rows_S<NT, 1, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
  else if (n <= 64)
    solve_rows_S<NT, 2, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
  else if (n <= 96)
    solve_rows_S<NT, 3, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
  else if (kMaxS <= 4 || n <= 128)
    solve_rows_S<NT, 4, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
  else if constexpr (kMaxS > 4) {
    if (n <= 160)
      solve_rows_S<NT, 5, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
    else if (n <= 192)
      solve_rows_S<NT, 6, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
    else if (n <= 224)
      solve_rows_S<NT, 7, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
    else
      solve_rows_S<NT, 8, kUpper>(L, ldk, dinv, n, X, ldx, row0, nrows);
  }
  Bar::sync();
}

}  // namespace qpgpu
