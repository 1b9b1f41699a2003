// qp_backward.cu -- implicit-function-theorem backward pass (Alg. 3).
//
// At the relaxed point the forward kernel cached the two-level factors of the
// Newton matrix (eq. 14 with the inactive dv eliminated):
//   K_I = Q + G_I' W_I G_I = L L',   Y = F L^-T with F = [G_A; A],
//   C = D + Y Y' = L_C L_C',         D = diag(1/W_A, 0),
// with W, the row -> position map and the relaxed (x, y, z).  eq. 14 is
// symmetric, so the adjoint solve of the implicit function theorem (App. A)
// is the same solve with right-hand side (-g, 0, 0), g = dl/dx:
//   u = L^-1 (-g),  C mu = Y u,  dx = L^-T (u - Y' mu),  mu = (lambda, dy),
//   dz_A = lambda (= W_A G_A dx),  dz_I = W_I (G_I dx)
// (dz = B_k(v) dv is eq. 13's fourth row with zero residuals).  Then, as
// printed in Alg. 3,
//   dQ = (dx x' + x dx')/2, dq = dx, dA = dy x' + y dx', db = -dy,
//   dG = dz x' + z dx',     dh = -dz.
// One CTA per instance.  The solves are short; the kernel's time is the
// streaming read of G and the cache and the write of the gradient blocks, so
// all outputs go out as coalesced 16-byte streaming stores where aligned.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qpgpu {

namespace {

struct BLayout {
  int ldk, ldc, ldx, nv, mv, pv, fv;
  int oK, oY, oC, oR, o_dinv, o_cdinv, o_mu, o_x, o_y, o_z, o_W, o_pos, o_dz, total;
};

__host__ __device__ inline BLayout make_blayout(int n, int m, int p, int amax) {
  BLayout B;
  const int f = amax + p;
  B.ldk = ld_odd(n);
  B.ldc = ld_odd(f > 0 ? f : 1);
  B.ldx = round4(n);
  B.nv = round4(n); B.mv = round4(m > 0 ? m : 1); B.pv = round4(p > 0 ? p : 1);
  B.fv = round4(f > 0 ? f : 1);
  int o = 0;
  auto take = [&](int c) -> int { int r = o; o += round4(c); return r; };
  B.oK = take(n * B.ldk);
  B.oY = take(f * B.ldk);
  B.oC = take(f * B.ldc);
  B.oR = take(B.ldx);
  B.o_dinv = take(B.nv); B.o_cdinv = take(B.fv); B.o_mu = take(B.fv);
  B.o_x = take(B.nv); B.o_y = take(B.pv); B.o_z = take(B.mv); B.o_W = take(B.mv);
  B.o_pos = take(B.mv); B.o_dz = take(B.mv);
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

template <int NT>
__global__ void __launch_bounds__(NT) qp_backward_kernel(const BwdParams P) {
  extern __shared__ __align__(16) float sm[];
  const int n = P.n, m = P.m, p = P.p, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int bi = blockIdx.x;
  const BLayout B = make_blayout(n, m, p, P.amax);
  const CacheLayout cl = cache_layout(n, m, p, P.amax);
  const float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
  float* K = sm + B.oK;
  float* Y = sm + B.oY;
  float* C = sm + B.oC;
  float* R = sm + B.oR;
  float* dinv = sm + B.o_dinv;
  float* cdinv = sm + B.o_cdinv;
  float* mu = sm + B.o_mu;
  float* xs = sm + B.o_x;
  float* ys = sm + B.o_y;
  float* zs = sm + B.o_z;
  float* Ws = sm + B.o_W;
  int* pos = reinterpret_cast<int*>(sm + B.o_pos);
  float* dz = sm + B.o_dz;
  const int a = reinterpret_cast<const int*>(c + cl.oHdr)[0];
  const int nf = reinterpret_cast<const int*>(c + cl.oHdr)[1];
  // a cache that was not written by a forward solve of this size cannot index
  // out of bounds: its gradients come out NaN instead
  const bool valid = a >= 0 && a <= P.amax && nf == a + p;
  // ---- load the cached factors and point ----
  for (int i = t; i < B.total; i += NT) sm[i] = 0.0f;
  __syncthreads();
  const int nl = n * (n + 1) / 2;
  for (int e = t; e < nl; e += NT) {
    const int i = tri_row(e), j = e - i * (i + 1) / 2;
    const float v = __ldg(c + cl.oL + e);
    K[i * B.ldk + j] = v;
    if (i == j) dinv[i] = 1.0f / v;
  }
  const int nfl = valid ? nf : 0;
  for (int e = t; e < nfl * n; e += NT) {
    const int k = e / n, i = e - k * n;
    Y[k * B.ldk + i] = __ldg(c + cl.oY + e);
  }
  const int fl = nfl * (nfl + 1) / 2;
  for (int e = t; e < fl; e += NT) {
    const int i = tri_row(e), j = e - i * (i + 1) / 2;
    const float v = __ldg(c + cl.oLC + e);
    C[i * B.ldc + j] = v;
    if (i == j) cdinv[i] = 1.0f / v;
  }
  for (int i = t; i < n; i += NT) {
    xs[i] = __ldg(c + cl.ox + i);
    R[i] = -__ldg(P.g + (size_t)bi * n + i);
  }
  for (int k = t; k < p; k += NT) ys[k] = __ldg(c + cl.oy + k);
  int bad = valid ? 0 : 1;
  for (int r = t; r < m; r += NT) {
    zs[r] = __ldg(c + cl.oz + r);
    Ws[r] = __ldg(c + cl.oW + r);
    int k = __ldg(reinterpret_cast<const int*>(c + cl.oPos) + r);
    if (k >= a || k < -1) { k = -1; bad = 1; }
    pos[r] = k;
  }
  if (__syncthreads_or(bad)) {
    const float nanv = NAN;
    if (P.dQ) for (int e = t; e < n * n; e += NT) P.dQ[(size_t)bi * n * n + e] = nanv;
    if (P.dq) for (int e = t; e < n; e += NT) P.dq[(size_t)bi * n + e] = nanv;
    if (P.dA) for (int e = t; e < p * n; e += NT) P.dA[(size_t)bi * p * n + e] = nanv;
    if (P.db) for (int e = t; e < p; e += NT) P.db[(size_t)bi * p + e] = nanv;
    if (P.dG) for (int e = t; e < m * n; e += NT) P.dG[(size_t)bi * m * n + e] = nanv;
    if (P.dh) for (int e = t; e < m; e += NT) P.dh[(size_t)bi * m + e] = nanv;
    return;
  }
  // ---- adjoint solve ----
  solve_rows<NT, false>(K, B.ldk, dinv, n, R, B.ldx, 0, 1);
  if (nf > 0) {
    for (int k = t; k < nf; k += NT) {
      float acc = 0.f;
      for (int i = 0; i < n; ++i) acc = fmaf(Y[k * B.ldk + i], R[i], acc);
      mu[k] = acc;
    }
    __syncthreads();
    if (w == 0) {
      if (nf <= 32) small_chol_solve<1>(C, B.ldc, cdinv, nf, mu);
      else if (nf <= 64) small_chol_solve<2>(C, B.ldc, cdinv, nf, mu);
      else if (nf <= 96) small_chol_solve<3>(C, B.ldc, cdinv, nf, mu);
      else small_chol_solve<4>(C, B.ldc, cdinv, nf, mu);
    }
    __syncthreads();
    for (int i = t; i < n; i += NT) {
      float acc = R[i];
      for (int k = 0; k < nf; ++k) acc = fmaf(-Y[k * B.ldk + i], mu[k], acc);
      R[i] = acc;
    }
    __syncthreads();
  }
  solve_rows<NT, true>(K, B.ldk, dinv, n, R, B.ldx, 0, 1);
  const float* dx = R;
  const float* dy = mu + a;
  // ---- dz: active rows from the multipliers, inactive rows W (G dx) ----
  const float* gG = P.G + (size_t)bi * m * n;
  for (int r = w; r < m; r += NT / 32) {
    const int k = pos[r];
    if (k >= 0) {
      if (lane == 0) dz[r] = mu[k];
      continue;
    }
    float acc = 0.f;
    for (int j = lane; j < n; j += 32) acc = fmaf(__ldg(gG + (size_t)r * n + j), dx[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) dz[r] = Ws[r] * acc;
  }
  __syncthreads();
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

size_t backward_smem_bytes(int n, int m, int p, int amax, int* nthreads) {
  if (nthreads) *nthreads = 256;
  if (n > 128 || amax + p > 128) return 0;
  BLayout B = make_blayout(n, m, p, amax);
  size_t bytes = (size_t)B.total * sizeof(float);
  return bytes > 227 * 1024 ? 0 : bytes;
}

cudaError_t launch_backward(const BwdParams& P, int nthreads, size_t smem, cudaStream_t st) {
  if (nthreads != 256) return cudaErrorInvalidValue;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(qp_backward_kernel<256>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  qp_backward_kernel<256><<<P.batch, 256, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace qpgpu
