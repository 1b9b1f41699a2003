// qp_backward.cu -- implicit-function-theorem backward pass (Alg. 3).
//
// At the relaxed point the forward kernel cached L (K = Q + G'WG = L L'),
// U' = L^-1 A', L_S (U'U = L_S L_S'), W and the relaxed (x, y, z).  For an
// upstream gradient g = dl/dx the adjoint of the Newton system (eq. 14 is
// symmetric, so the transpose solve is the same solve) is
//     K dx + A'dy = -g,   A dx = 0,   dz = W .* (G dx)
// (dz = B_k(v) dv is eq. 13's fourth row with zero residuals; with dv
// eliminated it equals W G dx).  Then, as printed in Alg. 3,
//     dQ = (dx x' + x dx')/2, dq = dx, dA = dy x' + y dx', db = -dy,
//     dG = dz x' + z dx',     dh = -dz.
// One CTA per instance.  The solves are short; the kernel's time is the
// streaming read of G and the cache and the write of the gradient blocks,
// so all outputs go out as coalesced 16-byte streaming stores where aligned.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qpgpu {

namespace {

struct BLayout {
  int ldk, ldx, lds, nv, mv, pv;
  int oK, oX, oS, o_dinv, o_sdinv, o_x, o_y, o_z, o_W, o_dz, o_dy, total;
};

__host__ __device__ inline BLayout make_blayout(int n, int m, int p) {
  BLayout B;
  B.ldk = ld_odd(n);
  B.ldx = round4(n);
  B.lds = ld_odd(p > 0 ? p : 1);
  B.nv = round4(n); B.mv = round4(m > 0 ? m : 1); B.pv = round4(p > 0 ? p : 1);
  int o = 0;
  auto take = [&](int c) { int r = o; o += round4(c); return r; };
  B.oK = take(n * B.ldk);
  B.oX = take((p + 1) * B.ldx);
  B.oS = take(p * B.lds);
  B.o_dinv = take(B.nv); B.o_sdinv = take(B.pv);
  B.o_x = take(B.nv); B.o_y = take(B.pv); B.o_z = take(B.mv); B.o_W = take(B.mv);
  B.o_dz = take(B.mv); B.o_dy = take(B.pv);
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

template <int NT>
__global__ void __launch_bounds__(NT) qp_backward_kernel(const BwdParams P) {
  extern __shared__ __align__(16) float sm[];
  const int n = P.n, m = P.m, p = P.p, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int bi = blockIdx.x;
  const BLayout B = make_blayout(n, m, p);
  const CacheLayout cl = cache_layout(n, m, p);
  const float* c = P.cache + (size_t)bi * (size_t)P.cache_stride;
  float* K = sm + B.oK;
  float* X = sm + B.oX;
  float* S = sm + B.oS;
  float* dinv = sm + B.o_dinv;
  float* sdinv = sm + B.o_sdinv;
  float* xs = sm + B.o_x;
  float* ys = sm + B.o_y;
  float* zs = sm + B.o_z;
  float* Ws = sm + B.o_W;
  float* dz = sm + B.o_dz;
  float* dy = sm + B.o_dy;
  // ---- load the cached factor and point ----
  for (int i = t; i < B.total; i += NT) sm[i] = 0.0f;
  __syncthreads();
  const int nl = n * (n + 1) / 2;
  for (int e = t; e < nl; e += NT) {
    const int i = tri_row(e), j = e - i * (i + 1) / 2;
    const float v = __ldg(c + cl.oL + e);
    K[i * B.ldk + j] = v;
    if (i == j) dinv[i] = 1.0f / v;
  }
  for (int e = t; e < p * n; e += NT) {
    const int k = e / n, i = e - k * n;
    X[k * B.ldx + i] = __ldg(c + cl.oU + e);
  }
  const int pl = p * (p + 1) / 2;
  for (int e = t; e < pl; e += NT) {
    const int i = tri_row(e), j = e - i * (i + 1) / 2;
    const float v = __ldg(c + cl.oLs + e);
    S[i * B.lds + j] = v;
    if (i == j) sdinv[i] = 1.0f / v;
  }
  for (int i = t; i < n; i += NT) {
    xs[i] = __ldg(c + cl.ox + i);
    X[p * B.ldx + i] = -__ldg(P.g + (size_t)bi * n + i);
  }
  for (int k = t; k < p; k += NT) ys[k] = __ldg(c + cl.oy + k);
  for (int r = t; r < m; r += NT) {
    zs[r] = __ldg(c + cl.oz + r);
    Ws[r] = __ldg(c + cl.oW + r);
  }
  __syncthreads();
  // ---- adjoint solve: u = L^-1(-g); S dy = U'u; dx = L^-T (u - U dy) ----
  solve_rows<NT, false>(K, B.ldk, dinv, n, X, B.ldx, p, 1);
  if (p > 0) {
    for (int a = t; a < p; a += NT) {
      float acc = 0.f;
      for (int i = 0; i < n; ++i) acc = fmaf(X[a * B.ldx + i], X[p * B.ldx + i], acc);
      dy[a] = acc;
    }
    __syncthreads();
    if (w == 0) {
      // p is at most 128 here (checked on the host)
      float r[1][4];
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) {
        const int i = lane + 32 * s2;
        r[0][s2] = i < p ? dy[i] : 0.f;
      }
      if (p <= 32) {
        float r1[1][1] = {{r[0][0]}};
        warp_lower_solve<1, 1>(S, B.lds, sdinv, p, r1);
        warp_upper_solve<1, 1>(S, B.lds, sdinv, p, r1);
        r[0][0] = r1[0][0];
      } else {
        warp_lower_solve<4, 1>(S, B.lds, sdinv, p, r);
        warp_upper_solve<4, 1>(S, B.lds, sdinv, p, r);
      }
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) {
        const int i = lane + 32 * s2;
        if (i < p) dy[i] = r[0][s2];
      }
    }
    __syncthreads();
    for (int i = t; i < n; i += NT) {
      float acc = X[p * B.ldx + i];
      for (int a = 0; a < p; ++a) acc = fmaf(-X[a * B.ldx + i], dy[a], acc);
      X[p * B.ldx + i] = acc;
    }
    __syncthreads();
  }
  solve_rows<NT, true>(K, B.ldk, dinv, n, X, B.ldx, p, 1);
  const float* dx = X + p * B.ldx;
  // ---- dz = W .* (G dx): one warp per row of G, coalesced reads ----
  const float* gG = P.G + (size_t)bi * m * n;
  for (int r = w; r < m; r += NT / 32) {
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

size_t backward_smem_bytes(int n, int m, int p, int* nthreads) {
  if (nthreads) *nthreads = 256;
  if (n > 128 || p > 128) return 0;
  BLayout B = make_blayout(n, m, p);
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
