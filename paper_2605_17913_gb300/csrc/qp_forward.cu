// qp_forward.cu -- host-side sizing and dispatch of the forward kernel.
#include "qp_forward.cuh"

namespace qpgpu {

template <int NT, bool kBig>
cudaError_t launch_forward_nt(const FwdParams& P, size_t smem, int grid, cudaStream_t st);
template <int NT, bool kBig>
int forward_blocks_per_sm_nt(size_t smem);

// Threads per CTA and the active-row cap amax by size.  amax = rows kept as
// multipliers: min(m, n) where possible (at a non-degenerate solution at most
// n - p rows are active, at a degenerate one up to n); rows beyond it with
// W > 1 would have to go to K_I (tau grows), which FP32 may not factor.  On
// chip (n <= 128, everything in shared memory): 128 threads up to n = 72
// (fewer warps per barrier, no register cap; 5 % faster than 256 threads at
// n = 50), else 512; amax lowered to fit shared memory but not below
// min(m, n - p), and amax + p <= 126 (warp solves hold at most 128 rows, two
// of them folded right-hand sides); onchip512 asks for 512 threads at every
// n <= 128 (one kernel for every size, as a persistent server runs it).
// Otherwise the large variant (n <= 256):
// 512 threads, K, G, A, Y, C in a global workspace, amax + p <= 318.
size_t forward_config(int n, int m, int p, int* nthreads, int* amax_out, long long* ws_floats,
                      bool warp_per_qp, int large_threads, bool onchip512) {
  if (nthreads) *nthreads = 0;
  if (amax_out) *amax_out = 0;
  if (ws_floats) *ws_floats = 0;
  if (n < 1 || n > 256 || p > n || p < 0 || m < 0) return 0;
  const size_t budget = 227 * 1024 - fwd::kStaticSmem;
  if (n <= 128) {
    const int nt = n <= 72 ? 128 : 512;
    int amax0 = m < n ? m : n;
    if (amax0 + p > 126) amax0 = 126 - p;
    int floor_a = m < n - p ? m : n - p;
    if (floor_a < 0) floor_a = 0;
    for (int amax = amax0; amax >= floor_a && amax >= 0; --amax) {
      const fwd::FLayout L = fwd::make_fwd_layout(n, m, p, amax, nt);
      size_t bytes = (size_t)L.total * sizeof(float);
      if (bytes <= budget) {
        int nt_used = nt;
        // one warp per QP: the same amax (its layout is no larger), so the
        // gradient cache and every size query are unchanged
        if (warp_per_qp && n <= 32) {
          nt_used = 32;
          bytes = (size_t)fwd::make_fwd_layout(n, m, p, amax, 32).total * sizeof(float);
        } else if (onchip512 && nt_used != 512) {
          // 512 threads at the same amax (the cache layout is unchanged), if
          // its layout fits
          bytes = (size_t)fwd::make_fwd_layout(n, m, p, amax, 512).total * sizeof(float);
          if (bytes > budget) return 0;
          nt_used = 512;
        }
        if (nthreads) *nthreads = nt_used;
        if (amax_out) *amax_out = amax;
        return bytes;
      }
    }
  }
  int amax = m < n ? m : n;
  if (amax + p > 318) amax = 318 - p;
  if (amax < 0) return 0;
  const int nt = large_threads == 256 ? 256 : 512;
  const fwd::FLayout L = fwd::make_fwd_layout(n, m, p, amax, nt, true);
  const size_t bytes = (size_t)L.total * sizeof(float);
  if (bytes > budget) return 0;
  if (nthreads) *nthreads = nt;
  if (amax_out) *amax_out = amax;
  if (ws_floats) *ws_floats = round4(L.big_total);
  return bytes;
}

cudaError_t launch_forward(const FwdParams& P, int nthreads, size_t smem, int grid,
                           cudaStream_t st) {
  if (P.ws) return nthreads == 512   ? launch_forward_nt<512, true>(P, smem, grid, st)
                  : nthreads == 256 ? launch_forward_nt<256, true>(P, smem, grid, st)
                                    : cudaErrorInvalidValue;
  switch (nthreads) {
    case 32: return launch_forward_nt<32, false>(P, smem, grid, st);
    case 128: return launch_forward_nt<128, false>(P, smem, grid, st);
    case 512: return launch_forward_nt<512, false>(P, smem, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

// Load every variant's module now (the runtime loads kernels lazily, on
// first use), so that no later launch pays for it.
void preload_forward_kernels() {
  forward_blocks_per_sm_nt<32, false>(1024);
  forward_blocks_per_sm_nt<128, false>(1024);
  forward_blocks_per_sm_nt<512, false>(1024);
  forward_blocks_per_sm_nt<512, true>(1024);
  forward_blocks_per_sm_nt<256, true>(1024);
  cudaGetLastError();
}

int forward_blocks_per_sm(int nthreads, size_t smem, bool split) {
  if (split) return nthreads == 512   ? forward_blocks_per_sm_nt<512, true>(smem)
                  : nthreads == 256 ? forward_blocks_per_sm_nt<256, true>(smem)
                                    : 0;
  switch (nthreads) {
    case 32: return forward_blocks_per_sm_nt<32, false>(smem);
    case 128: return forward_blocks_per_sm_nt<128, false>(smem);
    case 512: return forward_blocks_per_sm_nt<512, false>(smem);
    default: return 0;
  }
}

}  // namespace qpgpu
