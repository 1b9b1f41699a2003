// qp_forward.cu -- host-side sizing and dispatch of the forward kernel.
#include "qp_forward.cuh"

namespace qpgpu {

template <int NT>
cudaError_t launch_forward_nt(const FwdParams& P, size_t smem, int grid, cudaStream_t st);
template <int NT>
int forward_blocks_per_sm_nt(size_t smem);

// Threads per CTA by n (the 256-thread instantiation remains for callers of
// launch_forward that ask for it); amax = rows kept as multipliers, at most min(m, n)
// (at a non-degenerate solution at most n - p rows are active), lowered to
// fit shared memory but not more than 4 below min(m, n - p); amax + p <= 126
// (warp solves hold at most 128 rows, two of them folded right-hand sides).
// Rows beyond amax with W > 1 go to K_I with the smallest W first (tau grows).
size_t forward_config(int n, int m, int p, int* nthreads, int* amax_out) {
  // 128 threads up to n = 72: fewer warps per barrier, no register cap
  // (measured faster than 256 threads at n = 50 by 5 %)
  const int nt = n <= 72 ? 128 : 512;
  if (nthreads) *nthreads = nt;
  if (amax_out) *amax_out = 0;
  if (n < 1 || n > 128 || p > 128 || p > n || m < 0) return 0;
  int amax0 = m < n ? m : n;
  if (amax0 + p > 126) amax0 = 126 - p;
  int floor_a = (m < n - p ? m : n - p) - 4;
  if (floor_a < 0) floor_a = 0;
  const size_t budget = 227 * 1024 - fwd::kStaticSmem;
  for (int amax = amax0; amax >= floor_a && amax >= 0; --amax) {
    const fwd::FLayout L = fwd::make_fwd_layout(n, m, p, amax, nt);
    const size_t bytes = (size_t)L.total * sizeof(float);
    if (bytes <= budget) {
      if (amax_out) *amax_out = amax;
      return bytes;
    }
  }
  return 0;
}

cudaError_t launch_forward(const FwdParams& P, int nthreads, size_t smem, int grid,
                           cudaStream_t st) {
  switch (nthreads) {
    case 128: return launch_forward_nt<128>(P, smem, grid, st);
    case 256: return launch_forward_nt<256>(P, smem, grid, st);
    case 512: return launch_forward_nt<512>(P, smem, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

int forward_blocks_per_sm(int nthreads, size_t smem) {
  switch (nthreads) {
    case 128: return forward_blocks_per_sm_nt<128>(smem);
    case 256: return forward_blocks_per_sm_nt<256>(smem);
    case 512: return forward_blocks_per_sm_nt<512>(smem);
    default: return 0;
  }
}

}  // namespace qpgpu
