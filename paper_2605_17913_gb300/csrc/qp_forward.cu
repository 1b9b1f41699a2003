// qp_forward.cu -- host-side dispatch of the forward kernel by block size.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qpgpu {

template <int NT>
cudaError_t launch_forward_nt(const FwdParams& P, size_t smem, int grid, cudaStream_t st);
template <int NT>
int forward_blocks_per_sm_nt(size_t smem);

size_t forward_smem_bytes(int n, int m, int p, int* nthreads) {
  const int nt = n <= 24 ? 128 : (n <= 72 ? 256 : 512);
  const Layout L = make_layout(n, m, p, nt);
  const size_t bytes = (size_t)L.total * sizeof(float);
  if (nthreads) *nthreads = nt;
  if (n > 128 || p > 128 || bytes > 227 * 1024) return 0;
  return bytes;
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
