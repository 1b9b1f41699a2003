// qp_forward_32.cu -- forward kernel instantiated for one warp per CTA: one
// QP per warp for small problems (n <= 32) in large batches, many CTAs per SM.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<32, false>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<32, false>(size_t);
}  // namespace qpgpu
