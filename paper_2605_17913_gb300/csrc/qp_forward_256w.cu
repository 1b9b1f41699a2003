// qp_forward_256w.cu -- instantiation: large-problem variant, 256 threads
// per QP (two CTAs per SM), FP32 G'WG.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<256, true>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<256, true>(size_t);
}  // namespace qpgpu
