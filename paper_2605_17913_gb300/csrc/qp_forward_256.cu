// qp_forward_256.cu -- forward kernel instantiated for 256 threads per CTA.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<256>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<256>(size_t);
}  // namespace qpgpu

