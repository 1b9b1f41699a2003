// qp_forward_512.cu -- forward kernel instantiated for 512 threads per CTA.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<512>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<512>(size_t);
}  // namespace qpgpu

