// qp_forward_128.cu -- forward kernel instantiated for 128 threads per CTA
// (problems up to n = 72, all data in shared memory).
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<128, false>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<128, false>(size_t);
}  // namespace qpgpu
