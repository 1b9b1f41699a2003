// qp_forward_512.cu -- forward kernel instantiated for 512 threads per CTA
// (problems above n = 72 whose data fit in shared memory).
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<512, false>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<512, false>(size_t);
}  // namespace qpgpu
