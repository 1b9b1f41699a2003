// qp_forward_512.cu -- forward kernel instantiated for 512 threads per CTA.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<512>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<512>(size_t);
}  // namespace qpgpu

#ifdef QP_PHASE_TIMERS
extern "C" int qp_debug_phase_cycles_512(unsigned long long* host, int clear) {
  return qpgpu::read_phase_cycles(host, clear) == cudaSuccess ? 0 : -3;
}
#endif
