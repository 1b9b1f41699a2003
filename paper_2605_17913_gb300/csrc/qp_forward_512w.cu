// qp_forward_512w.cu -- the large-problem variant of the forward kernel: 512
// threads per CTA, the five matrices in a per-instance global workspace.
#include "qp_forward.cuh"

namespace qpgpu {
template cudaError_t launch_forward_nt<512, true>(const FwdParams&, size_t, int, cudaStream_t);
template int forward_blocks_per_sm_nt<512, true>(size_t);
}  // namespace qpgpu
