// qp_backward.cu -- the backward kernel of Alg. 3 (the per-instance pass is
// in qp_backward.cuh) and its host-side sizing and launch.
#include <mutex>

#include "qp_backward.cuh"

namespace qpgpu {

namespace {

// On chip: at most 102 registers with 128 threads, so that five CTAs fit an
// SM (the shared-memory layout is 42.8 KB at n = 50, m = 100, p = 10), and 128
// with 256 threads (two CTAs where shared memory allows).
template <int NT, bool kGlobal>
__global__ void __launch_bounds__(NT, kGlobal ? 1 : (NT == 128 ? 5 : 2))
    qp_backward_kernel(const BwdParams P) {
  // parameters in shared memory (the body takes them by reference); a ragged
  // launch substitutes this CTA's request, addressed as instance 0
  __shared__ BwdParams sP;
  if (threadIdx.x == 0) {
    sP = P;
    if (P.desc) {
      const ReqDesc& d = P.desc[blockIdx.x];
      sP.batch = 1; sP.n = d.n; sP.m = d.m; sP.p = d.p; sP.amax = d.amax;
      sP.Q = d.Q; sP.A = d.A; sP.G = d.G; sP.g = d.g;
      sP.cache = d.cache; sP.cache_stride = 0;
      sP.dQ = d.dQ; sP.dq = d.dq;
      sP.dA = d.p > 0 ? d.dA : nullptr; sP.db = d.p > 0 ? d.db : nullptr;
      sP.dG = d.m > 0 ? d.dG : nullptr; sP.dh = d.m > 0 ? d.dh : nullptr;
    }
  }
  __syncthreads();
  backward_body<NT, kGlobal>(sP, P.desc ? 0 : blockIdx.x);
}

}  // namespace

// dynamic shared memory left beside the kernel's static parameter copy
constexpr size_t kBwdBudget = 227 * 1024 - 512;

// Threads per CTA: 128 up to n = 72 (measured 25 % faster than 256 at n = 50),
// 256 above (33 % faster than 128 at n = 100) and for the large variant.
int backward_threads(int n, bool split) { return (!split && n <= 72) ? 128 : 256; }

size_t backward_smem_bytes(int n, int m, int p, int amax, bool split, int* nthreads) {
  const int nt = backward_threads(n, split);
  if (nthreads) *nthreads = nt;
  if (split ? (n > 256 || amax + p > 318) : (n > 128 || amax + p > 128)) return 0;
  const size_t bytes = (size_t)make_blayout(n, m, p, amax, nt, split).total * sizeof(float);
  return bytes <= kBwdBudget ? bytes : 0;
}

// The dynamic shared-memory limit is set once per variant, to the largest
// layout (setting it can wait for running kernels: not on the launch path).
template <int NT, bool kGlobal>
cudaError_t configure_backward_v() {
  static std::once_flag once;
  static cudaError_t set = cudaSuccess;
  std::call_once(once, [] {
    set = cudaFuncSetAttribute(qp_backward_kernel<NT, kGlobal>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdBudget);
  });
  return set;
}

template <int NT, bool kGlobal>
cudaError_t launch_backward_v(const BwdParams& P, size_t smem, cudaStream_t st) {
  const cudaError_t set = configure_backward_v<NT, kGlobal>();
  if (set != cudaSuccess) return set;
  qp_backward_kernel<NT, kGlobal><<<P.batch, NT, smem, st>>>(P);
  return cudaGetLastError();
}

// Load every variant's module and set its limit now (kernels load lazily).
void preload_backward_kernels() {
  configure_backward_v<128, false>();
  configure_backward_v<256, false>();
  configure_backward_v<256, true>();
  cudaGetLastError();
}

cudaError_t launch_backward(const BwdParams& P, int nthreads, size_t smem, cudaStream_t st) {
  if (P.split) return launch_backward_v<256, true>(P, smem, st);
  if (nthreads == 128) return launch_backward_v<128, false>(P, smem, st);
  if (nthreads == 256) return launch_backward_v<256, false>(P, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace qpgpu
