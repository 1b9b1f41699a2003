// qp_probe.cu -- FP32 FMA throughput probe (include/qp_probe.h): the
// denominator of the FP32-pipe roofline is derived from SM count x 128 FP32
// lanes x 2 FLOP x clock; this loop confirms it on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qp.h"
#include "qp_probe.h"

namespace {

// 8 independent chains per thread hide the FMA latency; the multiplier and
// addend keep the values bounded (x -> a x + b with |a| < 1).
__global__ void __launch_bounds__(1024) fma_probe_kernel(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int qp_fma_probe(int32_t blocks, int32_t threads, int32_t iters, float* out,
                            void* stream) {
  if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return QP_EINVAL;
  fma_probe_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-3f);
  if (cudaGetLastError() != cudaSuccess) return QP_ECUDA;
  return QP_OK;
}
