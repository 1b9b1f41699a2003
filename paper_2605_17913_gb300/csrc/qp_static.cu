// qp_static.cu -- qp_solve_backward_static: solve, relax and backward pass in
// one call, with the factor cache between them held in a fixed device array
// of this library, so that the call itself allocates no memory.
//
// The factor cache (qp_grad_cache_bytes) normally comes from the caller.  A
// caller that cannot provide it on the call path -- a fixed-rate control or
// planning loop that must not call cudaMalloc there (an allocation can
// synchronise the device and stall the loop for an unbounded time), or a
// host program whose device memory is owned by an arena that is not lent to
// libraries -- can still get gradients through this call, for batches whose
// cache fits in QP_STATIC_CACHE_BYTES.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qp.h"
#include "qp_internal.h"

// The scratch.  A __device__ variable exists once per device context, so
// every call on a device uses this same array from offset 0: calls whose
// device work overlaps in time (on different streams, or issued from
// different host threads without ordering) race on it; calls ordered on one
// stream do not.  Its contents need not start at any value: the solve writes
// every instance's slot header (a factor, or the unwritten mark of an instance
// with non-finite data) before the backward pass reads the slot.
static __device__ __align__(256) float g_static_cache[QP_STATIC_CACHE_BYTES / sizeof(float)];

namespace {

// The array's device address on the current device.  Looked up on every call
// (cheap once this library's device code is loaded in the context): a cached
// address could go stale when the context is destroyed and recreated
// (cudaDeviceReset), which reloads the module, possibly elsewhere.  The first
// lookup in a context loads the device code, which reserves the array.
int static_cache_on_current_device(float** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_cache);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return QP_ECUDA;
  }
  *out = static_cast<float*>(p);
  return QP_OK;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

}  // namespace

extern "C" int qp_solve_backward_static(qp_handle* h, const qp_settings* settings,
                                        const float* Q, const float* q, const float* A,
                                        const float* b, const float* G, const float* h_,
                                        const float* dl_dx, float* x, float* y, float* z,
                                        float* s, int32_t* status, int32_t* iters,
                                        float* kkt_res, float* dQ, float* dq, float* dA,
                                        float* db, float* dG, float* dh, void* stream) {
  if (!h || !settings) return QP_EINVAL;
  const qp_dims dims = qpgpu::handle_dims(h);
  if (dims.batch == 0) return QP_OK;
  // size limit first: a batch whose cache does not fit is refused outright
  if (qp_grad_cache_bytes(&dims) > (size_t)QP_STATIC_CACHE_BYTES) return QP_ENOTSUP;
  // arguments only the backward pass reads (the solve checks its own before
  // it enqueues anything)
  if (!dl_dx) return QP_EINVAL;
  const void* ptrs[] = {dl_dx, dQ, dq, dA, db, dG, dh};
  for (const void* p : ptrs)
    if (p && !aligned4(p)) return QP_EINVAL;
  float* cache = nullptr;
  int rc = static_cache_on_current_device(&cache);
  if (rc != QP_OK) return rc;
  rc = qp_solve_batch(h, settings, Q, q, A, b, G, h_, x, y, z, s, status, iters, kkt_res, cache,
                      stream);
  if (rc != QP_OK) return rc;
  return qp_backward_batch(h, cache, Q, A, G, dl_dx, dQ, dq, dA, db, dG, dh, stream);
}
