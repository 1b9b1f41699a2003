// qp_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace qpgpu {

// Parameters of one forward launch (all device pointers).
struct FwdParams {
  int batch, n, m, p;
  const float *Q, *q, *A, *b, *G, *h;
  float *x, *y, *z, *s;
  int32_t *status, *iters;
  float* kkt;
  // settings
  float tol, sigma, kappa_min, kappa_relax, relax_tol, step_frac;
  int max_iter, relax_max_iter, sigma_mode, formulation, norm_abs, warm_start, refine_steps;
  // gradient cache (nullptr: no relax, no cache)
  float* cache;
  long long cache_stride;
};

struct BwdParams {
  int batch, n, m, p;
  const float* G;
  const float* g;
  const float* cache;
  long long cache_stride;
  float *dQ, *dq, *dA, *db, *dG, *dh;
};

// Per-instance layout of the factor cache, in floats (offsets multiples of 4).
struct CacheLayout {
  int oL, oU, oLs, oW, ox, oy, oz, stride;
};

__host__ __device__ inline CacheLayout cache_layout(int n, int m, int p) {
  auto r4 = [](long long v) -> int { return (int)((v + 3) & ~3LL); };
  CacheLayout c;
  int o = 0;
  c.oL = o; o += r4((long long)n * (n + 1) / 2);
  c.oU = o; o += r4((long long)p * n);
  c.oLs = o; o += r4((long long)p * (p + 1) / 2);
  c.oW = o; o += r4(m);
  c.ox = o; o += r4(n);
  c.oy = o; o += r4(p);
  c.oz = o; o += r4(m);
  c.stride = o;
  return c;
}

// Shared-memory bytes of the forward kernel for a size (0 if unsupported),
// and the thread count it launches with.
size_t forward_smem_bytes(int n, int m, int p, int* nthreads);
cudaError_t launch_forward(const FwdParams& P, int nthreads, size_t smem, int grid,
                           cudaStream_t stream);
int forward_blocks_per_sm(int nthreads, size_t smem);

size_t backward_smem_bytes(int n, int m, int p, int* nthreads);
cudaError_t launch_backward(const BwdParams& P, int nthreads, size_t smem, cudaStream_t stream);

}  // namespace qpgpu
