// qp_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "qp.h"

namespace qpgpu {

// One request of a ragged launch (serving): its sizes and device pointers.
// A CTA that finds a descriptor table uses its own entry in place of the
// launch's uniform sizes and batch-strided pointers, with instance index 0.
struct ReqDesc {
  int n, m, p, amax;
  const float *Q, *q, *A, *b, *G, *h;
  float *x, *y, *z, *s;
  int32_t *status, *iters;
  float* kkt;
  float* cache;     // gradient cache (nullptr: no relax, no cache)
  float* ws;        // workspace of the large-problem variant
  const float* g;   // dl/dx for the backward pass
  float *dQ, *dq, *dA, *db, *dG, *dh;
  int bnt;          // threads of the backward pass (persistent serving kernel)
  int pad_;
};

// Parameters of one forward launch (all device pointers).
struct FwdParams {
  int batch, n, m, p;
  const float *Q, *q, *A, *b, *G, *h;
  float *x, *y, *z, *s;
  int32_t *status, *iters;
  float* kkt;
  int amax;  // rows kept as multipliers at most (shared-memory budget)
  // settings
  float tol, sigma, kappa_min, kappa_relax, relax_tol, step_frac;
  int max_iter, relax_max_iter, sigma_mode, formulation, norm_abs, warm_start, refine_steps;
  int gwg;  // G'WG products: 0 FP32, 1 TF32, 2 BF16 (tensor cores, large variant only)
  int chord;  // Alg. 2 reuses the factorisation of its first iterate (chord steps)
  int refine_fwd;  // refinement sweeps of each folded Newton solve (large variant)
  // gradient cache (nullptr: no relax, no cache)
  float* cache;
  long long cache_stride;
  // per-instance global workspace of the large-problem variant (K, G, A, Y, C
  // outside shared memory); nullptr for sizes that fit on chip
  float* ws;
  long long ws_stride;
  const ReqDesc* desc;  // ragged launch: one descriptor per CTA (nullptr: uniform batch)
  int32_t* diag;        // per-instance diagnostics word (nullptr: no stage tests)
#ifdef QP_PHASE_TIMERS
  unsigned long long* timers;  // device counters of the phase timers (tracing build)
#endif
};

struct BwdParams {
  int batch, n, m, p, amax;
  int split;  // cache in the unpacked (large-problem) layout
  const float *Q, *A, *G;
  const float* g;
  const float* cache;
  long long cache_stride;
  float *dQ, *dq, *dA, *db, *dG, *dh;
  const ReqDesc* desc;  // ragged launch: one descriptor per CTA (nullptr: uniform batch)
  int32_t* diag;        // per-instance diagnostics word (nullptr: not written)
};

// Per-instance layout of the gradient cache, in floats (offsets multiples of
// 4): header (active rows a, rows nf = a + p of F, refinement sweeps of the
// adjoint solve, as int32), L of
// K_I = Q + G_I'W_I G_I (packed lower), Y = F L^-T (nf rows of n), L_C of
// C = D + Y Y' (packed lower), W of the inactive rows and 1/W of the active
// rows, the row -> position map
// (int32, -1 for inactive rows) and the point (x, y, z); s completes the
// solve's snapshot (x, y, z, s) that the relax starts from.
// Large-problem variant (split): L, Y and L_C are stored unpacked with the
// forward kernel's workspace strides (ldk for L and Y, ldc for L_C: multiples
// of 4 floats whose quarter is odd), so that the backward pass reads them in
// place.
struct CacheLayout {
  int oHdr, oL, oY, oLC, oW, oPos, ox, oy, oz, os, stride;
  int ldk, ldc;  // strides of L / Y and of L_C (split layout; 0 when packed)
};

__host__ __device__ inline CacheLayout cache_layout(int n, int m, int p, int amax,
                                                    bool split = false) {
  auto r4 = [](long long v) -> int { return (int)((v + 3) & ~3LL); };
  const long long f = (long long)amax + p;
  CacheLayout c;
  int o = 0;
  // the forward's workspace strides: a multiple of 4 floats whose quarter is odd
  auto ldv = [](long long v) -> int {
    int l = (int)((v < 1 ? 1 : v) + 3) & ~3;
    return ((l >> 2) & 1) ? l : l + 4;
  };
  c.ldk = split ? ldv(n) : 0;
  c.ldc = split ? ldv(f + 2) : 0;
  c.oHdr = o; o += 4;
  c.oL = o; o += r4(split ? (long long)n * c.ldk : (long long)n * (n + 1) / 2);
  c.oY = o; o += r4(split ? f * c.ldk : f * n);
  c.oLC = o; o += r4(split ? f * c.ldc : f * (f + 1) / 2);
  c.oW = o; o += r4(m);
  c.oPos = o; o += r4(m);
  c.ox = o; o += r4(n);
  c.oy = o; o += r4(p);
  c.oz = o; o += r4(m);
  c.os = o; o += r4(m);
  c.stride = o;
  return c;
}

// Launch configuration of the forward kernel for a size: shared-memory bytes
// (0 if unsupported), threads per CTA, the active-row cap amax and, for the
// large-problem variant, the global workspace floats per instance (0 when
// everything fits in shared memory).  warp_per_qp: one warp per CTA for
// n <= 32 (throughput of large batches; the amax is the same either way).
// large_threads: threads per CTA of the large variant, 512 (one CTA per SM)
// or 256 (two; FP32 G'WG only).  onchip512: 512 threads for every n <= 128
// at the amax of the default (0 if that layout does not fit).
size_t forward_config(int n, int m, int p, int* nthreads, int* amax,
                      long long* ws_floats = nullptr, bool warp_per_qp = false,
                      int large_threads = 512, bool onchip512 = false);

// Batches from this size up run problems with n <= 32 one warp per QP.
constexpr int kWarpPerQpMinBatch = 2048;
cudaError_t launch_forward(const FwdParams& P, int nthreads, size_t smem, int grid,
                           cudaStream_t stream);
int forward_blocks_per_sm(int nthreads, size_t smem, bool split);

// Dynamic shared memory of the backward kernel (0: size not supported) and
// its threads per CTA.
size_t backward_smem_bytes(int n, int m, int p, int amax, bool split, int* nthreads);
// Uniform batch over P.batch instances, or (P.desc set) a ragged launch over
// P.desc[0 .. P.batch) with nthreads = backward_threads of its size class.
cudaError_t launch_backward(const BwdParams& P, int nthreads, size_t smem, cudaStream_t stream);
// Threads per CTA of the backward kernel for a size.
int backward_threads(int n, bool split);

// Load the kernels' modules ahead of their first launch (the runtime loads
// lazily); for callers whose launches must not pay for loading.
// Persistent serving kernel (qp_serve_persist.cu).  The ring, its
// completion words and the control block live in mapped host memory; head is
// a device counter of claimed requests.
struct ServeCtl {
  uint32_t tail;    // requests published (host: release store)
  uint32_t stop;    // host: CTAs leave their loop after the request they hold
  uint32_t exited;  // CTAs that left their loop (device: system-scope atomic)
  uint32_t pad_;
};
struct ServeParams {
  FwdParams base;          // solver settings of every request
  const ReqDesc* ring;     // cap descriptors; request s at s % cap
  uint32_t* done;          // done[s % cap] = s + 1 once request s is complete
  ServeCtl* ctl;
  uint32_t* head;          // device: next request to claim
  uint32_t cap;
  uint32_t pad_;
  unsigned long long idle_ns;  // a CTA with no request for this long leaves
  unsigned long long life_ns;  // a CTA takes no new request after this long
};
// Threads per CTA of the persistent kernel, and the dynamic shared memory it
// is launched with (every supported size's forward and backward fit).
constexpr int kServeThreads = 512;
size_t serve_kernel_smem();
cudaError_t launch_serve_kernel(const ServeParams& S, int grid, cudaStream_t stream);
// CTAs of the persistent kernel that fit one SM (0 on error).
int serve_kernel_blocks_per_sm();

void preload_forward_kernels();
void preload_backward_kernels();

// Problem sizes of a handle (struct qp_handle is private to qp_api.cu).
qp_dims handle_dims(const qp_handle* h);

// Validate solver settings and copy them into launch parameters (QP_OK,
// QP_EINVAL or QP_ENOTSUP).
int settings_to_params(const qp_settings* st, FwdParams* P);

}  // namespace qpgpu
