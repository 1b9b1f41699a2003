// qp_api.cu -- C ABI of libqpgpu (declared in include/qp.h): argument
// validation on the host, device workspace, kernel dispatch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "qp.h"
#include "qp_internal.h"

using namespace qpgpu;

struct qp_handle {
  qp_dims dims;
  int device;
  int num_sms;
  int fwd_threads, fwd_blocks_per_sm;
  size_t fwd_smem;
  size_t fwd_smem_tc;       // large variant: shared memory of the 512-thread kernel that the
                            // tensor-core G'WG runs in (one TMEM allocation per SM)
  int bwd_threads;
  size_t bwd_smem;
  int amax;
  long long cache_stride;  // floats per instance in the gradient cache
  bool split;              // large-problem variant (matrices in a global workspace)
  float* ws;               // its workspace, batch * ws_stride floats (owned)
  long long ws_stride;
  // qp_solve_backward_host: two streams and a two-slot device arena (owned,
  // created on its first call)
  cudaStream_t hstream[2];
  float* hbuf;
  size_t hbuf_bytes;
  int hchunk;
  int32_t* diag;  // per-instance diagnostics words (caller's device memory) or nullptr
};

static bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

static bool dims_ok(const qp_dims* d) {
  return d && d->batch >= 0 && d->n >= 1 && d->n_eq >= 0 && d->n_eq <= d->n && d->n_ineq >= 0;
}

#ifdef QP_PHASE_TIMERS
static unsigned long long* g_phase_counters = nullptr;
#endif

namespace qpgpu {
qp_dims handle_dims(const qp_handle* h) { return h->dims; }

int settings_to_params(const qp_settings* st, FwdParams* P) {
  if (!(st->tol > 0.0f) || st->max_iter < 0 || st->formulation < 0 || st->formulation > 2 ||
      st->sigma_mode < 0 || st->sigma_mode > 1 || !(st->kappa_relax >= 0.0f) ||
      st->residual_norm < 0 || st->residual_norm > 1 || st->refine_steps < 0 ||
      st->relax_chord < 0 || st->relax_chord > 1 || st->refine_forward < 0 ||
      st->refine_forward > 16)
    return QP_EINVAL;
  if (st->gwg_precision < QP_GWG_FP32 || st->gwg_precision > QP_GWG_BF16) return QP_EINVAL;
  if (st->sigma_mode == QP_SIGMA_CONSTANT && !(st->sigma >= 0.0f && st->sigma <= 1.0f))
    return QP_EINVAL;
  P->tol = st->tol;
  P->sigma = st->sigma;
  P->kappa_min = st->kappa_min > 0.0f ? st->kappa_min : 1e-2f * st->tol;
  P->kappa_relax = st->kappa_relax;
  P->relax_tol = st->relax_tol > 0.0f ? st->relax_tol : 0.1f * st->tol;
  P->step_frac = 1.0f;
  P->max_iter = st->max_iter;
  P->relax_max_iter = st->relax_max_iter > 0 ? st->relax_max_iter : st->max_iter;
  P->sigma_mode = st->sigma_mode;
  P->formulation = st->formulation;
  P->norm_abs = st->residual_norm == QP_NORM_ABS;
  P->warm_start = st->warm_start;
  P->refine_steps = st->refine_steps;
  P->gwg = st->gwg_precision;
  P->chord = st->relax_chord;
  P->refine_fwd = st->refine_forward;
  return QP_OK;
}
}  // namespace qpgpu

extern "C" {

#ifdef QP_PHASE_TIMERS
// Tracing build only: device array of 64 phase-cycle counters the forward
// kernel adds to (NULL turns the timers off).
void qp_debug_set_phase_counters(unsigned long long* dev) { g_phase_counters = dev; }
#endif

void qp_settings_default(qp_settings* s) {
  if (!s) return;
  memset(s, 0, sizeof(*s));
  s->tol = 1e-5f;
  s->max_iter = 100;
  s->sigma_mode = QP_SIGMA_MEHROTRA;
  s->sigma = 0.1f;
  s->kappa_min = 0.0f;
  s->kappa_relax = 1e-4f;
  s->relax_tol = 0.0f;
  s->relax_max_iter = 0;
  s->formulation = QP_IMPLICIT;
  s->residual_norm = QP_NORM_SCALED;
  s->gwg_precision = QP_GWG_FP32;
  s->refine_steps = 3;
  s->warm_start = 0;
  s->relax_chord = 0;
  s->refine_forward = 0;
}

const char* qp_status_string(int code) {
  switch (code) {
    case QP_OK: return "QP_OK / QP_SOLVED";
    case QP_PENDING: return "QP_PENDING / QP_MAX_ITER";
    case QP_STALLED: return "QP_STALLED";
    case QP_NUMERICAL: return "QP_NUMERICAL";
    case QP_BAD_INPUT: return "QP_BAD_INPUT";
    case QP_EINVAL: return "QP_EINVAL: invalid argument";
    case QP_ENOMEM: return "QP_ENOMEM: device allocation failed";
    case QP_ECUDA: return "QP_ECUDA: CUDA runtime error";
    case QP_EAGAIN: return "QP_EAGAIN: not admissible now";
    case QP_ETIMEOUT: return "QP_ETIMEOUT: bounded wait ran out";
    case QP_ENOTSUP: return "QP_ENOTSUP: size or option not supported";
    case QP_ESTATE: return "QP_ESTATE: call out of order";
    default: return "unknown code";
  }
}

size_t qp_smem_bytes(int32_t n, int32_t n_eq, int32_t n_ineq) {
  if (n < 1 || n_eq < 0 || n_eq > n || n_ineq < 0) return 0;
  return forward_config(n, n_ineq, n_eq, nullptr, nullptr);
}

size_t qp_workspace_bytes(const qp_dims* dims) {
  if (!dims_ok(dims)) return 0;
  long long ws = 0;
  if (forward_config(dims->n, dims->n_ineq, dims->n_eq, nullptr, nullptr, &ws) == 0) return 0;
  return (size_t)dims->batch * (size_t)ws * sizeof(float);
}

int qp_handle_create(const qp_dims* dims, qp_handle** out) {
  return qp_handle_create_threads(dims, 0, out);
}

int qp_handle_create_threads(const qp_dims* dims, int32_t threads_per_qp, qp_handle** out) {
  if (!out || !dims_ok(dims)) return QP_EINVAL;
  *out = nullptr;
  if (threads_per_qp != 0 && threads_per_qp != 32 && threads_per_qp != 128 &&
      threads_per_qp != 256 && threads_per_qp != 512)
    return QP_ENOTSUP;
  qp_handle* h = (qp_handle*)calloc(1, sizeof(qp_handle));
  if (!h) return QP_ENOMEM;
  h->dims = *dims;
  const int n = dims->n, m = dims->n_ineq, p = dims->n_eq;
  const bool warp = threads_per_qp == 32 ||
                    (threads_per_qp == 0 && dims->batch >= kWarpPerQpMinBatch);
  h->fwd_smem = forward_config(n, m, p, &h->fwd_threads, &h->amax, &h->ws_stride, warp,
                               threads_per_qp == 256 ? 256 : 512, threads_per_qp == 512);
  if (threads_per_qp != 0 && h->fwd_threads != threads_per_qp) {
    free(h);
    return QP_ENOTSUP;
  }
  h->split = h->ws_stride > 0;
  h->fwd_smem_tc = h->split ? forward_config(n, m, p, nullptr, nullptr, nullptr, false, 512) : 0;
  h->bwd_smem = backward_smem_bytes(n, m, p, h->amax, h->split, &h->bwd_threads);
  h->cache_stride = cache_layout(n, m, p, h->amax, h->split).stride;
  if (h->fwd_smem == 0 || h->bwd_smem == 0) {
    free(h);
    return QP_ENOTSUP;
  }
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
          cudaSuccess) {
    cudaGetLastError();
    free(h);
    return QP_ECUDA;
  }
  h->fwd_blocks_per_sm = forward_blocks_per_sm(h->fwd_threads, h->fwd_smem, h->split);
  if (h->fwd_blocks_per_sm < 1) {
    cudaGetLastError();
    free(h);
    return QP_ENOTSUP;
  }
  if (h->split && dims->batch > 0) {
    const size_t bytes = (size_t)dims->batch * (size_t)h->ws_stride * sizeof(float);
    if (cudaMalloc((void**)&h->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      free(h);
      return QP_ENOMEM;
    }
  }
  *out = h;
  return QP_OK;
}

int qp_handle_query(const qp_handle* h, qp_handle_info* out) {
  if (!h || !out) return QP_EINVAL;
  out->fwd_threads = h->fwd_threads;
  out->fwd_blocks_per_sm = h->fwd_blocks_per_sm;
  out->bwd_threads = h->bwd_threads;
  out->max_active = h->amax;
  out->large_variant = h->split ? 1 : 0;
  out->fwd_smem_bytes = h->fwd_smem;
  return QP_OK;
}

int qp_handle_set_diag(qp_handle* h, int32_t* diag) {
  if (!h || (diag && !aligned4(diag))) return QP_EINVAL;
  h->diag = diag;
  return QP_OK;
}

int qp_handle_destroy(qp_handle* h) {
  if (!h) return QP_EINVAL;
  if (h->ws) cudaFree(h->ws);
  if (h->hbuf) cudaFree(h->hbuf);
  for (cudaStream_t s : h->hstream)
    if (s) cudaStreamDestroy(s);
  free(h);
  return QP_OK;
}

size_t qp_grad_cache_bytes(const qp_dims* dims) {
  if (!dims_ok(dims)) return 0;
  int amax = 0;
  long long ws = 0;
  if (forward_config(dims->n, dims->n_ineq, dims->n_eq, nullptr, &amax, &ws) == 0) return 0;
  return (size_t)dims->batch *
         (size_t)cache_layout(dims->n, dims->n_ineq, dims->n_eq, amax, ws > 0).stride *
         sizeof(float);
}

namespace {
// The forward kernel over B instances (B <= the handle's batch) of the given
// arrays; ws: the large variant's workspace for them.
int solve_impl(qp_handle* h, const qp_settings* st, int B, float* ws, const float* Q,
               const float* q, const float* A, const float* b, const float* G, const float* hv,
               float* x, float* y, float* z, float* s, int32_t* status, int32_t* iters,
               float* kkt_res, float* grad_cache, cudaStream_t stream);
int backward_impl(qp_handle* h, int B, const float* grad_cache, const float* Q, const float* A,
                  const float* G, const float* dl_dx, float* dQ, float* dq, float* dA, float* db,
                  float* dG, float* dh, cudaStream_t stream);
}  // namespace

int qp_solve_batch(qp_handle* h, const qp_settings* st, const float* Q, const float* q,
                   const float* A, const float* b, const float* G, const float* hv, float* x,
                   float* y, float* z, float* s, int32_t* status, int32_t* iters, float* kkt_res,
                   float* grad_cache, void* stream) {
  if (!h || !st) return QP_EINVAL;
  return solve_impl(h, st, h->dims.batch, h->ws, Q, q, A, b, G, hv, x, y, z, s, status, iters,
                    kkt_res, grad_cache, (cudaStream_t)stream);
}

int qp_backward_batch(qp_handle* h, const float* grad_cache, const float* Q, const float* A,
                      const float* G, const float* dl_dx, float* dQ, float* dq, float* dA,
                      float* db, float* dG, float* dh, void* stream) {
  if (!h) return QP_EINVAL;
  return backward_impl(h, h->dims.batch, grad_cache, Q, A, G, dl_dx, dQ, dq, dA, db, dG, dh,
                       (cudaStream_t)stream);
}

}  // extern "C"

namespace {
int solve_impl(qp_handle* h, const qp_settings* st, int B, float* ws, const float* Q,
               const float* q, const float* A, const float* b, const float* G, const float* hv,
               float* x, float* y, float* z, float* s, int32_t* status, int32_t* iters,
               float* kkt_res, float* grad_cache, cudaStream_t stream) {
  const int n = h->dims.n, m = h->dims.n_ineq, p = h->dims.n_eq;
  if (B == 0) return QP_OK;
  if (!Q || !q || !x || (p > 0 && (!A || !b || !y)) || (m > 0 && (!G || !hv || !z || !s)))
    return QP_EINVAL;
  const void* ptrs[] = {Q, q, A, b, G, hv, x, y, z, s, status, iters, kkt_res};
  for (const void* ptr : ptrs)
    if (ptr && !aligned4(ptr)) return QP_EINVAL;
  if (grad_cache && (reinterpret_cast<uintptr_t>(grad_cache) & 15)) return QP_EINVAL;
  FwdParams P;
  memset(&P, 0, sizeof(P));
  const int rc = settings_to_params(st, &P);
  if (rc != QP_OK) return rc;
  // tensor-core G'WG exists in the large-problem variant only
  if (P.gwg != QP_GWG_FP32 && !h->split) return QP_ENOTSUP;
  P.batch = B; P.n = n; P.m = m; P.p = p; P.amax = h->amax;
  P.Q = Q; P.q = q; P.A = A; P.b = b; P.G = G; P.h = hv;
  P.x = x; P.y = y; P.z = z; P.s = s;
  P.status = status; P.iters = iters; P.kkt = kkt_res;
  P.cache = grad_cache;
  P.cache_stride = h->cache_stride;
  P.ws = ws;
  P.ws_stride = h->ws_stride;
  // the handle's diagnostics array covers its uniform batch (not the host
  // path's chunks, which pass their own arrays)
  P.diag = (B == h->dims.batch && ws == h->ws) ? h->diag : nullptr;
#ifdef QP_PHASE_TIMERS
  P.timers = g_phase_counters;
#endif
  // one CTA per instance: the block scheduler hands a new instance to an SM
  // as soon as one finishes, which balances uneven iteration counts
  // the tensor-core G'WG runs in the 512-thread large variant
  const bool tc512 = h->split && P.gwg != QP_GWG_FP32;
  cudaError_t e = launch_forward(P, tc512 ? 512 : h->fwd_threads,
                                 tc512 ? h->fwd_smem_tc : h->fwd_smem, B, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QP_ECUDA;
  }
  return QP_OK;
}

int backward_impl(qp_handle* h, int B, const float* grad_cache, const float* Q, const float* A,
                  const float* G, const float* dl_dx, float* dQ, float* dq, float* dA, float* db,
                  float* dG, float* dh, cudaStream_t stream) {
  const int n = h->dims.n, m = h->dims.n_ineq, p = h->dims.n_eq;
  if (B == 0) return QP_OK;
  if (!grad_cache || !dl_dx || !Q || (m > 0 && !G) || (p > 0 && !A)) return QP_EINVAL;
  if (reinterpret_cast<uintptr_t>(grad_cache) & 15) return QP_EINVAL;
  const void* ptrs[] = {Q, A, G, dl_dx, dQ, dq, dA, db, dG, dh};
  for (const void* ptr : ptrs)
    if (ptr && !aligned4(ptr)) return QP_EINVAL;
  BwdParams P;
  memset(&P, 0, sizeof(P));
  P.batch = B; P.n = n; P.m = m; P.p = p; P.amax = h->amax;
  P.split = h->split ? 1 : 0;
  P.Q = Q; P.A = A; P.G = G; P.g = dl_dx; P.cache = grad_cache; P.cache_stride = h->cache_stride;
  P.dQ = dQ; P.dq = dq; P.dA = p > 0 ? dA : nullptr; P.db = p > 0 ? db : nullptr;
  P.dG = m > 0 ? dG : nullptr; P.dh = m > 0 ? dh : nullptr;
  P.diag = B == h->dims.batch ? h->diag : nullptr;
  cudaError_t e = launch_backward(P, h->bwd_threads, h->bwd_smem, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QP_ECUDA;
  }
  return QP_OK;
}
// Floats per instance of the host path's device arrays, each region of a
// slot rounded up to 64 floats (the cache needs 16-byte alignment).
struct HostLayout {
  long long Q, q, A, b, G, h, g, x, y, z, s, st, it, kkt, dQ, dq, dA, db, dG, dh, cache, total;
};

long long r64(long long v) { return (v + 63) & ~63LL; }

HostLayout host_layout(const qp_handle* h, long long C) {
  const long long n = h->dims.n, m = h->dims.n_ineq, p = h->dims.n_eq;
  HostLayout L;
  long long o = 0;
  auto take = [&](long long per) { const long long r = o; o += r64(C * per); return r; };
  L.Q = take(n * n); L.q = take(n); L.A = take(p * n); L.b = take(p); L.G = take(m * n);
  L.h = take(m); L.g = take(n);
  L.x = take(n); L.y = take(p); L.z = take(m); L.s = take(m);
  L.st = take(1); L.it = take(1); L.kkt = take(1);
  L.dQ = take(n * n); L.dq = take(n); L.dA = take(p * n); L.db = take(p); L.dG = take(m * n);
  L.dh = take(m);
  L.cache = take(h->cache_stride);
  L.total = o;
  return L;
}
}  // namespace

extern "C" {

int qp_solve_backward_host(qp_handle* h, const qp_settings* st, const float* Q, const float* q,
                           const float* A, const float* b, const float* G, const float* hv,
                           const float* dl_dx, float* x, float* y, float* z, float* s,
                           int32_t* status, int32_t* iters, float* kkt_res, float* dQ, float* dq,
                           float* dA, float* db, float* dG, float* dh) {
  if (!h || !st) return QP_EINVAL;
  const int B = h->dims.batch, n = h->dims.n, m = h->dims.n_ineq, p = h->dims.n_eq;
  if (B == 0) return QP_OK;
  if (!Q || !q || !x || (p > 0 && (!A || !b || !y)) || (m > 0 && (!G || !hv || !z || !s)))
    return QP_EINVAL;
  const bool grad = dl_dx != nullptr;
  FwdParams chk;
  memset(&chk, 0, sizeof(chk));
  int rc = settings_to_params(st, &chk);
  if (rc != QP_OK) return rc;
  if (chk.gwg != QP_GWG_FP32 && !h->split) return QP_ENOTSUP;
  // about four chunks per batch, each a whole number of waves of resident
  // CTAs: a partial last wave per chunk left SMs idle (chunks of 1024 at
  // 456 resident: 5 % slower than 912)
  if (h->hchunk == 0) {
    const long long resident = (long long)h->fwd_blocks_per_sm * h->num_sms;
    long long waves = (B + 2 * resident) / (4 * resident);
    if (waves < 1) waves = 1;
    long long C = waves * resident;
    if (C > B) C = B;
    h->hchunk = (int)C;
  }
  if (!h->hbuf) {
    const size_t bytes = 2 * (size_t)host_layout(h, h->hchunk).total * sizeof(float);
    if (cudaMalloc((void**)&h->hbuf, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->hbuf = nullptr;
      return QP_ENOMEM;
    }
    h->hbuf_bytes = bytes;
  }
  for (cudaStream_t& sm : h->hstream) {
    if (!sm && cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      sm = nullptr;
      return QP_ECUDA;
    }
  }
  const long long C = h->hchunk;
  const HostLayout L = host_layout(h, C);
  bool ok = true;
  auto h2d = [&](float* dst, const void* src, long long count, cudaStream_t sm) {
    if (ok && count > 0 && src)
      ok = cudaMemcpyAsync(dst, src, (size_t)count * 4, cudaMemcpyHostToDevice, sm) == cudaSuccess;
  };
  auto d2h = [&](void* dst, const float* src, long long count, cudaStream_t sm) {
    if (ok && count > 0 && dst)
      ok = cudaMemcpyAsync(dst, src, (size_t)count * 4, cudaMemcpyDeviceToHost, sm) == cudaSuccess;
  };
  // chunk i runs on stream i % 2 in slot i % 2: the slot's previous chunk is
  // earlier on the same stream, so reuse needs no further synchronisation
  for (long long c0 = 0, i = 0; c0 < B && ok && rc == QP_OK; c0 += C, ++i) {
    const long long nb = (B - c0) < C ? (B - c0) : C;
    cudaStream_t sm = h->hstream[i & 1];
    float* d = h->hbuf + (i & 1) * L.total;
    h2d(d + L.Q, Q + c0 * n * n, nb * n * n, sm);
    h2d(d + L.q, q + c0 * n, nb * n, sm);
    if (p > 0) { h2d(d + L.A, A + c0 * p * n, nb * p * n, sm); h2d(d + L.b, b + c0 * p, nb * p, sm); }
    if (m > 0) { h2d(d + L.G, G + c0 * m * n, nb * m * n, sm); h2d(d + L.h, hv + c0 * m, nb * m, sm); }
    if (grad) h2d(d + L.g, dl_dx + c0 * n, nb * n, sm);
    if (!ok) break;
    float* ws = h->ws ? h->ws + c0 * h->ws_stride : nullptr;
    rc = solve_impl(h, st, (int)nb, ws, d + L.Q, d + L.q, d + L.A, d + L.b, d + L.G, d + L.h,
                    d + L.x, d + L.y, d + L.z, d + L.s, reinterpret_cast<int32_t*>(d + L.st),
                    reinterpret_cast<int32_t*>(d + L.it), d + L.kkt, grad ? d + L.cache : nullptr,
                    sm);
    if (rc == QP_OK && grad)
      rc = backward_impl(h, (int)nb, d + L.cache, d + L.Q, d + L.A, d + L.G, d + L.g, d + L.dQ,
                         d + L.dq, d + L.dA, d + L.db, d + L.dG, d + L.dh, sm);
    if (rc != QP_OK) break;
    d2h(x + c0 * n, d + L.x, nb * n, sm);
    if (p > 0) d2h(y + c0 * p, d + L.y, nb * p, sm);
    if (m > 0) { d2h(z + c0 * m, d + L.z, nb * m, sm); d2h(s + c0 * m, d + L.s, nb * m, sm); }
    d2h(status ? status + c0 : nullptr, d + L.st, nb, sm);
    d2h(iters ? iters + c0 : nullptr, d + L.it, nb, sm);
    d2h(kkt_res ? kkt_res + c0 : nullptr, d + L.kkt, nb, sm);
    if (grad) {
      d2h(dQ ? dQ + c0 * n * n : nullptr, d + L.dQ, nb * n * n, sm);
      d2h(dq ? dq + c0 * n : nullptr, d + L.dq, nb * n, sm);
      if (p > 0) {
        d2h(dA ? dA + c0 * p * n : nullptr, d + L.dA, nb * p * n, sm);
        d2h(db ? db + c0 * p : nullptr, d + L.db, nb * p, sm);
      }
      if (m > 0) {
        d2h(dG ? dG + c0 * m * n : nullptr, d + L.dG, nb * m * n, sm);
        d2h(dh ? dh + c0 * m : nullptr, d + L.dh, nb * m, sm);
      }
    }
  }
  // wait for everything enqueued, also after an error
  for (cudaStream_t sm : h->hstream)
    if (cudaStreamSynchronize(sm) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    return QP_ECUDA;
  }
  return rc;
}

}  // extern "C"
