// qp_serve_persist.cu -- the persistent serving kernel: CTAs that stay
// resident and take requests one at a time from a ring that the host
// publishes in mapped host memory.
//
// Each CTA (512 threads, one per SM) loops: thread 0 claims the next published
// request (a device counter against the host's tail, read with acquire
// semantics at system scope); the CTA solves it with the 512-thread forward
// (the on-chip variant up to n = 128, the large-problem variant above: Alg. 1
// and, with gradients, Alg. 2), runs Alg. 3 on its first 128 or 256 threads
// when the request asked for gradients (the backward kernel's code and width),
// and thread 0 publishes completion (release at system scope, after every
// thread's stores).  Outputs go straight to mapped host memory.  So a request
// starts as soon as any CTA is free, while the others are in the middle of
// their own Newton iterations, and its arithmetic is that of a batch-1 solve
// at width 512 followed by the backward kernel: results are equal bit for bit.
//
// Every wait is bounded: a CTA that finds no request for idle_ns, that has run
// for life_ns, or that sees the host's stop word leaves the loop (after the
// request it holds) and counts itself out; the host starts CTAs again when
// work arrives.  Memory that one request leaves behind is reused by later
// ones within the kernel's lifetime, so the solver reads its data and the
// factor cache through L2 (kCoh: the read-only path does not see such
// memory change), and the forward's stores are made visible at device scope
// before the backward reads them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "qp_backward.cuh"
#include "qp_forward.cuh"

namespace qpgpu {
namespace {

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Alg. 3 on the CTA's first NT threads, as a function of its own (compiled
// apart from the kernel body, like the forward's run).
template <int NT, bool kGlobal>
__device__ __noinline__ void serve_backward(const BwdParams& B) {
  backward_body<NT, kGlobal, GroupBar<NT>, true>(B, 0);
}

// The parameters of the phase running now: the forward's, then the
// backward's (the forward is done with its own by then).
union ServeShared {
  FwdParams f;
  BwdParams b;
};

__global__ void __launch_bounds__(kServeThreads, 1) qp_serve_kernel(const ServeParams S) {
  using Big = fwd::Solver<kServeThreads, true, true>;
  using Chip = fwd::Solver<kServeThreads, false, true>;
  __shared__ ServeShared sp;
  __shared__ uint32_t s_seq;
  __shared__ int s_have, s_grad, s_bnt;
  const int tid = threadIdx.x;
  const unsigned long long t_start = global_ns();
  Big::init_async();  // the bulk-copy / tensor-core barriers, once (ends with a barrier)
  const bool tc = S.base.gwg != 0;
  if (tc) {
    // TMEM of the tensor-core G'WG, for the CTA's whole life (one CTA per SM)
    if (tid < 32) {
      tc::tmem_alloc(&fwd::fwd_state.tmem, tc::kTmemCols);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  for (;;) {
    if (tid == 0) {
      int have = 0;
      uint32_t seq = 0;
      const unsigned long long t0 = global_ns();
      if (t0 - t_start < S.life_ns) {
        for (;;) {
          if (ld_acquire_sys(&S.ctl->stop)) break;
          const uint32_t tail = ld_acquire_sys(&S.ctl->tail);
          const uint32_t h = ld_relaxed_gpu(S.head);
          if ((int32_t)(tail - h) > 0) {
            if (atomicCAS(S.head, h, h + 1u) == h) {
              have = 1;
              seq = h;
              break;
            }
            continue;  // another CTA took it: try the next one
          }
          if (global_ns() - t0 > S.idle_ns) break;
          __nanosleep(256);
        }
      }
      s_have = have;
      s_seq = seq;
      if (have) {
        const volatile ReqDesc* d = S.ring + (seq % S.cap);
        FwdParams& P = sp.f;
        P = S.base;
        P.batch = 1;
        P.n = d->n; P.m = d->m; P.p = d->p; P.amax = d->amax;
        P.Q = d->Q; P.q = d->q; P.A = d->A; P.b = d->b; P.G = d->G; P.h = d->h;
        P.x = d->x; P.y = d->y; P.z = d->z; P.s = d->s;
        P.status = d->status; P.iters = d->iters; P.kkt = d->kkt;
        P.cache = d->cache; P.cache_stride = 0;
        P.ws = d->ws; P.ws_stride = 0;
        P.desc = nullptr;
        P.diag = nullptr;
        s_grad = d->g != nullptr;
        s_bnt = d->bnt;
      }
    }
    __syncthreads();
    if (!s_have) break;
    const bool split = sp.f.ws != nullptr;
    if (split) {
      Big::init(sp.f.n, sp.f.m, sp.f.p, sp.f.amax, sp.f.ws, sp.f.gwg, sp.f.refine_fwd, true);
      Big::run(sp.f, 0);
    } else {
      Chip::init(sp.f.n, sp.f.m, sp.f.p, sp.f.amax, nullptr, sp.f.gwg, sp.f.refine_fwd, true);
      Chip::run(sp.f, 0);
    }
    if (s_grad) {
      // the cache this CTA just wrote, at device scope before the L2 reads
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const volatile ReqDesc* d = S.ring + (s_seq % S.cap);
        BwdParams& B = sp.b;
        B.batch = 1;
        B.n = d->n; B.m = d->m; B.p = d->p; B.amax = d->amax;
        B.split = split ? 1 : 0;
        B.Q = d->Q; B.A = d->A; B.G = d->G; B.g = d->g;
        B.cache = d->cache; B.cache_stride = 0;
        B.dQ = d->dQ; B.dq = d->dq;
        B.dA = B.p > 0 ? d->dA : nullptr; B.db = B.p > 0 ? d->db : nullptr;
        B.dG = B.m > 0 ? d->dG : nullptr; B.dh = B.m > 0 ? d->dh : nullptr;
        B.desc = nullptr;
        B.diag = nullptr;
      }
      __syncthreads();
      if (split) {
        if (tid < 256) serve_backward<256, true>(sp.b);
      } else if (s_bnt == 128) {
        if (tid < 128) serve_backward<128, false>(sp.b);
      } else {
        if (tid < 256) serve_backward<256, false>(sp.b);
      }
    }
    // every thread's output stores, then the completion word
    __threadfence_system();
    __syncthreads();
    if (tid == 0) st_release_sys(S.done + (s_seq % S.cap), s_seq + 1u);
    // copies that a bounded wait gave up on may still land: this CTA's
    // barriers are no longer trusted, it takes no further request
    if (fwd::fwd_state.async_lost) break;
  }
  if (tc) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(fwd::fwd_state.tmem, tc::kTmemCols);
  }
  if (tid == 0) {
    __threadfence_system();
    atomicAdd_system(&S.ctl->exited, 1u);
  }
}

constexpr size_t kServeSmem = 227 * 1024 - fwd::kStaticSmem;

cudaError_t configure_serve_kernel() {
  static std::once_flag once;
  static cudaError_t set = cudaSuccess;
  std::call_once(once, [] {
    cudaFuncAttributes fa;
    set = cudaFuncGetAttributes(&fa, qp_serve_kernel);
    if (set == cudaSuccess && fa.sharedSizeBytes > (size_t)fwd::kStaticSmem)
      set = cudaErrorInvalidConfiguration;  // the forward's dynamic budget would not fit
    if (set == cudaSuccess)
      set = cudaFuncSetAttribute(qp_serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kServeSmem);
  });
  return set;
}

}  // namespace

size_t serve_kernel_smem() { return kServeSmem; }

cudaError_t launch_serve_kernel(const ServeParams& S, int grid, cudaStream_t stream) {
  const cudaError_t e = configure_serve_kernel();
  if (e != cudaSuccess) return e;
  qp_serve_kernel<<<grid, kServeThreads, kServeSmem, stream>>>(S);
  return cudaGetLastError();
}

int serve_kernel_blocks_per_sm() {
  if (configure_serve_kernel() != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, qp_serve_kernel, kServeThreads,
                                                    kServeSmem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace qpgpu
