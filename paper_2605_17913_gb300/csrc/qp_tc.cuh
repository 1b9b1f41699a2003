// qp_tc.cuh -- G'WG on the fifth-generation tensor cores (tcgen05) for the
// large-problem variant: K_I = Q + sum_k W_k g_k g_k' over the inactive rows,
// with the products in TF32 or BF16 and the sums in FP32 (TMEM).
//
// Operand staging.  The rows g_k are scaled by sqrt(W_k) (W <= tau on the
// inactive rows, so the scaling is bounded) and written to shared memory as
// the n x Kc matrix G_hat' in the K-major canonical layout without swizzle:
// core matrices of 8 rows x 16 bytes (4 TF32 or 8 BF16 values of K),
// 128 contiguous bytes each; 8-row groups adjacent (stride 128 B, the
// descriptor's stride-dimension offset), 16-byte K slabs one after another
// (stride NG * 128 B, its leading-dimension offset).  Both MMA operands are
// the same buffer: D = A B' with A the 128 rows of one tile and B the first
// N rows, so D is a block of G_hat' G_hat.
//
// Tiles.  Rows are padded to 128 * tiles (tiles = ceil(n / 128) <= 2): tile t
// holds rows [128 t, 128 t + 128) and columns [0, 128 (t + 1)) -- the lower
// triangle and the diagonal block -- in TMEM columns [col0(t), col0(t) + N).
// One thread issues the MMAs of a chunk (Kc rows of G) for both tiles and
// commits them to the chunk buffer's mbarrier; two buffers alternate, so the
// next chunk is staged while the tensor cores work.  The epilogue reads TMEM
// with 32x32b loads (warp w reads lanes 32 (w % 4) .. + 31) and writes
// K = Q + D into the lower triangle.  Every mbarrier wait is bounded; on a
// timeout the routine reports failure and the caller falls back to FP32.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "qp_device.cuh"

namespace qpgpu {
namespace tc {

constexpr int kKc = 32;           // rows of G per staged chunk
constexpr uint32_t kTmemCols = 512;  // TMEM columns per CTA (two tiles use 384)
constexpr int kWaitIters = 1 << 22;  // bound on mbarrier polls

__host__ __device__ inline int tiles_for(int n) { return (n + 127) / 128; }
// bytes of one staging buffer (the routine uses two); element size 4 (TF32) or 2 (BF16)
__host__ __device__ inline int stage_bytes(int n, int esize) {
  return (kKc * esize / 16) * (tiles_for(n) * 16) * 128;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kWaitIters; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo / sbo in bytes
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; base offset 0, no swizzle
  return d;
}

// instruction descriptor: FP32 accumulator, A and B of one type (2 = TF32 for
// kind::tf32, 1 = BF16 for kind::f16), both K-major, M = 128, N
__device__ __forceinline__ uint32_t instr_desc(uint32_t ab_type, uint32_t N) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((N >> 3) << 17) | ((128u >> 4) << 24);
}

template <bool kBF16>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t accumulate) {
  if (kBF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// K (lower triangle, stride ldk) = Q + sum over rows[0 .. nrows) of
// W[r] G[r]' G[r], products on the tensor cores.  Q from K's strict upper
// triangle and qd.  stage: two buffers of stage_bytes(n, esize), 128-byte
// aligned; mbar: two mbarriers; tmem: this CTA's TMEM base (kTmemCols).
// Returns false (K untouched) if a wait ran out.  Ends with a barrier.
template <int NT, bool kBF16>
__device__ bool syrk_gwg_tc(float* K, int ldk, const float* qd, const float* G, int ldg,
                            const float* W, const int* rows, int nrows, int n, char* stage,
                            uint64_t* mbar, uint32_t tmem, int* flag) {
  constexpr int esize = kBF16 ? 2 : 4;
  constexpr int per16 = 16 / esize;    // K values per 16-byte core-matrix row
  constexpr int kslabs = kKc / per16;  // 16-byte K slabs per chunk
  const int tid = threadIdx.x;
  const int tiles = tiles_for(n);
  const int npad = 128 * tiles;
  const int NG = npad / 8;
  const uint32_t slab = (uint32_t)NG * 128u;
  const uint32_t bufb = (uint32_t)kslabs * slab;
  const int nchunks = (nrows + kKc - 1) / kKc;
  if (tid == 0) {
    *flag = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int issued = 0;  // chunks whose MMAs were committed
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    char* buf = stage + b * bufb;
    // buffer b is free once the MMAs of chunk c - 2 (its latest commit) are done
    if (c >= 2 && !mbar_wait(&mbar[b], (uint32_t)(((c - 2) >> 1) & 1))) atomicOr(flag, 1);
    if (__syncthreads_or(*flag)) break;
    // stage chunk c: item (i, j) = row i of G_hat' (variable i), K slab j
    for (int it = tid; it < npad * kslabs; it += NT) {
      const int i = it % npad, j = it / npad;
      float v[per16];
#pragma unroll
      for (int u = 0; u < per16; ++u) {
        const int kk = c * kKc + j * per16 + u;
        float x = 0.f;
        if (i < n && kk < nrows) {
          const int r = rows[kk];
          x = sqrtf(W[r]) * G[r * ldg + i];
        }
        v[u] = x;
      }
      uint4 word;
      if (kBF16) {
        uint32_t w2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
          w2[u] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        word = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      } else {
        word = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
      }
      *reinterpret_cast<uint4*>(buf + j * slab + (i >> 3) * 128 + (i & 7) * 16) = word;
    }
    fence_async_smem();  // the tensor cores read shared memory through the async proxy
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
      const uint32_t base = smem_u32(buf);
      for (int s = 0; s < kslabs / 2; ++s) {
        for (int t = 0; t < tiles; ++t) {
          const uint32_t N = 128u * (uint32_t)(t + 1);
          const uint32_t col0 = t == 0 ? 0u : 128u;
          const uint64_t ad = smem_desc(base + 2u * s * slab + (uint32_t)t * 2048u, slab, 128u);
          const uint64_t bd = smem_desc(base + 2u * s * slab, slab, 128u);
          mma<kBF16>(tmem + col0, ad, bd, instr_desc(kBF16 ? 1u : 2u, N),
                     (c > 0 || s > 0) ? 1u : 0u);
        }
      }
      commit(&mbar[b]);
    }
    issued = c + 1;
  }
  // wait (bounded, also after a failure) for everything committed: the latest
  // commit of each buffer, chunks issued - 1 and issued - 2
  if (issued >= 1 && !mbar_wait(&mbar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1)))
    atomicOr(flag, 1);
  if (issued >= 2 && !mbar_wait(&mbar[(issued - 2) & 1], (uint32_t)(((issued - 2) >> 1) & 1)))
    atomicOr(flag, 1);
  const bool ok = __syncthreads_or(*flag) == 0;
  fence_after_sync();
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and a quarter of the columns
    const int w = tid >> 5, lane = tid & 31;
    const int lq = w & 3, cg = w >> 2;
    constexpr int ncg = NT / 128;  // warps per lane quarter
    for (int t = 0; t < tiles; ++t) {
      const int N = 128 * (t + 1);
      const uint32_t col0 = t == 0 ? 0u : 128u;
      const int i = 128 * t + 32 * lq + lane;
      for (int j0 = cg * 8; j0 < N; j0 += 8 * ncg) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + col0 + (uint32_t)j0, v);
        tmem_ld_wait();
        if (nchunks == 0) {
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int j = j0 + k;
          if (i < n && j <= i) K[i * ldk + j] = (j == i ? qd[i] : K[j * ldk + i]) + v[k];
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  return ok;
}

}  // namespace tc
}  // namespace qpgpu
