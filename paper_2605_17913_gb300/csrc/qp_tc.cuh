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

// arrive on an mbarrier (count 1) announcing `bytes` of bulk-copy transactions
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// one-dimensional bulk copy (TMA engine) global -> this CTA's shared memory,
// completing `bytes` transactions on `bar`; both addresses 16-byte aligned,
// bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// order this thread's earlier generic-proxy writes to global memory before
// later reads of the same memory by the async proxy (bulk copies)
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
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
// aligned; mbar: two mbarriers initialised once per CTA (count 1) and used
// only here; *chunks: the chunks this CTA has committed through them so far
// (the phase parity of each barrier follows from it; updated here); tmem:
// this CTA's TMEM base (kTmemCols).  Returns false (K untouched) if a wait
// ran out.  Ends with a barrier.
template <int NT, bool kBF16>
__device__ bool syrk_gwg_tc(float* K, int ldk, const float* qd, const float* G, int ldg,
                            const float* W, const int* rows, int nrows, int n, char* stage,
                            uint64_t* mbar, uint32_t* chunks, uint32_t tmem, int* flag) {
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
  // chunk g (counted over the CTA's calls) uses buffer g & 1 and is that
  // buffer's (g >> 1)-th commit, completing its barrier's phase of parity
  // (g >> 1) & 1; every call waits for all of its commits before returning
  const uint32_t g0 = *chunks;
  if (tid == 0) *flag = 0;
  __syncthreads();
  int issued = 0;  // chunks whose MMAs were committed
  for (int c = 0; c < nchunks; ++c) {
    const uint32_t g = g0 + (uint32_t)c;
    const int b = (int)(g & 1u);
    char* buf = stage + b * bufb;
    // buffer b is free once the MMAs of chunk g - 2 (its latest commit) are done
    if (g >= 2 && !mbar_wait(&mbar[b], ((g - 2) >> 1) & 1u)) atomicOr(flag, 1);
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
  // commit of each buffer, chunks g0 + issued - 1 and g0 + issued - 2
  for (int k = 1; k <= 2 && k <= issued; ++k) {
    const uint32_t g = g0 + (uint32_t)(issued - k);
    if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) atomicOr(flag, 1);
  }
  const bool ok = __syncthreads_or(*flag) == 0;
  if (tid == 0) *chunks = g0 + (uint32_t)issued;
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
        float base[8];  // read before any store (a store may alias a later load)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int j = j0 + k;
          base[k] = (i < n && j <= i) ? (j == i ? qd[i] : K[j * ldk + i]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int j = j0 + k;
          if (i < n && j <= i) K[i * ldk + j] = base[k] + v[k];
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------
// K (lower triangle, stride ldk) = Q + sum over rows[0 .. nrows) of
// W[r] G[r]' G[r] in FP32 on the CUDA cores, for G in global memory (the
// large variant).  The listed rows are gathered kKc at a time into shared
// memory by one-dimensional bulk copies (the TMA engine; one copy per row of
// round4(n) floats -- G's pad columns are zero), two buffers alternating, so
// the next chunk streams in while the current one is multiplied; each arrived
// row is scaled by sqrt(W) once.  Each thread
// keeps the same 4 x 4 tiles of K for every chunk and adds the chunk's
// partial sums to them (the first chunk starts from Q), so K needs no
// barrier between chunks.  stage: two buffers of kKc * round4(n) floats,
// 16-byte aligned; mbar: two mbarriers initialised once per CTA (count 1) and
// used only here, *chunks the copies' chunk count so far (phase parity; updated
// here).  G must not have been written by this CTA since its last
// fence_async_global.  Returns false if a wait ran out (K then holds a
// partial sum; the caller recomputes it); *fail is set if copies may still be
// in flight after the bounded final waits.  Ends with a barrier.
// ---------------------------------------------------------------------------
template <int NT>
__device__ bool syrk_gwg_staged(float* K, int ldk, const float* qd, const float* G, int ldg,
                                const float* W, const int* rows, int nrows, int n, float* stage,
                                uint64_t* mbar, uint32_t* chunks, int* flag, int* fail,
                                unsigned long long* sub = nullptr) {
  const int tid = threadIdx.x;
  const int rowf = round4(n);
  const uint32_t rowb = (uint32_t)rowf * 4u;
  const int nt = (n + 3) >> 2;
  const int T = nt * (nt + 1) / 2;
  const int nchunks = (nrows + kKc - 1) / kKc;
  const uint32_t g0 = *chunks;
  if (tid == 0) *flag = 0;
  __syncthreads();
  // chunk g (counted over the CTA's calls) goes to buffer g & 1 and completes
  // that buffer's barrier phase of parity (g >> 1) & 1
  auto issue = [&](int c) {
    const uint32_t g = g0 + (uint32_t)c;
    float* buf = stage + (size_t)(g & 1u) * kKc * rowf;
    const int k0 = c * kKc, kn = min(kKc, nrows - k0);
    mbar_expect_tx(&mbar[g & 1u], (uint32_t)kn * rowb);
    for (int k = 0; k < kn; ++k)
      bulk_g2s(buf + k * rowf, G + (size_t)rows[k0 + k] * ldg, rowb, &mbar[g & 1u]);
  };
  if (tid == 0) {
    for (int c = 0; c < 2 && c < nchunks; ++c) issue(c);
  }
  int done = 0;  // chunks consumed
  for (int c = 0; c < nchunks; ++c) {
    const uint32_t g = g0 + (uint32_t)c;
    const long long ts0 = sub ? clock64() : 0;
    if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) atomicOr(flag, 1);
    if (__syncthreads_or(*flag)) break;
    const long long ts1 = sub ? clock64() : 0;
    float* const buf = stage + (size_t)(g & 1u) * kKc * rowf;
    const int k0 = c * kKc, kn = min(kKc, nrows - k0);
    // scale the chunk's rows by sqrt(W) once (W <= tau on the inactive rows),
    // so the products below need no per-row weight
    for (int e = tid; e < kn * rowf; e += NT) {
      const int k = e / rowf;
      buf[e] *= sqrtf(W[rows[k0 + k]]);
    }
    __syncthreads();
    const long long ts2 = sub ? clock64() : 0;
    for (int t = tid; t < T; t += NT) {
      const float x8 = 8.0f * (float)t + 1.0f;
      int I = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
      while ((I + 1) * (I + 2) / 2 <= t) ++I;
      while (I * (I + 1) / 2 > t) --I;
      const int J = t - I * (I + 1) / 2;
      // the tile's current values, read first: Q on the first chunk, else
      // the partial sum so far (read before any store, and early, so that
      // their latency overlaps the products)
      float old[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = 4 * I + a, j = 4 * J + b;
          old[a][b] = (i < n && j <= i)
                          ? (c != 0 ? K[i * ldk + j] : (j == i ? qd[i] : K[j * ldk + i]))
                          : 0.f;
        }
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
      for (int k = 0; k < kn; ++k) {
        const float4 u = *reinterpret_cast<const float4*>(buf + k * rowf + 4 * I);
        const float4 v = *reinterpret_cast<const float4*>(buf + k * rowf + 4 * J);
        const float aw[4] = {u.x, u.y, u.z, u.w};
        const float cv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(aw[a], cv[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = 4 * I + a, j = 4 * J + b;
          if (i < n && j <= i) K[i * ldk + j] = old[a][b] + acc[a][b];
        }
    }
    done = c + 1;
    // every thread is done with this buffer, whose generic-proxy writes (the
    // scaling) must be ordered before the bulk copy that refills it
    fence_async_smem();
    __syncthreads();
    if (sub && tid == 0) {
      // tracing builds: waiting for the copies, scaling, products
      atomicAdd(&sub[0], (unsigned long long)(ts1 - ts0));
      atomicAdd(&sub[1], (unsigned long long)(ts2 - ts1));
      atomicAdd(&sub[2], (unsigned long long)(clock64() - ts2));
    }
    if (tid == 0 && c + 2 < nchunks) issue(c + 2);
  }
  if (nchunks == 0) {
    // no inactive rows: K = Q
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e - i * n;
      if (j <= i) K[i * ldk + j] = j == i ? qd[i] : K[j * ldk + i];
    }
  }
  // after a failure: wait (bounded) for the copies already issued, chunks
  // done .. min(done + 2, nchunks) - 1
  int bad = 0;
  if (tid == 0) {
    for (int c = done; c < nchunks && c < done + 2; ++c) {
      const uint32_t g = g0 + (uint32_t)c;
      if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) bad = 1;
    }
    if (bad) *fail = 1;
    *chunks = g0 + (uint32_t)min(nchunks, done + 2);
  }
  const bool ok = __syncthreads_or(*flag) == 0;
  return ok;
}

// ---------------------------------------------------------------------------
// The same sum with each thread's share of K held in registers across all
// chunks (NT = 512): thread t owns the 8 x 8 block t of K's lower triangle
// (blocks numbered row by row; diagonal blocks computed whole and stored
// below the diagonal), starts it from Q, adds every chunk's rows to it and
// stores it once.  Per row of a chunk that is 4 shared-memory vector loads
// per 64 FMAs, and K is read and written once per call instead of once per
// chunk.  Up to n = 248 there are at most 496 blocks (one per thread, the
// rest idle); at n = 256 (528 blocks) the last 16 blocks are dealt out as 512
// pairs of adjacent elements, one more per thread.  Stage rows have stride
// rs = round8(n) (the bulk copy fills round4(n) floats; the columns beyond n
// only feed sums that are never stored).  When a chunk has landed, the
// scaling pass also reorders each row in place so that columns 8J..8J+3 sit
// at 4J and 8J+4..8J+7 at rs/2 + 4J: consecutive blocks then read
// consecutive 16-byte words (no bank conflicts).  Same contract as
// syrk_gwg_staged.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __noinline__ bool syrk_gwg_staged_blocks(float* K, int ldk, const float* qd,
                                                    const float* G, int ldg, const float* W,
                                                    const int* rows, int nrows, int n,
                                                    float* stage, uint64_t* mbar,
                                                    uint32_t* chunks, int* flag, int* fail,
                                                    unsigned long long* sub = nullptr) {
  static_assert(NT == 512, "one 8 x 8 block per thread needs 512 threads up to n = 256");
  const int tid = threadIdx.x;
  const int rowf = round4(n);          // floats copied per row
  const int rs = (n + 7) & ~7;         // row stride of the stage buffers
  const uint32_t rowb = (uint32_t)rowf * 4u;
  const int n8 = rs >> 3;
  const int U = n8 * (n8 + 1) / 2;     // 8 x 8 blocks of the lower triangle
  const int E2 = U > NT ? (U - NT) * 32 : 0;  // element pairs of the blocks beyond NT
  const int nchunks = (nrows + kKc - 1) / kKc;
  const uint32_t g0 = *chunks;
  // this thread's block (I, J), J <= I
  const bool has_blk = tid < U && tid < NT;
  int I = 0, J = 0;
  if (has_blk) {
    const float x8 = 8.0f * (float)tid + 1.0f;
    I = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= tid) ++I;
    while (I * (I + 1) / 2 > tid) --I;
    J = tid - I * (I + 1) / 2;
  }
  // this thread's extra element pair (i, j), (i, j + 1) of a block beyond NT
  const bool has_pair = tid < E2;
  int ie = 0, je = 0;
  if (has_pair) {
    const int u = NT + tid / 32, loc = tid & 31;
    const float x8 = 8.0f * (float)u + 1.0f;
    int Iu = (int)((x8 * rsqrtf(x8) - 1.0f) * 0.5f);
    while ((Iu + 1) * (Iu + 2) / 2 <= u) ++Iu;
    while (Iu * (Iu + 1) / 2 > u) --Iu;
    const int Ju = u - Iu * (Iu + 1) / 2;
    ie = 8 * Iu + (loc >> 2);
    je = 8 * Ju + ((loc & 3) << 1);
  }
  const long long tp0 = sub ? clock64() : 0;
  if (tid == 0) *flag = 0;
  __syncthreads();
  auto issue = [&](int c) {
    const uint32_t g = g0 + (uint32_t)c;
    float* buf = stage + (size_t)(g & 1u) * kKc * rs;
    const int k0 = c * kKc, kn = min(kKc, nrows - k0);
    mbar_expect_tx(&mbar[g & 1u], (uint32_t)kn * rowb);
    for (int k = 0; k < kn; ++k)
      bulk_g2s(buf + k * rs, G + (size_t)rows[k0 + k] * ldg, rowb, &mbar[g & 1u]);
  };
  if (tid == 0) {
    for (int c = 0; c < 2 && c < nchunks; ++c) issue(c);
  }
  // the running sums start from Q: its strict lower triangle is K's upper
  // triangle (read transposed), its diagonal qd
  float acc[8][8];
  // whole off-diagonal blocks of 16-byte aligned rows move as float4 rows
  const bool vec = has_blk && J < I && 8 * I + 8 <= n && (ldk & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(K) & 15) == 0;
  if (vec) {
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float* q = K + (8 * J + b) * ldk + 8 * I;
      const float4 q0 = *reinterpret_cast<const float4*>(q);
      const float4 q1 = *reinterpret_cast<const float4*>(q + 4);
      acc[0][b] = q0.x; acc[1][b] = q0.y; acc[2][b] = q0.z; acc[3][b] = q0.w;
      acc[4][b] = q1.x; acc[5][b] = q1.y; acc[6][b] = q1.z; acc[7][b] = q1.w;
    }
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int i = 8 * I + a, j = 8 * J + b;
        acc[a][b] = (has_blk && i < n && j <= i) ? (j == i ? qd[i] : K[j * ldk + i]) : 0.f;
      }
  }
  float ex0 = 0.f, ex1 = 0.f;
  if (has_pair) {
    if (ie < n && je <= ie) ex0 = je == ie ? qd[ie] : K[je * ldk + ie];
    if (ie < n && je + 1 <= ie) ex1 = je + 1 == ie ? qd[ie] : K[(je + 1) * ldk + ie];
  }
  int done = 0;  // chunks consumed
  if (sub && tid == 0) atomicAdd(&sub[3], (unsigned long long)(clock64() - tp0));
  for (int c = 0; c < nchunks; ++c) {
    const uint32_t g = g0 + (uint32_t)c;
    const long long ts0 = sub ? clock64() : 0;
    if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) atomicOr(flag, 1);
    if (__syncthreads_or(*flag)) break;
    const long long ts1 = sub ? clock64() : 0;
    float* const buf = stage + (size_t)(g & 1u) * kKc * rs;
    const int k0 = c * kKc, kn = min(kKc, nrows - k0);
    // scale the chunk's rows by sqrt(W) once (W <= tau on the inactive rows)
    // and reorder them: read every 8-column group, then (after the barrier)
    // write its halves to 4J and rs/2 + 4J.  At most kKc * 32 groups: two per
    // thread.
    {
      float4 ga[2], gb[2];
      int gk[2], gJ[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = tid + q * NT;
        gk[q] = -1;
        if (e < kn * n8) {
          const int k = e / n8, Jg = e - k * n8;
          const float sw = sqrtf(W[rows[k0 + k]]);
          const float4 x0 = *reinterpret_cast<const float4*>(buf + k * rs + 8 * Jg);
          const float4 x1 = *reinterpret_cast<const float4*>(buf + k * rs + 8 * Jg + 4);
          ga[q] = make_float4(x0.x * sw, x0.y * sw, x0.z * sw, x0.w * sw);
          gb[q] = make_float4(x1.x * sw, x1.y * sw, x1.z * sw, x1.w * sw);
          gk[q] = k;
          gJ[q] = Jg;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (gk[q] >= 0) {
          float* row = buf + gk[q] * rs;
          *reinterpret_cast<float4*>(row + 4 * gJ[q]) = ga[q];
          *reinterpret_cast<float4*>(row + (rs >> 1) + 4 * gJ[q]) = gb[q];
        }
      }
    }
    __syncthreads();
    const long long ts2 = sub ? clock64() : 0;
    if (has_blk) {
      const float* pu = buf + 4 * I;
      const float* pv = buf + 4 * J;
      const int h2 = rs >> 1;
#pragma unroll 2
      for (int k = 0; k < kn; ++k) {
        const float4 u0 = *reinterpret_cast<const float4*>(pu + k * rs);
        const float4 u1 = *reinterpret_cast<const float4*>(pu + k * rs + h2);
        const float4 v0 = *reinterpret_cast<const float4*>(pv + k * rs);
        const float4 v1 = *reinterpret_cast<const float4*>(pv + k * rs + h2);
        const float uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(uu[a], vv[b], acc[a][b]);
      }
    }
    if (has_pair) {
      // positions of columns ie and je, je + 1 in the reordered rows
      const int pi = ((ie & 4) ? (rs >> 1) : 0) + 4 * (ie >> 3) + (ie & 3);
      const int pj = ((je & 4) ? (rs >> 1) : 0) + 4 * (je >> 3) + (je & 3);
      for (int k = 0; k < kn; ++k) {
        const float ue = buf[k * rs + pi];
        const float2 ve = *reinterpret_cast<const float2*>(buf + k * rs + pj);
        ex0 = fmaf(ue, ve.x, ex0);
        ex1 = fmaf(ue, ve.y, ex1);
      }
    }
    done = c + 1;
    // every thread is done with this buffer, whose generic-proxy writes (the
    // scaling) must be ordered before the bulk copy that refills it
    fence_async_smem();
    __syncthreads();
    if (sub && tid == 0) {
      atomicAdd(&sub[0], (unsigned long long)(ts1 - ts0));
      atomicAdd(&sub[1], (unsigned long long)(ts2 - ts1));
      atomicAdd(&sub[2], (unsigned long long)(clock64() - ts2));
    }
    if (tid == 0 && c + 2 < nchunks) issue(c + 2);
  }
  const long long te0 = sub ? clock64() : 0;
  const bool ok = __syncthreads_or(*flag) == 0;
  if (ok) {
    // K's lower triangle (its upper triangle, Q, is read above and kept)
    if (vec) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float* k = K + (8 * I + a) * ldk + 8 * J;
        *reinterpret_cast<float4*>(k) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        *reinterpret_cast<float4*>(k + 4) =
            make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
      }
    } else if (has_blk) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int i = 8 * I + a, j = 8 * J + b;
          if (i < n && j <= i) K[i * ldk + j] = acc[a][b];
        }
    }
    if (has_pair) {
      if (ie < n && je <= ie) K[ie * ldk + je] = ex0;
      if (ie < n && je + 1 <= ie) K[ie * ldk + je + 1] = ex1;
    }
  }
  // after a failure: wait (bounded) for the copies already issued, chunks
  // done .. min(done + 2, nchunks) - 1
  int bad = 0;
  if (tid == 0) {
    for (int c = done; c < nchunks && c < done + 2; ++c) {
      const uint32_t g = g0 + (uint32_t)c;
      if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) bad = 1;
    }
    if (bad) *fail = 1;
    *chunks = g0 + (uint32_t)min(nchunks, done + 2);
  }
  __syncthreads();
  if (sub && tid == 0) atomicAdd(&sub[4], (unsigned long long)(clock64() - te0));
  return ok;
}

// ---------------------------------------------------------------------------
// Back substitution L' x_v = x_v (block_trsv's upper solve) for L in global
// memory (n x n lower, row stride ld: a multiple of 4 floats, rows 16-byte
// aligned) with each 32-row block staged in shared memory by bulk copies:
// block bk (rows j0 .. j0+jb) needs those rows' columns 0 .. j0+jb, one copy
// per row, issued two blocks ahead into two buffers (stage: 2 x 32 x sld
// floats, sld >= round4(n) a multiple of 4, 16-byte aligned) on the mbarriers
// mbar with the chunk count *chunks (shared with syrk_gwg_staged*).  Warp 0
// solves the block's diagonal part from shared memory, then every thread
// applies the block to one remaining entry.  L must not have been written by
// this CTA since its last fence_async_global, except by the calling threads
// just before the call (the call fences first).  A wait that runs out sets
// *flag and the rest of the solve reads L in global memory (same
// arithmetic); *fail is set if copies may still be in flight after the
// bounded final waits.  Returns whether every block was staged.  Ends with a
// barrier.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __noinline__ bool block_trsv_upper_staged(const float* L, int ld, const float* dinv,
                                                     int n, float* x0, float* x1, float* stage,
                                                     int sld, uint64_t* mbar, uint32_t* chunks,
                                                     int* flag, int* fail) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int nblk = (n + 31) >> 5;
  const uint32_t g0 = *chunks;
  if (tid == 0) *flag = 0;
  // the factor was stored through the generic proxy, and so were the stage
  // buffers' earlier contents: order both before the bulk copies
  fence_async_global();
  fence_async_smem();
  __syncthreads();
  auto issue = [&](int bk) {
    const uint32_t g = g0 + (uint32_t)bk;
    float* buf = stage + (size_t)(g & 1u) * 32 * sld;
    const int j0 = 32 * (nblk - 1 - bk), jb = min(32, n - j0);
    const uint32_t bytes = (uint32_t)round4(j0 + jb) * 4u;
    mbar_expect_tx(&mbar[g & 1u], (uint32_t)jb * bytes);
    for (int k = 0; k < jb; ++k) bulk_g2s(buf + k * sld, L + (size_t)(j0 + k) * ld, bytes, &mbar[g & 1u]);
  };
  if (tid == 0) {
    for (int bk = 0; bk < 2 && bk < nblk; ++bk) issue(bk);
  }
  int issued = min(2, nblk), done = 0;
  bool staged = true;
  for (int bk = 0; bk < nblk; ++bk) {
    const uint32_t g = g0 + (uint32_t)bk;
    const int j0 = 32 * (nblk - 1 - bk), jb = min(32, n - j0);
    if (staged) {
      if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) atomicOr(flag, 1);
      staged = __syncthreads_or(*flag) == 0;
      if (staged) done = bk + 1;
    }
    // row k of the block: src[k * sst + column]
    const float* src = staged ? stage + (size_t)(g & 1u) * 32 * sld : L + (size_t)j0 * ld;
    const int sst = staged ? sld : ld;
    if (tid < 32) {
      // lane l holds column l of the diagonal part: r[k] = L[j0+k][j0+l], k >= l
      float r[32];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        r[k] = (lane < jb && k < jb && k >= lane) ? src[k * sst + j0 + lane] : 0.f;
      float v0 = lane < jb ? x0[j0 + lane] : 0.f;
      float v1 = (x1 && lane < jb) ? x1[j0 + lane] : 0.f;
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) {
        const int k = 31 - kk;
        if (k < jb) {
          const float dk = dinv[j0 + k];
          const float s0 = __shfl_sync(kFull, v0 * dk, k);
          const float s1 = __shfl_sync(kFull, v1 * dk, k);
          if (lane == k) { v0 = s0; v1 = s1; }
          if (lane < k) {
            v0 = fmaf(-r[k], s0, v0);
            v1 = fmaf(-r[k], s1, v1);
          }
        }
      }
      if (lane < jb) {
        x0[j0 + lane] = v0;
        if (x1) x1[j0 + lane] = v1;
      }
    }
    __syncthreads();
    // the entries above the block: x_i -= sum_k L[j0+k][i] x_{j0+k}
    for (int i = tid; i < j0; i += NT) {
      float acc0 = x0[i], acc1 = x1 ? x1[i] : 0.f;
#pragma unroll 8
      for (int k = 0; k < jb; ++k) {
        const float l = src[k * sst + i];
        acc0 = fmaf(-l, x0[j0 + k], acc0);
        if (x1) acc1 = fmaf(-l, x1[j0 + k], acc1);
      }
      x0[i] = acc0;
      if (x1) x1[i] = acc1;
    }
    // this buffer is read (generic proxy) before the copy that refills it
    fence_async_smem();
    __syncthreads();
    if (staged && tid == 0 && bk + 2 < nblk) issue(bk + 2);
    if (staged && bk + 2 < nblk) issued = bk + 3;
  }
  // copies issued but not waited for (after a wait ran out): wait, bounded
  if (tid == 0) {
    int bad = 0;
    for (int bk = done; bk < issued; ++bk) {
      const uint32_t g = g0 + (uint32_t)bk;
      if (!mbar_wait(&mbar[g & 1u], (g >> 1) & 1u)) bad = 1;
    }
    if (bad) *fail = 1;
    *chunks = g0 + (uint32_t)issued;
  }
  __syncthreads();
  return done == nblk;
}

}  // namespace tc
}  // namespace qpgpu
