/*
 * qp_probe.h -- measurement aid of libqpgpu (no counterpart in the paper):
 * the FP32 FMA throughput of the device, which bounds the on-chip solve
 * kernels (their roofline is the FP32 pipe, not HBM or the tensor cores).
 */
#ifndef QPGPU_QP_PROBE_H
#define QPGPU_QP_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueue an FMA loop on `stream`: `blocks` CTAs of `threads` threads, each
 * thread running 8 independent FP32 fused multiply-add chains for `iters`
 * rounds, so the launch performs blocks * threads * iters * 8 FMA
 * (2 FLOP each).  `out` (device, blocks * threads floats) receives each
 * thread's result so that no work is optimised away.  Time the launch with
 * CUDA events around it.  Returns QP_OK (0), QP_EINVAL (-1) for a null `out`,
 * non-positive sizes or threads > 1024, or QP_ECUDA (-3). */
int qp_fma_probe(int32_t blocks, int32_t threads, int32_t iters, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QPGPU_QP_PROBE_H */
