/*
 * mqct_probe.h -- arithmetic-throughput probes of the GPU the library runs on.
 *
 * Not part of the paper's method: the roofline of the FP64 trajectory kernels is the
 * FP64 fused-multiply-add rate, which the measured-peaks file of the machine does not
 * hold, so the library measures it.  Each probe launches independent FMA chains on every
 * SM, times them with CUDA events on `cuda_stream`, synchronises, and writes the rate in
 * GFLOP/s (2 flops per FMA) to *gflops (host pointer).
 *   kind 0: FP64 FMA (DFMA)     kind 1: FP32 FMA (FFMA)
 * Errors: MQCT_ERR_INVALID_ARG (unknown kind, NULL output), MQCT_ERR_CUDA.
 */
#ifndef MQCT_PROBE_H
#define MQCT_PROBE_H

#include "mqct.h"

#ifdef __cplusplus
extern "C" {
#endif

mqct_status mqct_probe_fma_rate(int32_t kind, double *gflops, void *cuda_stream);

/* Latency of one operation in a dependent chain, in SM clock cycles per operation, with `warps`
 * warps (1..32) of one CTA each running its own chain (the slowest warp is reported):
 *   kind 0: FP64 FMA   kind 1: FP32 FMA   kind 2: FP64 division (plus one FP64 add)
 *   kind 3: FP64 -> FP32 conversion, FP32 multiply, FP32 -> FP64 conversion.
 * It shows how the FP64 work of a kernel serialises on this GPU (one FP64 warp instruction holds
 * its sub-partition's FP64 pipe for tens of cycles whatever the number of active lanes).
 * Synchronises `cuda_stream`; *cycles is a host pointer.
 * Errors: MQCT_ERR_INVALID_ARG, MQCT_ERR_CUDA. */
mqct_status mqct_probe_op_latency(int32_t kind, int32_t warps, double *cycles, void *cuda_stream);

/* Check of the library's 5th-generation tensor-core path (tcgen05 MMA, tensor-memory
 * accumulator, shared-memory operand descriptors): D = A * B^T on one CTA.
 *   a [128][k] BF16, b [n][k] BF16, d [128][n] FP32 -- all DEVICE pointers, row-major;
 *   16 <= n, k <= 256, multiples of 16.  Synchronises `cuda_stream`.
 * Errors: MQCT_ERR_INVALID_ARG, MQCT_ERR_TIMEOUT (the bounded completion wait ran out),
 * MQCT_ERR_CUDA.  No counterpart in the paper (a building-block check). */
mqct_status mqct_probe_tc_gemm(int32_t n, int32_t k, const void *a, const void *b, float *d, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MQCT_PROBE_H */
