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

#ifdef __cplusplus
}
#endif

#endif /* MQCT_PROBE_H */
