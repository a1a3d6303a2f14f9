// FMA-throughput probes (include/mqct_probe.h): the denominators of the ALU rooflines.
#include <cuda_runtime.h>

#include "internal.h"
#include "mqct_probe.h"

namespace mqct {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <class T>
__global__ void k_fma_probe(T *out, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == (T)-1.2345) out[0] = s;  // keeps the chains alive; never true for these inputs
}

}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_probe_fma_rate(int32_t kind, double *gflops, void *cuda_stream)
{
    if (!gflops || (kind != 0 && kind != 1)) return fail(MQCT_ERR_INVALID_ARG, "mqct_probe_fma_rate: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, 16, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (kind == 0) k_fma_probe<double><<<blocks, threads, 0, st>>>((double *)out, 0.999999, 1e-7);
        else k_fma_probe<float><<<blocks, threads, 0, st>>>((float *)out, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess) return cuda_fail(e, "fma probe");
    double fmas = (double)blocks * threads * kChains * (double)kIters;
    *gflops = 2.0 * fmas / (best * 1e-3) * 1e-9;
    return MQCT_OK;
}
