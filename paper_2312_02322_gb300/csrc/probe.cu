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

// dependent chains of one operation on `warps` warps of one CTA; each warp's lane 0 writes the
// clock cycles its chain took
template <int KIND>
__global__ void k_latency_probe(long long *cycles, int iters, double a, double b)
{
    double x = a + threadIdx.x * 1e-9;
    float xf = (float)x, bf = (float)b;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        if (KIND == 0) x = fma(x, b, 1e-7);         // FP64 fused multiply-add
        if (KIND == 1) xf = fmaf(xf, bf, 1e-7f);    // FP32 fused multiply-add
        if (KIND == 2) x = 1.0 / (x + 1.0);         // FP64 division (and one add)
        if (KIND == 3) x = (double)((float)x * bf);  // FP64 -> FP32, FP32 multiply, FP32 -> FP64
    }
    __syncwarp();
    const long long t1 = clock64();
    if ((threadIdx.x & 31) == 0) cycles[threadIdx.x >> 5] = t1 - t0;
    if (x == -1.2345 || xf == -1.2345f) cycles[63] = 0;  // keeps the chain alive; never true here
}

}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_probe_op_latency(int32_t kind, int32_t warps, double *cycles, void *cuda_stream)
{
    if (!cycles || kind < 0 || kind > 3 || warps < 1 || warps > 32)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_probe_op_latency: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    long long *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, 64 * sizeof(long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    const int iters = 2048;
    for (int rep = 0; rep < 2; ++rep) {  // the first run loads the module and warms the clocks
        switch (kind) {
            case 0: k_latency_probe<0><<<1, 32 * warps, 0, st>>>(d, iters, 1.0000001, 0.9999999); break;
            case 1: k_latency_probe<1><<<1, 32 * warps, 0, st>>>(d, iters, 1.0000001, 0.9999999); break;
            case 2: k_latency_probe<2><<<1, 32 * warps, 0, st>>>(d, iters, 1.0000001, 0.9999999); break;
            default: k_latency_probe<3><<<1, 32 * warps, 0, st>>>(d, iters, 1.0000001, 0.9999999); break;
        }
    }
    long long h[64] = {0};
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "latency probe");
    long long mx = 0;
    for (int w = 0; w < warps; ++w) mx = h[w] > mx ? h[w] : mx;
    *cycles = (double)mx / iters;
    return MQCT_OK;
}

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
