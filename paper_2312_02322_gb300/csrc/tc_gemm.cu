// 5th-generation tensor-core (tcgen05) building blocks for sm_103a and a GEMM probe that
// checks them: D[128][N] = A[128][K] * B[N][K]^T, BF16 operands staged in shared memory in the
// canonical K-major layout without swizzle, FP32 accumulator in tensor memory (TMEM).
//
// Canonical K-major, no-swizzle layout: the operand is cut into core matrices of 8 rows x 16
// bytes (8 BF16 values of K); element (r, k) sits at
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2      bytes,
// here with LBO = 128 (K-adjacent core matrices contiguous) and SBO = 128 * K / 8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "mqct_probe.h"
#include "tc_ptx.cuh"

namespace mqct {

constexpr long long kTcWaitLimit = 1ll << 24;  // bounded mbarrier polls

__global__ void __launch_bounds__(128) k_tc_gemm_probe(int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *Bm,
                                                        float *D, int *status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kch = K / 8;
    unsigned char *sA = sm, *sB = sm + 128 * K * 2;
    for (int i = tid; i < 128 * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__nv_bfloat16 *>(sA + tc_kmajor_offset(r, k, kch)) = A[i];
    }
    for (int i = tid; i < N * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__nv_bfloat16 *>(sB + tc_kmajor_offset(r, k, kch)) = Bm[i];
    }
    tc_fence_proxy_async();
    const uint32_t ncols = tc_tmem_cols(N);
    if (warp == 0) {
        tc_tmem_alloc(&tmem_base, ncols);
        tc_tmem_relinquish();
    }
    if (tid == 0) tc_mbar_init(&mbar, 1);
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t taddr = tmem_base;
    if (tid == 0) {
        const uint32_t idesc = tc_idesc_bf16_f32(128, N);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc_sdesc(tc_smem_addr(sA) + ks * 256, 128, kch * 128);
            const uint64_t bd = tc_sdesc(tc_smem_addr(sB) + ks * 256, 128, kch * 128);
            tc_mma_bf16(taddr, ad, bd, idesc, ks > 0);
        }
        tc_commit(&mbar);
    }
    const bool ok = tc_mbar_wait(&mbar, 0, kTcWaitLimit);
    tc_fence_after_sync();
    if (!ok && tid == 0) atomicExch(status, 1);
    if (ok) {
        const int row = warp * 32 + lane;
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc_ld_32x32b_x8(taddr + ((uint32_t)(warp * 32) << 16) + c, v);
            tc_wait_ld();
            for (int j = 0; j < 8; ++j) D[row * N + c + j] = v[j];
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc_tmem_dealloc(taddr, ncols);
}

}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_probe_tc_gemm(int32_t n, int32_t k, const void *a, const void *b, float *d, void *cuda_stream)
{
    if (n < 16 || n > 256 || (n % 16) || k < 16 || k > 256 || (k % 16) || !a || !b || !d)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_probe_tc_gemm: need 16 <= n, k <= 256, multiples of 16, device pointers");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *status = nullptr;
    cudaError_t e = cudaMallocAsync(&status, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(status, 0, sizeof(int), st);
    const size_t smem = (size_t)(128 + n) * k * 2;
    cudaFuncSetAttribute(k_tc_gemm_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_gemm_probe<<<1, 128, smem, st>>>(n, k, (const __nv_bfloat16 *)a, (const __nv_bfloat16 *)b, d, status);
    e = cudaGetLastError();
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(status, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 probe");
    if (hs) return fail(MQCT_ERR_TIMEOUT, "mqct_probe_tc_gemm: the MMA completion wait ran out");
    return MQCT_OK;
}
