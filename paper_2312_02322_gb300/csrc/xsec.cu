// Cross sections from final populations (Sec. II): the final |a|^2 are summed over the
// states of each final level, weighted per trajectory (impact-parameter quadrature and the
// average over initial degenerate states) and summed over the trajectories of a group.
// Two deterministic passes: per-trajectory level sums, then one thread per (group, level)
// summing over trajectories in index order.
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace mqct {

// one warp per trajectory: Q[t][l] = weight[t] * sum_{s in l} pop[t][s]
__global__ void k_level_sums(const DevSys *sys, const double *pop, const double *weight, int n, double *Q)
{
    extern __shared__ double acc[];
    const DevSys &S = *sys;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *my = acc + (size_t)warp * S.n_levels;
    for (int t = blockIdx.x * warps + warp; t < n; t += gridDim.x * warps) {
        for (int l = lane; l < S.n_levels; l += 32) my[l] = 0.0;
        __syncwarp();
        // serial per level keeps the order fixed: lane l owns level l
        for (int s = 0; s < S.n; ++s) {
            const int l = S.lev[S.inv[s]];
            if ((l & 31) == lane) my[l] += pop[(size_t)t * S.n + s];
        }
        __syncwarp();
        const double w = weight[t];
        for (int l = lane; l < S.n_levels; l += 32) Q[(size_t)t * S.n_levels + l] = w * my[l];
        __syncwarp();
    }
}

__global__ void k_group_sums(const double *Q, const int *group, int n, int n_groups, int n_levels, double *sigma)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_groups * n_levels) return;
    const int g = i / n_levels, l = i % n_levels;
    double s = 0.0;
    for (int t = 0; t < n; ++t)
        if (group[t] == g) s += Q[(size_t)t * n_levels + l];
    sigma[i] = s;
}

}  // namespace mqct

using namespace mqct;

namespace {
bool is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" mqct_status mqct_cross_sections(mqct_system sys, const double *final_pop, const double *weight,
                                           const int32_t *group, int32_t n, int32_t n_groups, double *sigma_out,
                                           void *cuda_stream)
{
    reset_launches();
    if (!sys || !sigma_out) return fail(MQCT_ERR_INVALID_ARG, "mqct_cross_sections: NULL argument");
    if (n < 0 || n_groups < 0) return fail(MQCT_ERR_INVALID_ARG, "mqct_cross_sections: negative size");
    if (n > 0 && (!final_pop || !weight || !group)) return fail(MQCT_ERR_INVALID_ARG, "mqct_cross_sections: NULL input");
    if (n_groups == 0) return MQCT_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const DevSys &h = sys->s.h;
    const int N = h.n, NL = h.n_levels;
    cudaError_t e;
    std::vector<void *> tmp;
    auto get = [&](void **p, size_t b) {
        cudaError_t r = cudaMallocAsync(p, b ? b : 16, st);
        if (r == cudaSuccess) tmp.push_back(*p);
        return r;
    };
    auto cleanup = [&]() { for (void *p : tmp) cudaFreeAsync(p, st); };
    const double *dpop = final_pop, *dw = weight;
    const int *dg = group;
    double *dsig = sigma_out, *Q = nullptr;
    const bool host_out = !is_dev(sigma_out);
    if ((e = get((void **)&Q, sizeof(double) * (size_t)(n > 0 ? n : 1) * NL)) != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaMallocAsync"); }
    if (n > 0 && !is_dev(final_pop)) {
        double *p;
        if ((e = get((void **)&p, sizeof(double) * (size_t)n * N)) != cudaSuccess ||
            (e = cudaMemcpyAsync(p, final_pop, sizeof(double) * (size_t)n * N, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "staging final_pop");
        }
        dpop = p;
    }
    if (n > 0 && !is_dev(weight)) {
        double *p;
        if ((e = get((void **)&p, sizeof(double) * (size_t)n)) != cudaSuccess ||
            (e = cudaMemcpyAsync(p, weight, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "staging weight");
        }
        dw = p;
    }
    if (n > 0 && !is_dev(group)) {
        int *p;
        if ((e = get((void **)&p, sizeof(int) * (size_t)n)) != cudaSuccess ||
            (e = cudaMemcpyAsync(p, group, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "staging group");
        }
        dg = p;
    }
    if (host_out && (e = get((void **)&dsig, sizeof(double) * (size_t)n_groups * NL)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync");
    }
    if (n > 0) {
        const int threads = 256, warps = threads / 32;
        const size_t smem = sizeof(double) * warps * NL;
        if (smem > 48 * 1024) {
            cleanup();
            return fail(MQCT_ERR_UNSUPPORTED, "mqct_cross_sections: too many levels");
        }
        int blocks = (n + warps - 1) / warps;
        if (blocks > 4096) blocks = 4096;
        k_level_sums<<<blocks, threads, smem, st>>>(sys->s.d, dpop, dw, n, Q);
    }
    k_group_sums<<<(n_groups * NL + 127) / 128, 128, 0, st>>>(Q, dg, n, n_groups, NL, dsig);
    count_launches(n > 0 ? 2 : 1);
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_fail(e, "cross-section kernels"); }
    if (host_out) {
        if ((e = cudaMemcpyAsync(sigma_out, dsig, sizeof(double) * (size_t)n_groups * NL, cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "cudaMemcpyAsync");
        }
        cleanup();
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        return MQCT_OK;
    }
    cleanup();
    return MQCT_OK;
}
