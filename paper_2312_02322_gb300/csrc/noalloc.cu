// mqct_propagate_noalloc: the FP64 persistent trajectory launch without any allocation.
//
// Some callers cannot allocate GPU memory while they run us: a host framework that
// owns a fixed memory pool and forbids cudaMalloc / cudaFree after start-up, a real-time
// or embedded loop where allocation latency and fragmentation are not acceptable, or a
// process that must not make the driver's pool grow.  mqct_propagate needs a little
// scratch memory (the device work-queue counter and the array of system views), which it
// takes with stream-ordered allocation.  This entry point takes that scratch from one
// file-scope device array instead, so it allocates nothing.  The caller still passes its
// own device buffers for every input and output.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace mqct {

// Scratch of every mqct_propagate_noalloc call on a device: the work-queue counter in the
// first 256 bytes, then the system views.  Every GPU that loads the library holds it until
// the process exits.
constexpr int kNoallocMaxSystems = 16;
constexpr size_t kNoallocQueueBytes = 256;
constexpr size_t kNoallocBytes = kNoallocQueueBytes + sizeof(DevSys) * kNoallocMaxSystems;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// One launch writes the system views into the scratch array and clears the work counter: the
// views travel by value in the launch's parameter block, so the call stages nothing in host
// memory and needs no copy from a host buffer that might be gone before the copy runs.
struct NoallocViews {
    DevSys v[kNoallocMaxSystems];
};
static_assert(sizeof(NoallocViews) <= 30000, "system views exceed the kernel parameter space");

__global__ void k_noalloc_setup(NoallocViews views, int n_systems, DevSys *dst, int *queue)
{
    const int i = threadIdx.x;
    if (i < n_systems) dst[i] = views.v[i];
    if (i == 0) *queue = 0;  // the counter keeps the previous call's value
}

namespace {

// The array's name is a host-side stand-in for it; its device address is looked up with the
// device current, the first time a call runs in a CUDA context (the primary context of a device
// unless the caller made another current).  The cache is keyed by the context's unique id, so a
// context created after cudaDeviceReset (whose module load may place the array elsewhere) gets a
// fresh lookup instead of the old address.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void *addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

cudaError_t current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    return cudaSuccess;
}

cudaError_t scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    ScratchAddr &c = g_scratch_addr[dev];
    if (!c.addr || c.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        c.addr = p;
        c.ctx_id = id;
    }
    *out = static_cast<unsigned char *>(c.addr);
    return cudaSuccess;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_propagate_noalloc(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs,
                                              int32_t n, double *final_pop, double *final_amp, mqct_diag *diag,
                                              void *cuda_stream)
{
    reset_launches();
    if (!systems || n_systems < 1) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: no systems");
    if (n_systems > kNoallocMaxSystems)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: more than 16 systems (size of its static scratch)");
    if (n < 0) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: n < 0");
    int nmax = 0, maxlev = 0, max_slices = 0;
    for (int i = 0; i < n_systems; ++i) {
        if (!systems[i]) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: NULL system");
        const DevSys &h = systems[i]->s.h;
        if (h.precision != MQCT_FP64)
            return fail(MQCT_ERR_UNSUPPORTED, "mqct_propagate_noalloc: FP64 systems only");
        if (i > 0 && h.path != systems[0]->s.h.path)
            return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: systems differ in path");
        nmax = std::max(nmax, h.n);
        maxlev = std::max(maxlev, h.n_levels);
        max_slices = std::max(max_slices, h.n_slices);
    }
    if (n == 0) return MQCT_OK;
    if (!trajs || !on_device(trajs)) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: trajs must be device memory");
    if ((final_pop && !on_device(final_pop)) || (final_amp && !on_device(final_amp)) || (diag && !on_device(diag)))
        return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate_noalloc: outputs must be device memory (or NULL)");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char *scratch = nullptr;
    if ((e = scratch_address(dev, &scratch)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
    int *queue = reinterpret_cast<int *>(scratch);
    DevSys *dsys = reinterpret_cast<DevSys *>(scratch + kNoallocQueueBytes);
    NoallocViews views;
    for (int i = 0; i < n_systems; ++i) views.v[i] = systems[i]->s.h;
    k_noalloc_setup<<<1, 32, 0, st>>>(views, n_systems, dsys, queue);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_noalloc_setup launch");

    const int maxw = kPropThreads / 32;
    const int per = (max_slices + maxw - 1) / maxw;
    const int nwarps = std::max(4, std::min(maxw, (max_slices + per - 1) / per));
    const int threads = nwarps * 32;
    bool adapt = false;
    for (int i = 0; i < n_systems; ++i) adapt |= systems[i]->s.h.adapt_tol > 0.0;
    const size_t smem = sizeof(double2) * ((adapt ? 8 : 6) * (size_t)nmax + 2 * (size_t)maxlev);
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaFuncSetAttribute(k_propagate_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute (basis too large for shared memory)");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate_fp64, threads, smem)) != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(MQCT_ERR_UNSUPPORTED, "mqct_propagate_noalloc: kernel does not fit on an SM");
    PropArgs pa{};
    pa.sys = dsys; pa.trajs = trajs; pa.order = nullptr; pa.n = n; pa.n_systems = n_systems; pa.queue = queue;
    pa.pop = final_pop; pa.amp = final_amp; pa.diag = diag; pa.nmax = nmax; pa.smem_n = nmax; pa.smem_lev = maxlev;
    pa.adapt = adapt ? 1 : 0;
    k_propagate_fp64<<<std::min(n, sms * per_sm), threads, smem, st>>>(pa);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_propagate_fp64 launch");
    return MQCT_OK;
}
