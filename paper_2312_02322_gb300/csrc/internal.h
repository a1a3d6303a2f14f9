// Internal layout shared by the host builder and the kernels of the MQCT library.
// Not part of the C ABI (see include/mqct.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mqct.h"

namespace mqct {

// four spline coefficients (c0..c3) of one interval, 32-byte aligned
struct alignas(32) dbl4 {
    double x, y, z, w;
};
inline __host__ __device__ dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

constexpr int kSlice = 32;     // rows per SELL slice (one warp)
constexpr int kMaxTerms = 64;  // expansion terms held in shared memory per stage
constexpr int kMaxWarps = 32;

// Device view of one system; an array of these lives in device memory so that one
// persistent launch can serve trajectories of several systems (uneven basis sizes).
// State indices are INTERNAL: states sorted by m-block (Eq. 6: M is block-diagonal in m),
// so that each block is contiguous; perm[] maps back to the caller's order.
struct DevSys {
    int n, n_levels, L, n_int, n_slices, P;
    int path, precision, flags;
    double mu, r_min, h, inv_h;
    int grid_log;              // splines in x = ln R (MQCT_GRID_LOG) instead of x = R
    double adapt_tol;          // > 0: adaptive step control (FP64 kernel)
    double adapt_hmax;         // largest adaptive step / dt
    double x0;                 // first knot in the spline variable (r_min or ln r_min)
    const double *lev_energy;  // [n_levels]
    const float *lev_energy_f; // [n_levels] FP32 copy (mixed-precision systems)
    const int *lev;            // [n]  level of each internal state
    const int *perm;           // [n]  internal -> caller index
    const int *inv;            // [n]  caller -> internal index
    const int *up, *dn;        // [n]  Coriolis partners m+1 / m-1 (self when absent)
    const double *aup, *adn;   // [n]  ladder factors (0 when absent or Coriolis off)
    const double *diag_g;      // [L][n] G^lambda_ss (initial mean-field energy)
    const dbl4 *vcoef;      // [L][n_int] spline coefficients of v_lambda (c0..c3)
    const dbl4 *dvcoef;     // [P][L][n_int] spline coefficients of dv_lambda/dtheta_p
    const float4 *dvcoef_f; // FP32 copy (mixed-precision systems with parameters)
    // PLAIN path: sliced-ELL (32-row slices) spline table of the non-zero M_nm(R)
    const int *sl_off;         // [n_slices+1] entry offsets (multiples of 32)
    const int *cols;           // [nnz_pad] internal column (padding: row itself, zero coefficients)
    const double2 *T01;        // [n_int][nnz_pad] (c0, c1)
    const double2 *T23;        // [n_int][nnz_pad] (c2, c3)
    const float4 *T4f;         // PLAIN + FP32: [n_int][nnz_pad] (c0, c1, c2, c3) of each element
    long long nnz_pad;
    // FACTORISED path: per stored term f (a lambda whose G is not the identity) a sliced-ELL
    // matrix; identity terms are applied directly (id_mask bit lambda).
    int n_f;
    unsigned long long id_mask;
    const int *f_term;         // [n_f] lambda of stored term f
    const int *f_sl_off;       // [n_f][n_slices+1] offsets into f_cols / f_val
    const int *f_cols;
    const double *f_val;
    const float *f_valf;       // FP32 copy of f_val (mixed-precision systems)
    const int2 *f_cvf;         // f_cols and f_valf interleaved: (column, FP32 value bits) per entry,
                               // one 8-byte load per entry (mixed-precision systems)
    // Batched mixed-precision paths: FP32 spline coefficients of v_lambda, ladder factors
    const float4 *vcoef_f;     // [L][n_int]
    const float *aupf, *adnf;  // [n] FP32 ladder factors
    // Tensor-core path (BF16X3): m-blocks packed into row tiles of <= 128 rows; for every
    // stored term f and tile t the 128 x 128 block-diagonal G^f tile as BF16 hi and lo parts in
    // the canonical K-major layout of the MMA A operand (tile-major: [f][t][hi,lo][16384]).
    int n_tiles;
    const int *tile_r0;        // [n_tiles + 1] first row of each tile
    const uint16_t *g_tiles;   // [n_f][n_tiles][2][128 * 128]
    const uint8_t *g_kmask;    // [n_f][n_tiles] bit ks set: K columns 16 ks .. 16 ks + 15 hold a non-zero
};

struct System {
    DevSys h;                  // host copy of the device view (pointers are device pointers)
    DevSys *d = nullptr;       // device copy
    std::vector<void *> allocs;
    mqct_system_info_t info{};
    // host copies needed by the host side of later calls
    std::vector<int> perm, inv, lev;
    int max_block = 0;
};

void set_error(const std::string &msg);
const char *last_error_cstr();

// arguments of the persistent FP64 launch (propagate.cu)
constexpr int kPropThreads = 512;  // upper bound of the block size (register budget)
struct PropArgs {
    const DevSys *sys;
    const mqct_traj *trajs;
    const int *order;  // work order (trajectory indices), or nullptr for the caller's order
    int n, n_systems;
    int *queue;        // work counter, zero at launch
    double *pop;
    double *amp;
    mqct_diag *diag;
    long long *t_start, *t_done;  // optional device clock (ns) at start / end of each trajectory
    int nmax;      // row stride of pop / amp
    int smem_n;    // shared-memory vector length (max n over systems)
    int smem_lev;  // max n_levels over systems
    int adapt;     // some system uses adaptive steps: two more vectors of smem_n in shared memory
};
#ifdef __CUDACC__
__global__ void __launch_bounds__(kPropThreads) k_propagate_fp64(PropArgs a);
// device clock in nanoseconds (the global timer every SM shares)
__device__ __forceinline__ long long mqct_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}
#endif

// arguments of the tensor-core launch sequence (tc_batched.cu): one system
struct BatchArgs {
    const DevSys *sys;
    const mqct_traj *trajs;
    const int *order;
    int n;
    int *queue;
    double *pop;
    double *amp;
    mqct_diag *diag;
    long long *t_start, *t_done;  // optional device clock (ns) at start / end of each trajectory
    int nmax;
    int sys_idx;   // trajectories must name this system
    int tc_slots;  // trajectories in flight (0 = automatic)
};

// arguments of the FP32 batched launch over one or several systems (batched.cu)
constexpr int kBatchMaxSystems = 16;
struct BatchMultiArgs {
    const DevSys *sys;            // [n_systems] device views
    const mqct_traj *trajs;
    const int *lists;             // [n_systems][n] work list of each system (trajectory indices, longest first)
    const int *counts;            // [n_systems] lengths of the lists, or nullptr (one system, length n)
    int *queues;                  // [n_systems] work counters, zero at launch
    const double *work;           // [n_systems] estimated work of each system, or nullptr
    int n, n_systems;
    int sys_base;                 // trajectories name system sys_base + s
    int slots[kBatchMaxSystems];  // slots per CTA of each system (set by run_batched)
    double *pop;
    double *amp;
    mqct_diag *diag;
    long long *t_start, *t_done;  // optional device clock (ns) at start / end of each trajectory
    int nmax;
};
// the (slots per CTA at most, threads) instances of the FP32 batched kernel; batched_auto_shape
// picks one from the trajectory count and the slots each shape gives the systems
constexpr int kBatchShapes[7][2] = {{32, 512}, {16, 512}, {8, 256}, {8, 512}, {4, 512}, {16, 256}, {4, 256}};
// the automatic shape index (0-based) for n trajectories over the systems hs; -1 if none fits
int batched_auto_shape(const std::vector<const DevSys *> &hs, int n, int sms);
// true when shape index i (0-based) fits the system's basis with at least four slots
bool batched_shape_fits(const DevSys &h, int i);
int batched_width(const DevSys &h);
// one persistent FP32 launch over the systems hs (device views a.sys; at most kBatchMaxSystems);
// shape 0 = automatic, else a kBatchShapes index + 1
cudaError_t run_batched(BatchMultiArgs a, const std::vector<const DevSys *> &hs, int shape, cudaStream_t st);
// stage-synchronous tensor-core launch sequence (tc_batched.cu); allocates its scratch with
// stream-ordered allocation and synchronises `st` between chunks of steps
mqct_status run_tc_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st);

mqct_status fail(mqct_status st, const std::string &msg);
mqct_status cuda_fail(cudaError_t e, const char *what);
// launches of this library's kernels made by the current C-ABI call on this thread
void reset_launches();
void count_launches(long long n);

// host helpers of the built-in system builders (diatom.cpp)
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
mqct_status finish_desc(mqct_system_desc *out, const char *who, const std::vector<double> &energy,
                        const std::vector<int32_t> &level, const std::vector<int32_t> &jq,
                        const std::vector<int32_t> &mq, double mu, int L, const std::vector<int32_t> &gt,
                        const std::vector<int32_t> &gr, const std::vector<int32_t> &gc, const std::vector<double> &gv,
                        const double *A, const double *beta, double c6, double rd, int ng, double r_min, double r_max,
                        bool with_params, int path, int precision, int grid_kind);

}  // namespace mqct

struct mqct_system_s {
    mqct::System s;
};
