// Device helpers shared by the batched trajectory kernels (FP32 CUDA-core path, batched.cu, and
// BF16x3 tensor-core path, tc_batched.cu): phase factors, spline interval location, trajectory
// validation and initial conditions.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace mqct {

// ---- phase factors exp(-i E t) of Eq. 4 at the RK4 stage times t = n_half dt / 2 -------------
// The phase argument E t is carried as a 64-bit fixed-point fraction of a turn:
//     phi = n_half * inc  (mod 2^64),   inc = frac(E dt / (4 pi)) 2^64,
// so the reduction modulo 2 pi is exact integer wrap-around.  inc comes from one FP64 evaluation
// per level and trajectory (relative error ~1e-16, i.e. <= 6e-13 turn after 2e5 half steps --
// the size of the rounding error of an FP64 product E t at those times), and the angle that
// reaches the FP32 sine and cosine is the top 32 bits of phi (resolution 2^-32 turn).
__device__ __forceinline__ unsigned long long phase_increment(double e, double dt)
{
    double x = e * dt * 0.079577471545947668;  // 1 / (4 pi)
    x -= floor(x);
    const double hi = floor(x * 4294967296.0);
    const double lo = floor((x * 4294967296.0 - hi) * 4294967296.0);
    return ((unsigned long long)hi << 32) + (unsigned long long)lo;
}

// exp(-i phi) for phi = n_half * inc (mod one turn), as (cos, -sin)
__device__ __forceinline__ float2 phase_factor(unsigned long long inc, unsigned int n_half)
{
    const unsigned long long phi = inc * (unsigned long long)n_half;
    const int turn = (int)(phi >> 32);                    // [-2^31, 2^31) <-> [-pi, pi)
    const float ang = (float)turn * 1.46291807926715968e-9f;  // 2 pi / 2^32
    float s, c;
    sincosf(ang, &s, &c);
    return make_float2(c, -s);
}

// ---- spline interval of R (Sec. III): the spline variable X is R, or ln R on the logarithmic
// grid; k = floor((X - X_0)/h) clamped, x = X - X_k; *below is set when R < r_min (the end cubic
// is extrapolated)
__device__ __forceinline__ void locate_interval(const DevSys &S, double R, int &k, double &x, bool &below)
{
    const double X = S.grid_log ? log(R) : R;
    const int kr = __double2int_rd((X - S.x0) * S.inv_h);
    below = kr < 0;
    k = kr < 0 ? 0 : (kr > S.n_int - 1 ? S.n_int - 1 : kr);
    x = X - (S.x0 + k * S.h);
}

// a trajectory that lives in device memory was not seen by the host: validate it here
__device__ __forceinline__ bool traj_valid(const mqct_traj &tr, const DevSys &S, int sys_idx)
{
    return tr.system_idx == sys_idx && tr.dt > 0.0 && tr.e_coll > 0.0 && tr.b >= 0.0 && tr.r0 > 0.0 &&
           tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0 && tr.init_state >= 0 && tr.init_state < S.n;
}

// initial classical state (R, P_R, Phi, P_Phi) of a trajectory: R = r0, Phi = 0, P_Phi = b sqrt(2 mu E),
// P_R = -sqrt(2 mu (E - M_ss(r0)) - P_Phi^2 / r0^2) with the initial mean field M_ss(r0) = m00
__device__ __forceinline__ void initial_state(const DevSys &S, const mqct_traj &tr, double m00, double q[4])
{
    const double lz = tr.b * sqrt(2.0 * S.mu * tr.e_coll);
    q[0] = tr.r0;
    q[1] = -sqrt(2.0 * S.mu * (tr.e_coll - m00) - lz * lz / (tr.r0 * tr.r0));
    q[2] = 0.0;
    q[3] = lz;
}

// v_l(R) from the FP64 spline coefficients of term l in interval k at offset x
__device__ __forceinline__ double spline_fp64(const DevSys &S, int l, int k, double x)
{
    const dbl4 c = S.vcoef[(size_t)l * S.n_int + k];
    return c.x + x * (c.y + x * (c.z + x * c.w));
}

// error-free sum of two FP32 numbers: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// comparisons that keep off the FP64 pipe: for a finite x >= 0 and y >= 0, x >= y compares the bit
// patterns; a double is finite unless its exponent bits are all ones
__device__ __forceinline__ bool ge_pos(double x, double y)
{
    return __double_as_longlong(x) >= __double_as_longlong(y);
}
__device__ __forceinline__ bool finite64(double x)
{
    return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

// RK4 stage update of one classical component (Eqs. 7-10): derivative l = alpha X + beta,
// accumulator (weights 1, 2, 2, 1), next stage input (s < 3: step hdt, hdt, dt) or the step update
// (s = 3: q + dt/6 lacc).  A look-ahead that calls it with the same operands gets the same bits.
__device__ __forceinline__ void stage_component(int s, double alpha, double X, double beta, double hdt, double dt,
                                                double h6, double q, double &qs, double &lacc)
{
    const double l = fma(alpha, X, beta);
    if (s == 0) lacc = l;
    else lacc = fma((s == 1 || s == 2) ? 2.0 : 1.0, l, lacc);
    if (s < 3) qs = fma(s == 2 ? dt : hdt, l, q);
    else qs = fma(h6, lacc, q);
}

}  // namespace mqct
