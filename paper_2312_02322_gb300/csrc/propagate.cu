// Persistent RK4 trajectory kernels and mqct_propagate.
//
// One CTA integrates one trajectory at a time, claiming trajectories from a device
// work queue (longest estimated first) until the queue is empty; the whole RK4 loop of a
// trajectory runs on the device with its amplitudes resident in shared memory.  Per
// RK4 stage (Eq. 4-10):
//   P3  coupling: w = M(R) c and u = M'(R) c for the phase-rotated stage amplitudes
//       c = exp(-i E t_s) a_s, row by row over 32-row sliced-ELL slices (one warp per slice)
//         PLAIN:      M_nm(R) from the spline table of Sec. III, M = sum_p T_p x^p,
//                     computed as w = sum_p x^p (T_p c), u = sum_p p x^(p-1) (T_p c);
//         FACTORISED: w = sum_l v_l(R) (G^l c), u = sum_l v_l'(R) (G^l c)  (Eq. 12);
//   P4  derivative assembly: da/dt = -i exp(iEt) w + (dPhi/dt / 2)(J+ - J-) a (Eq. 5),
//       torque Re(c^dag (J+ - J-) w) (Eq. 10), RK4 accumulation, next stage input and
//       its phase rotation; block reduction of force / torque / diagnostics;
//   C   classical stage update of R, P_R, Phi, P_Phi (Eqs. 7-9) by one thread in FP64.
// Phase arguments E_n t are FP64 and evaluated per level (states of a level share E_n).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>
#include <vector>

#include "internal.h"

namespace mqct {

struct Ctl {
    double q[4], qs[4], lacc[4];
    double phidot, x, dinv, dt, r_end;  // dinv: dx/dR of the spline variable (1, or 1/R on the log grid)
    double line_b, line_v, line_t0;  // prescribed straight line (MQCT_PRESCRIBED_TRAJ)
    double e0, j0, ndev, edev, jdev;
    double v[kMaxTerms], dv[kMaxTerms];
    double vid, dvid;
    double q0[4], err, tcur;  // adaptive steps: classical state at the start, error, time
    int kint, status, steps, done, max_steps, t, item;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// spline of the expansion terms at R (factorised path and initial mean field)
__device__ __forceinline__ void term_at(const DevSys &S, int l, int k, double x, double &v, double &dv)
{
    dbl4 c = S.vcoef[(size_t)l * S.n_int + k];
    v = c.x + x * (c.y + x * (c.z + x * c.w));
    dv = c.y + x * (2.0 * c.z + 3.0 * x * c.w);
}

// interval and local coordinate of R; the spline variable is R, or ln R on the log grid (Sec. III)
__device__ __forceinline__ void locate(const DevSys &S, double R, int &k, double &x)
{
    const double X = S.grid_log ? log(R) : R;
    int kk = (int)floor((X - S.x0) * S.inv_h);
    kk = kk < 0 ? 0 : (kk > S.n_int - 1 ? S.n_int - 1 : kk);
    k = kk;
    x = X - (S.x0 + kk * S.h);
}

// prescribed straight line at time t
__device__ __forceinline__ double line_r(const Ctl &c, double t)
{
    const double s = c.line_v * (t - c.line_t0);
    return sqrt(c.line_b * c.line_b + s * s);
}

// thread 0: stage quantities at the classical stage state qs
__device__ void prepare_stage(const DevSys &S, Ctl &c)
{
    double R = c.qs[0];
    locate(S, R, c.kint, c.x);
    c.dinv = S.grid_log ? 1.0 / R : 1.0;
    c.phidot = (S.flags & MQCT_PRESCRIBED_TRAJ) ? c.line_b * c.line_v / (R * R) : c.qs[3] / (S.mu * R * R);
    if (R < S.r_min) c.status |= MQCT_TRAJ_TABLE_RANGE;
    if (S.path == MQCT_PATH_FACTORISED) {
        double vid = 0.0, dvid = 0.0;
        for (int l = 0; l < S.L; ++l) {
            double v, dv;
            term_at(S, l, c.kint, c.x, v, dv);
            dv *= c.dinv;
            c.v[l] = v;
            c.dv[l] = dv;
            if ((S.id_mask >> l) & 1ull) { vid += v; dvid += dv; }
        }
        c.vid = vid;
        c.dvid = dvid;
    } else if (S.flags & MQCT_DECOUPLED_TRAJ) {
        // the isotropic potential that drives the decoupled classical motion
        double vid = 0.0, dvid = 0.0;
        for (int l = 0; l < S.L; ++l) {
            if (!((S.id_mask >> l) & 1ull)) continue;
            double v, dv;
            term_at(S, l, c.kint, c.x, v, dv);
            vid += v;
            dvid += dv * c.dinv;
        }
        c.vid = vid;
        c.dvid = dvid;
    }
}

// P3: coupling for the rows of this warp; writes W[r] and returns the partial sums
// -Re(c_r^* u_r) (force) and Re(c_r^* w_r) (mean-field energy).
__device__ __forceinline__ void coupling_fp64(const DevSys &S, const Ctl &c, const double2 *__restrict__ C,
                                              double2 *__restrict__ W, int warp, int nwarps, int lane,
                                              double &force, double &vc)
{
    const double x = c.x;
    for (int sl = warp; sl < S.n_slices; sl += nwarps) {
        const int r = sl * kSlice + lane;
        double2 w, u;
        if (S.path == MQCT_PATH_PLAIN) {
            const int off = S.sl_off[sl], width = (S.sl_off[sl + 1] - off) / kSlice;
            const size_t base = (size_t)c.kint * S.nnz_pad + off + lane;
            const double2 *t01 = S.T01 + base, *t23 = S.T23 + base;
            const int *cl = S.cols + off + lane;
            double2 u0 = {0, 0}, u1 = {0, 0}, u2 = {0, 0}, u3 = {0, 0};
            for (int k = 0; k < width; ++k) {
                const int col = __ldg(cl + k * kSlice);
                const double2 a = __ldg(t01 + k * kSlice), b = __ldg(t23 + k * kSlice);
                const double2 z = C[col];
                u0.x = fma(a.x, z.x, u0.x); u0.y = fma(a.x, z.y, u0.y);
                u1.x = fma(a.y, z.x, u1.x); u1.y = fma(a.y, z.y, u1.y);
                u2.x = fma(b.x, z.x, u2.x); u2.y = fma(b.x, z.y, u2.y);
                u3.x = fma(b.y, z.x, u3.x); u3.y = fma(b.y, z.y, u3.y);
            }
            w.x = fma(x, fma(x, fma(x, u3.x, u2.x), u1.x), u0.x);
            w.y = fma(x, fma(x, fma(x, u3.y, u2.y), u1.y), u0.y);
            u.x = fma(x, fma(3.0 * x, u3.x, 2.0 * u2.x), u1.x) * c.dinv;
            u.y = fma(x, fma(3.0 * x, u3.y, 2.0 * u2.y), u1.y) * c.dinv;
        } else {
            const double2 z0 = r < S.n ? C[r] : make_double2(0.0, 0.0);
            w = make_double2(c.vid * z0.x, c.vid * z0.y);
            u = make_double2(c.dvid * z0.x, c.dvid * z0.y);
            for (int f = 0; f < S.n_f; ++f) {
                const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
                const int off = so[sl], width = (so[sl + 1] - off) / kSlice;
                const int *cl = S.f_cols + off + lane;
                const double *gv = S.f_val + off + lane;
                double2 y = {0, 0};
                for (int k = 0; k < width; ++k) {
                    const double g = __ldg(gv + k * kSlice);
                    const double2 z = C[__ldg(cl + k * kSlice)];
                    y.x = fma(g, z.x, y.x);
                    y.y = fma(g, z.y, y.y);
                }
                const int l = S.f_term[f];
                const double v = c.v[l], dv = c.dv[l];
                w.x = fma(v, y.x, w.x); w.y = fma(v, y.y, w.y);
                u.x = fma(dv, y.x, u.x); u.y = fma(dv, y.y, u.y);
            }
        }
        if (r < S.n) {
            W[r] = w;
            const double2 z = C[r];
            force -= z.x * u.x + z.y * u.y;
            vc += z.x * w.x + z.y * w.y;
        }
    }
}

// one RK4 step of length h from the state at t0 (A, C = exp(-iEt0) A, the classical stage input and
// the stage quantities of prepare_stage): the amplitudes end in A and C (phases at t0 + h), the
// classical state in c.q; t_next is the prescribed line's time at the end (t0 + h up to rounding);
// with first set the diagnostics of the start state also reset e0 and j0.  Every thread calls it.
__device__ void rk4_step(const DevSys &S, Ctl &c, double2 *A, double2 *Y0, double2 *Y1, double2 *ACC, double2 *C,
                         double2 *W, double2 *PHa, double2 *PHb, double (*red)[6], double t0, double h, double t_next,
                         bool first, int &ycur)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int n = S.n;
    for (int s = 0; s < 4; ++s) {
        double2 *Yc = ycur ? Y1 : Y0, *Yn = ycur ? Y0 : Y1;
        const double2 *PHc = (s == 0 || s == 3) ? PHa : PHb;
        const double2 *PHn = (s == 0 || s == 1) ? PHb : PHa;
        // P3 (+ phases of the next distinct stage time)
        if (s == 0 || s == 2) {
            const double tn = s == 0 ? t0 + 0.5 * h : t0 + h;
            double2 *dst = s == 0 ? PHb : PHa;
            for (int l = tid; l < S.n_levels; l += nt) {
                double sn, cs;
                sincos(S.lev_energy[l] * tn, &sn, &cs);
                dst[l] = make_double2(cs, -sn);
            }
        }
        double force = 0.0, vc = 0.0;
        coupling_fp64(S, c, C, W, warp, nwarps, lane, force, vc);
        __syncthreads();
        // P4
        const double hp = 0.5 * c.phidot;
        const double wk = (s == 1 || s == 2) ? 2.0 : 1.0;
        const double bn = s == 2 ? h : 0.5 * h;
        double torque = 0.0, nrm = 0.0, erot = 0.0, jy = 0.0;
        for (int r = tid; r < n; r += nt) {
            const int ru = S.up[r], rd = S.dn[r];
            const double au = S.aup[r], ad = S.adn[r];
            const double2 y = Yc[r], yu = Yc[ru], yd = Yc[rd];
            const double2 w = W[r], wu = W[ru], wd = W[rd];
            const double2 z = C[r];
            const double2 p = PHc[S.lev[r]];
            const double2 Dy = make_double2(ad * yd.x - au * yu.x, ad * yd.y - au * yu.y);
            const double2 Dw = make_double2(ad * wd.x - au * wu.x, ad * wd.y - au * wu.y);
            torque += z.x * Dw.x + z.y * Dw.y;
            // k = -i conj(p) w + (phidot/2) D y
            double2 k;
            k.x = fma(hp, Dy.x, p.x * w.y - p.y * w.x);
            k.y = fma(hp, Dy.y, -(p.x * w.x + p.y * w.y));
            if (s == 0) {
                const double pp = y.x * y.x + y.y * y.y;
                nrm += pp;
                erot += S.lev_energy[S.lev[r]] * pp;
                jy += y.x * Dy.y - y.y * Dy.x;
                ACC[r] = k;
            } else {
                double2 acc = ACC[r];
                acc.x = fma(wk, k.x, acc.x);
                acc.y = fma(wk, k.y, acc.y);
                ACC[r] = acc;
                if (s == 3) {
                    double2 an = A[r];
                    an.x = fma(h / 6.0, acc.x, an.x);
                    an.y = fma(h / 6.0, acc.y, an.y);
                    A[r] = an;
                    Yn[r] = an;
                    const double2 pn = PHn[S.lev[r]];
                    C[r] = make_double2(pn.x * an.x - pn.y * an.y, pn.x * an.y + pn.y * an.x);
                }
            }
            if (s < 3) {
                const double2 a0 = A[r];
                const double2 yn = make_double2(fma(bn, k.x, a0.x), fma(bn, k.y, a0.y));
                Yn[r] = yn;
                const double2 pn = PHn[S.lev[r]];
                C[r] = make_double2(pn.x * yn.x - pn.y * yn.y, pn.x * yn.y + pn.y * yn.x);
            }
        }
        // block reduction
        force = warp_sum(force);
        torque = warp_sum(torque);
        if (s == 0) {
            vc = warp_sum(vc); nrm = warp_sum(nrm); erot = warp_sum(erot); jy = warp_sum(jy);
        }
        if (lane == 0) {
            red[warp][0] = force; red[warp][1] = torque;
            if (s == 0) { red[warp][2] = vc; red[warp][3] = nrm; red[warp][4] = erot; red[warp][5] = jy; }
        }
        __syncthreads();
        if (tid == 0) {
            double F = 0, T = 0, V = 0, NR = 0, ER = 0, JY = 0;
            for (int w2 = 0; w2 < nwarps; ++w2) {
                F += red[w2][0]; T += red[w2][1];
                if (s == 0) { V += red[w2][2]; NR += red[w2][3]; ER += red[w2][4]; JY += red[w2][5]; }
            }
            const double R = c.qs[0], PR = c.qs[1], PP = c.qs[3], mu = S.mu;
            const bool dec = S.flags & MQCT_DECOUPLED_TRAJ;
            if (dec) { F = -c.dvid; T = 0.0; }  // isotropic potential alone, no torque
            double l[4] = {PR / mu, F + PP * PP / (mu * R * R * R), c.phidot, T};
            const bool presc = S.flags & MQCT_PRESCRIBED_TRAJ;
            if (presc) l[0] = l[1] = l[2] = l[3] = 0.0;  // the motion is prescribed
            if (s == 0) {
                const double et = PR * PR / (2.0 * mu) + PP * PP / (2.0 * mu * R * R) + (dec ? c.vid : ER + V);
                const double jt = dec ? PP : PP + 0.5 * JY;
                if (first) { c.e0 = et; c.j0 = jt; }
                c.ndev = fmax(c.ndev, fabs(NR - 1.0));
                c.edev = fmax(c.edev, fabs(et - c.e0));
                c.jdev = fmax(c.jdev, fabs(jt - c.j0));
                for (int i = 0; i < 4; ++i) c.lacc[i] = l[i];
            } else {
                for (int i = 0; i < 4; ++i) c.lacc[i] = fma(wk, l[i], c.lacc[i]);
            }
            if (s < 3) {
                for (int i = 0; i < 4; ++i) c.qs[i] = fma(bn, l[i], c.q[i]);
            } else {
                for (int i = 0; i < 4; ++i) { c.q[i] = fma(h / 6.0, c.lacc[i], c.q[i]); c.qs[i] = c.q[i]; }
                bool fin = isfinite(c.q[0]) && isfinite(c.q[1]) && isfinite(c.q[2]) && isfinite(c.q[3]);
                if (!fin) { c.status |= MQCT_TRAJ_NONFINITE; c.done = 1; }
            }
            if (presc) {
                // R of the next stage on the line (stage times as in the phase factors)
                const double tn = s == 3 ? t_next : (s == 2 ? t0 + h : t0 + 0.5 * h);
                c.qs[0] = line_r(c, tn);
                if (s == 3) c.q[0] = c.qs[0];
            }
            if (!(c.status & MQCT_TRAJ_NONFINITE)) prepare_stage(S, c);
        }
        ycur ^= 1;
        __syncthreads();
    }
}

// back to the start of an adaptive step: amplitudes A0 at time t (also the next stage input Y and
// C = exp(-iEt) A0 with fresh phase factors PHa), classical state c.q0, stage quantities
__device__ void restore_start(const DevSys &S, Ctl &c, double2 *A, const double2 *A0, double2 *Y, double2 *C,
                              double2 *PHa, double t)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int l = tid; l < S.n_levels; l += nt) {
        double sn, cs;
        sincos(S.lev_energy[l] * t, &sn, &cs);
        PHa[l] = make_double2(cs, -sn);
    }
    __syncthreads();
    for (int r = tid; r < S.n; r += nt) {
        const double2 a0 = A0[r], p = PHa[S.lev[r]];
        A[r] = a0;
        Y[r] = a0;
        C[r] = make_double2(p.x * a0.x - p.y * a0.y, p.x * a0.y + p.y * a0.x);
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) c.q[i] = c.qs[i] = c.q0[i];
        c.status &= ~MQCT_TRAJ_NONFINITE;
        c.done = 0;
        prepare_stage(S, c);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPropThreads) k_propagate_fp64(PropArgs a)
{
    extern __shared__ double2 smem[];
    __shared__ Ctl c;
    __shared__ DevSys S;
    __shared__ double red[kMaxWarps][6];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int NN = a.smem_n;
    double2 *A = smem, *Y0 = A + NN, *Y1 = Y0 + NN, *ACC = Y1 + NN, *C = ACC + NN, *W = C + NN;
    double2 *PHa = W + NN, *PHb = PHa + a.smem_lev;
    double2 *A0 = PHb + a.smem_lev, *A1 = A0 + NN;  // adaptive steps only (a.adapt)

    for (;;) {
        if (tid == 0) c.item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = c.item;
        if (item >= a.n) break;
        const int t = a.order ? a.order[item] : item;
        const mqct_traj tr = a.trajs[t];
        // trajectories that live in device memory were not seen by the host: validate here
        bool ok = tr.system_idx >= 0 && tr.system_idx < a.n_systems && tr.dt > 0.0 && tr.e_coll > 0.0 &&
                  tr.b >= 0.0 && tr.r0 > 0.0 && tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0;
        if (ok) ok = tr.init_state >= 0 && tr.init_state < a.sys[tr.system_idx].n;
        if (!ok) {
            if (a.diag && tid == 0) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                a.diag[t] = d;
            }
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            S = a.sys[tr.system_idx];
            if (a.t_start) a.t_start[t] = mqct_clock_ns();
        }
        __syncthreads();
        const int n = S.n;
        const int s0 = S.inv[tr.init_state];
        // ---- initial state
        for (int r = tid; r < n; r += nt) {
            double2 v = make_double2(r == s0 ? 1.0 : 0.0, 0.0);
            A[r] = v; Y0[r] = v; C[r] = v;  // phase at t = 0 is 1
        }
        for (int l = tid; l < S.n_levels; l += nt) PHa[l] = make_double2(1.0, 0.0);
        if (tid == 0) {
            int k; double x;
            locate(S, tr.r0, k, x);
            double m00 = 0.0;
            const bool dec = S.flags & MQCT_DECOUPLED_TRAJ;
            for (int l = 0; l < S.L; ++l) {
                double v, dv;
                term_at(S, l, k, x, v, dv);
                // decoupled motion starts in the isotropic potential, not the state's mean field
                m00 += dec ? (((S.id_mask >> l) & 1ull) ? v : 0.0) : v * S.diag_g[(size_t)l * n + s0];
            }
            const double lz = tr.b * sqrt(2.0 * S.mu * tr.e_coll);
            c.q[0] = tr.r0; c.q[2] = 0.0; c.q[3] = lz;
            c.q[1] = -sqrt(2.0 * S.mu * (tr.e_coll - m00) - lz * lz / (tr.r0 * tr.r0));
            if (S.flags & MQCT_PRESCRIBED_TRAJ) {
                // the straight line R(t) = sqrt(b^2 + v^2 (t - t_0)^2), time-symmetric about t_0
                c.line_b = tr.b;
                c.line_v = sqrt(2.0 * tr.e_coll / S.mu);
                c.line_t0 = 0.5 * tr.max_steps * tr.dt;
                c.q[0] = line_r(c, 0.0);
                c.q[1] = c.q[2] = c.q[3] = 0.0;
            }
            for (int i = 0; i < 4; ++i) c.qs[i] = c.q[i];
            c.dt = tr.dt; c.r_end = tr.r_end; c.max_steps = tr.max_steps;
            c.status = 0; c.steps = 0; c.done = tr.max_steps <= 0;
            if (c.done) c.status |= MQCT_TRAJ_MAX_STEPS;
            c.ndev = c.edev = c.jdev = 0.0;
            c.t = t;
            prepare_stage(S, c);
        }
        __syncthreads();
        int ycur = 0;
        const double dt = tr.dt;
        // ---- RK4 steps
        if (S.adapt_tol > 0.0) {
            // step doubling (the adaptive step of Sec. III in the reading of the header): one step of
            // h against two of h/2 from the same state; the two-half result is kept when
            // max_n |a_n(halves) - a_n(one step)| <= tol or h = dt, else h halves and the step is
            // retried; h doubles (up to hmax) after a step whose error was <= tol / 64
            const double hmax = dt * S.adapt_hmax;
            double h = hmax, tcur = 0.0;
            while (!c.done) {
                for (int r = tid; r < n; r += nt) A0[r] = A[r];
                if (tid == 0)
                    for (int i = 0; i < 4; ++i) c.q0[i] = c.q[i];
                __syncthreads();
                rk4_step(S, c, A, Y0, Y1, ACC, C, W, PHa, PHb, red, tcur, h, tcur + h, c.steps == 0, ycur);
                for (int r = tid; r < n; r += nt) A1[r] = A[r];
                __syncthreads();
                restore_start(S, c, A, A0, ycur ? Y1 : Y0, C, PHa, tcur);
                rk4_step(S, c, A, Y0, Y1, ACC, C, W, PHa, PHb, red, tcur, 0.5 * h, tcur + 0.5 * h, false, ycur);
                if (!(c.status & MQCT_TRAJ_NONFINITE))
                    rk4_step(S, c, A, Y0, Y1, ACC, C, W, PHa, PHb, red, tcur + 0.5 * h, 0.5 * h, tcur + h, false, ycur);
                // error: max over the states of |a(halves) - a(one step)| (independent of the order)
                double err = 0.0;
                for (int r = tid; r < n; r += nt) {
                    const double2 x = A[r], y = A1[r];
                    err = fmax(err, hypot(x.x - y.x, x.y - y.y));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
                if (lane == 0) red[warp][0] = err;
                __syncthreads();
                if (tid == 0) {
                    double e2 = 0.0;
                    for (int w2 = 0; w2 < nwarps; ++w2) e2 = fmax(e2, red[w2][0]);
                    c.err = e2;
                }
                __syncthreads();
                if (!(c.status & MQCT_TRAJ_NONFINITE) && !(c.err <= S.adapt_tol) && h > dt) {
                    restore_start(S, c, A, A0, ycur ? Y1 : Y0, C, PHa, tcur);
                    h *= 0.5;
                    continue;
                }
                if (tid == 0) {
                    c.steps += 1;
                    if (!(c.status & MQCT_TRAJ_NONFINITE)) {
                        if (c.q[0] >= c.r_end && c.q[1] > 0.0) c.done = 1;
                        else if (c.steps >= c.max_steps) { c.status |= MQCT_TRAJ_MAX_STEPS; c.done = 1; }
                    }
                    c.tcur = tcur + h;
                }
                __syncthreads();
                tcur = c.tcur;
                if (64.0 * c.err <= S.adapt_tol && h < hmax) h *= 2.0;
            }
        } else {
            while (!c.done) {
                const int step = c.steps;
                const double t0 = step * dt;
                rk4_step(S, c, A, Y0, Y1, ACC, C, W, PHa, PHb, red, t0, dt, (step + 1) * dt, step == 0, ycur);
                if (tid == 0) {
                    const bool presc = S.flags & MQCT_PRESCRIBED_TRAJ;
                    c.steps = step + 1;
                    if (!(c.status & MQCT_TRAJ_NONFINITE)) {
                        if (!presc && c.q[0] >= c.r_end && c.q[1] > 0.0) c.done = 1;
                        else if (c.steps >= c.max_steps) { c.status |= presc ? 0 : MQCT_TRAJ_MAX_STEPS; c.done = 1; }
                    }
                    c.tcur = c.steps * dt;
                }
                __syncthreads();
            }
        }
        // ---- diagnostics of the final state (C holds exp(-iEt) a at t = steps dt)
        if (!(c.status & MQCT_TRAJ_NONFINITE)) {
            double force = 0.0, vc = 0.0;
            coupling_fp64(S, c, C, W, warp, nwarps, lane, force, vc);
            double nrm = 0.0, erot = 0.0, jy = 0.0;
            for (int r = tid; r < n; r += nt) {
                const double2 y = A[r], yu = A[S.up[r]], yd = A[S.dn[r]];
                const double2 Dy = make_double2(S.adn[r] * yd.x - S.aup[r] * yu.x, S.adn[r] * yd.y - S.aup[r] * yu.y);
                const double pp = y.x * y.x + y.y * y.y;
                nrm += pp;
                erot += S.lev_energy[S.lev[r]] * pp;
                jy += y.x * Dy.y - y.y * Dy.x;
            }
            vc = warp_sum(vc); nrm = warp_sum(nrm); erot = warp_sum(erot); jy = warp_sum(jy);
            __syncthreads();
            if (lane == 0) { red[warp][2] = vc; red[warp][3] = nrm; red[warp][4] = erot; red[warp][5] = jy; }
            __syncthreads();
            if (tid == 0) {
                double V = 0, NR = 0, ER = 0, JY = 0;
                for (int w2 = 0; w2 < nwarps; ++w2) { V += red[w2][2]; NR += red[w2][3]; ER += red[w2][4]; JY += red[w2][5]; }
                const double R = c.q[0], PR = c.q[1], PP = c.q[3], mu = S.mu;
                const bool dec = S.flags & MQCT_DECOUPLED_TRAJ;
                const double et = PR * PR / (2.0 * mu) + PP * PP / (2.0 * mu * R * R) + (dec ? c.vid : ER + V);
                const double jt = dec ? PP : PP + 0.5 * JY;
                if (c.steps == 0) { c.e0 = et; c.j0 = jt; }
                c.ndev = fmax(c.ndev, fabs(NR - 1.0));
                c.edev = fmax(c.edev, fabs(et - c.e0));
                c.jdev = fmax(c.jdev, fabs(jt - c.j0));
            }
        }
        __syncthreads();
        // ---- outputs in the caller's state order
        if (a.pop)
            for (int r = tid; r < n; r += nt) {
                const double2 y = A[r];
                a.pop[(size_t)t * a.nmax + S.perm[r]] = y.x * y.x + y.y * y.y;
            }
        if (a.amp)
            for (int r = tid; r < n; r += nt) {
                const double2 y = A[r];
                a.amp[((size_t)t * a.nmax + S.perm[r]) * 2] = y.x;
                a.amp[((size_t)t * a.nmax + S.perm[r]) * 2 + 1] = y.y;
            }
        if (a.diag && tid == 0) {
            mqct_diag d;
            d.steps = c.steps; d.status = c.status;
            d.norm_dev = c.ndev; d.energy_dev = c.edev; d.angmom_dev = c.jdev;
            d.t_final = c.tcur;
            a.diag[t] = d;
        }
        if (a.t_done && tid == 0) a.t_done[t] = mqct_clock_ns();
        __syncthreads();
    }
}

// work-order keys: estimated cost of a trajectory (steps ~ 2 r0 / v, work per step ~ nnz)
__global__ void k_order_keys(const DevSys *sys, int n_systems, const mqct_traj *trajs, int n, float *keys, int *idx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const mqct_traj tr = trajs[i];
    idx[i] = i;
    if (tr.system_idx < 0 || tr.system_idx >= n_systems) { keys[i] = 0.0f; return; }
    const DevSys &S = sys[tr.system_idx];
    double v = sqrt(2.0 * fmax(tr.e_coll, 1e-30) / S.mu);
    double steps = fmin(2.0 * tr.r0 / (v * tr.dt), (double)tr.max_steps);
    double work = S.path == MQCT_PATH_PLAIN ? (double)S.nnz_pad : (double)S.n * (S.n_f + 1);
    keys[i] = (float)(-(steps * (work + 64.0 * S.n)));  // ascending sort = longest first
}

}  // namespace mqct

using namespace mqct;

namespace {

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct StreamAllocs {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit StreamAllocs(cudaStream_t s) : st(s) {}
    cudaError_t get(void **p, size_t bytes)
    {
        cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~StreamAllocs()
    {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

}  // namespace

namespace {

// trajectory index i of the work order belongs to system s
struct IsSystem {
    const mqct_traj *tr;
    int s;
    __device__ bool operator()(const int &i) const { return tr[i].system_idx == s; }
};

// estimated work of each system: sum of its trajectories' (negated) order keys
__global__ void k_system_work(const mqct_traj *trajs, const int *order, const float *keys, int n, int n_systems,
                              double *work)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = trajs[order[i]].system_idx;
    if (s >= 0 && s < n_systems) atomicAdd(work + s, -(double)keys[i]);
}

}  // namespace

extern "C" mqct_status mqct_propagate(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs, int32_t n,
                                      double *final_pop, double *final_amp, mqct_diag *diag, void *cuda_stream)
{
    return mqct_propagate_ex(systems, n_systems, trajs, n, final_pop, final_amp, diag, nullptr, cuda_stream);
}

extern "C" mqct_status mqct_propagate_ex(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs,
                                         int32_t n, double *final_pop, double *final_amp, mqct_diag *diag,
                                         const mqct_propagate_opts *opts, void *cuda_stream)
{
    reset_launches();
    const mqct_propagate_opts no_opts{};
    const mqct_propagate_opts &op = opts ? *opts : no_opts;
    auto shape_of = [&](int i) { return op.batch_shape ? op.batch_shape[i] : 0; };
    auto slots_of = [&](int i) { return op.tc_slots ? op.tc_slots[i] : 0; };
    for (int i = 0; i < std::max(0, (int)n_systems); ++i) {
        if (shape_of(i) < 0 || shape_of(i) > 7) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: batch_shape outside [0, 7]");
        if (slots_of(i) < 0 || slots_of(i) > 8192) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: tc_slots outside [0, 8192]");
    }
    if (!systems || n_systems < 1) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: no systems");
    if (n < 0) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: n < 0");
    if (n > 0 && !trajs) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: trajs is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int nmax = 0, maxlev = 0, max_slices = 0;
    int path = -1, prec = -1;
    for (int i = 0; i < n_systems; ++i) {
        if (!systems[i]) return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: NULL system");
        const DevSys &h = systems[i]->s.h;
        nmax = std::max(nmax, h.n);
        maxlev = std::max(maxlev, h.n_levels);
        max_slices = std::max(max_slices, h.n_slices);
        if (path < 0) { path = h.path; prec = h.precision; }
        if (h.path != path || h.precision != prec)
            return fail(MQCT_ERR_INVALID_ARG, "mqct_propagate: systems differ in path or precision");
    }
    // FP32 factorised systems run the persistent batched kernel; FP32 PLAIN systems (large bases
    // with the FP32 spline table) and BF16X3 systems the stage-synchronous path
    const bool stage_sync = prec == MQCT_BF16X3 || (prec == MQCT_FP32 && path == MQCT_PATH_PLAIN);
    if (prec == MQCT_FP32 && !stage_sync)
        for (int i = 0; i < n_systems; ++i) {
            const DevSys &h = systems[i]->s.h;
            if (batched_width(h) == 0) return fail(MQCT_ERR_UNSUPPORTED, "mqct_propagate: basis too large for the batched kernel");
            if (shape_of(i) > 0 && !batched_shape_fits(h, shape_of(i) - 1))
                return fail(MQCT_ERR_UNSUPPORTED, "mqct_propagate: batch_shape does not fit a system's basis");
        }
    if (n == 0) return MQCT_OK;

    const bool trajs_dev = is_device_ptr(trajs);
    // host trajectories are validated on the host
    if (!trajs_dev) {
        for (int i = 0; i < n; ++i) {
            const mqct_traj &t = trajs[i];
            if (t.system_idx < 0 || t.system_idx >= n_systems) return fail(MQCT_ERR_INVALID_ARG, "trajectory system_idx out of range");
            const DevSys &h = systems[t.system_idx]->s.h;
            if (t.init_state < 0 || t.init_state >= h.n) return fail(MQCT_ERR_INVALID_ARG, "trajectory init_state out of range");
            if (!(t.dt > 0) || !(t.e_coll > 0) || !(t.b >= 0) || !(t.r0 > 0) || t.max_steps < 0 || !std::isfinite(t.r_end))
                return fail(MQCT_ERR_INVALID_ARG, "trajectory with invalid e_coll, b, r0, r_end, dt or max_steps");
            double q = 2.0 * h.mu * t.e_coll - 2.0 * h.mu * t.e_coll * (t.b * t.b) / (t.r0 * t.r0);
            if (!(q > 0)) return fail(MQCT_ERR_INVALID_ARG, "trajectory starts inside its centrifugal barrier (b >= r0)");
        }
    }
    StreamAllocs sa(st);
    cudaError_t e;
    // device view of the system array
    DevSys *dsys = nullptr;
    {
        std::vector<DevSys> hv(n_systems);
        for (int i = 0; i < n_systems; ++i) hv[i] = systems[i]->s.h;
        if ((e = sa.get((void **)&dsys, sizeof(DevSys) * n_systems)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        if ((e = cudaMemcpyAsync(dsys, hv.data(), sizeof(DevSys) * n_systems, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync");
    }
    const mqct_traj *dtr = trajs;
    if (!trajs_dev) {
        mqct_traj *p = nullptr;
        if ((e = sa.get((void **)&p, sizeof(mqct_traj) * n)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
        if ((e = cudaMemcpyAsync(p, trajs, sizeof(mqct_traj) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync");
        dtr = p;
    }
    // outputs: device pointers are written directly, host ones through staging buffers
    const bool pop_dev = is_device_ptr(final_pop), amp_dev = is_device_ptr(final_amp), diag_dev = is_device_ptr(diag);
    const bool any_host = (final_pop && !pop_dev) || (final_amp && !amp_dev) || (diag && !diag_dev);
    double *dpop = final_pop, *damp = final_amp;
    mqct_diag *ddiag = nullptr;
    if (final_pop && !pop_dev && (e = sa.get((void **)&dpop, sizeof(double) * (size_t)n * nmax)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
    if (final_amp && !amp_dev && (e = sa.get((void **)&damp, sizeof(double) * 2 * (size_t)n * nmax)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
    if (diag && diag_dev) ddiag = diag;
    else if ((diag || any_host) && (e = sa.get((void **)&ddiag, sizeof(mqct_diag) * (size_t)n)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
    long long *dts = reinterpret_cast<long long *>(op.t_start_ns), *dtd = reinterpret_cast<long long *>(op.t_done_ns);
    const bool ts_host = op.t_start_ns && !is_device_ptr(op.t_start_ns), td_host = op.t_done_ns && !is_device_ptr(op.t_done_ns);
    if (ts_host && (e = sa.get((void **)&dts, sizeof(long long) * (size_t)n)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    if (td_host && (e = sa.get((void **)&dtd, sizeof(long long) * (size_t)n)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    // work order: longest estimated trajectory first
    float *keys = nullptr, *keys2 = nullptr;
    int *idx = nullptr, *order = nullptr, *queue = nullptr;
    if ((e = sa.get((void **)&keys, sizeof(float) * n)) != cudaSuccess || (e = sa.get((void **)&keys2, sizeof(float) * n)) != cudaSuccess ||
        (e = sa.get((void **)&idx, sizeof(int) * n)) != cudaSuccess || (e = sa.get((void **)&order, sizeof(int) * n)) != cudaSuccess ||
        (e = sa.get((void **)&queue, sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync");
    k_order_keys<<<(n + 255) / 256, 256, 0, st>>>(dsys, n_systems, dtr, n, keys, idx);
    count_launches(1);
    size_t tmp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys2, idx, order, n, 0, 32, st);
    void *tmp = nullptr;
    if ((e = sa.get(&tmp, tmp_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys2, idx, order, n, 0, 32, st)) != cudaSuccess)
        return cuda_fail(e, "cub::DeviceRadixSort");
    if ((e = cudaMemsetAsync(queue, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    if (prec != MQCT_FP64) {
        // uneven batch of several systems: the work order split per system (stable, so each list
        // stays longest first) and the estimated work of each system, all on the device
        int *lists = order, *counts = nullptr, *queues = queue;
        double *work = nullptr;
        if (n_systems > 1) {
            if ((e = sa.get((void **)&lists, sizeof(int) * (size_t)n * n_systems)) != cudaSuccess ||
                (e = sa.get((void **)&counts, sizeof(int) * n_systems)) != cudaSuccess ||
                (e = sa.get((void **)&queues, sizeof(int) * n_systems)) != cudaSuccess ||
                (e = sa.get((void **)&work, sizeof(double) * n_systems)) != cudaSuccess)
                return cuda_fail(e, "cudaMallocAsync");
            cudaMemsetAsync(queues, 0, sizeof(int) * n_systems, st);
            cudaMemsetAsync(work, 0, sizeof(double) * n_systems, st);
            k_system_work<<<(n + 255) / 256, 256, 0, st>>>(dtr, order, keys2, n, n_systems, work);
            count_launches(1);
            size_t sel_bytes = 0;
            cub::DeviceSelect::If(nullptr, sel_bytes, order, lists, counts, n, IsSystem{dtr, 0}, st);
            void *sel_tmp = nullptr;
            if ((e = sa.get(&sel_tmp, sel_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
            for (int i = 0; i < n_systems; ++i)
                if ((e = cub::DeviceSelect::If(sel_tmp, sel_bytes, order, lists + (size_t)i * n, counts + i, n,
                                               IsSystem{dtr, i}, st)) != cudaSuccess)
                    return cuda_fail(e, "cub::DeviceSelect");
        }
        if (!stage_sync) {
            // one persistent launch over every system of the call (at most kBatchMaxSystems per
            // launch): CTAs bind to systems on the device
            BatchMultiArgs ma{};
            ma.trajs = dtr; ma.pop = dpop; ma.amp = damp; ma.diag = ddiag; ma.nmax = nmax;
            ma.t_start = dts; ma.t_done = dtd; ma.n = n;
            int shape = 0;
            for (int i = 0; i < n_systems && !shape; ++i) shape = shape_of(i);
            for (int g0 = 0; g0 < n_systems; g0 += kBatchMaxSystems) {
                const int ng = std::min(kBatchMaxSystems, n_systems - g0);
                ma.sys = dsys + g0; ma.lists = lists + (size_t)g0 * n; ma.counts = counts ? counts + g0 : nullptr;
                ma.queues = queues + g0; ma.work = work ? work + g0 : nullptr; ma.n_systems = ng; ma.sys_base = g0;
                std::vector<const DevSys *> hs;
                for (int i = 0; i < ng; ++i) hs.push_back(&systems[g0 + i]->s.h);
                if ((e = run_batched(ma, hs, shape, st)) != cudaSuccess) return cuda_fail(e, "batched launch");
            }
        } else {
            BatchArgs ba{};
            ba.trajs = dtr; ba.pop = dpop; ba.amp = damp; ba.diag = ddiag; ba.nmax = nmax;
            ba.t_start = dts; ba.t_done = dtd;
            if (n_systems == 1) {
                ba.sys = systems[0]->s.d; ba.order = order; ba.n = n; ba.queue = queue; ba.sys_idx = 0;
                ba.tc_slots = slots_of(0);
                const mqct_status ts = run_tc_batched(ba, systems[0]->s.h, st);
                if (ts != MQCT_OK) return ts;
            } else {
                // the stage-synchronous path fills the GPU with one system at a time
                std::vector<int> hc(n_systems);
                if ((e = cudaMemcpyAsync(hc.data(), counts, sizeof(int) * n_systems, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(st)) != cudaSuccess)
                    return cuda_fail(e, "work partition");
                for (int i = 0; i < n_systems; ++i) {
                    if (hc[i] == 0) continue;
                    BatchArgs bi = ba;
                    bi.sys = systems[i]->s.d; bi.order = lists + (size_t)i * n; bi.n = hc[i]; bi.queue = queues + i;
                    bi.sys_idx = i; bi.tc_slots = slots_of(i);
                    const mqct_status ts = run_tc_batched(bi, systems[i]->s.h, st);
                    if (ts != MQCT_OK) return ts;
                }
            }
        }
    } else {
    // launch shape: one warp per 32-row slice (balanced), persistent grid
    const int maxw = kPropThreads / 32;
    int per = (max_slices + maxw - 1) / maxw;
    int nwarps = std::max(4, std::min(maxw, (max_slices + per - 1) / per));
    int threads = nwarps * 32;
    bool adapt = false;
    for (int i = 0; i < n_systems; ++i) adapt |= systems[i]->s.h.adapt_tol > 0.0;
    size_t smem = sizeof(double2) * ((adapt ? 8 : 6) * (size_t)nmax + 2 * (size_t)maxlev);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaFuncSetAttribute(k_propagate_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute (basis too large for shared memory)");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate_fp64, threads, smem)) != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(MQCT_ERR_UNSUPPORTED, "mqct_propagate: kernel does not fit on an SM");
    int grid = std::min(n, sms * per_sm);
    PropArgs pa{};
    pa.sys = dsys; pa.trajs = dtr; pa.order = order; pa.n = n; pa.n_systems = n_systems; pa.queue = queue;
    pa.pop = dpop; pa.amp = damp; pa.diag = ddiag; pa.nmax = nmax; pa.smem_n = nmax; pa.smem_lev = maxlev;
    pa.t_start = dts; pa.t_done = dtd; pa.adapt = adapt ? 1 : 0;
    k_propagate_fp64<<<grid, threads, smem, st>>>(pa);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_propagate_fp64 launch");
    }

    if (ts_host && (e = cudaMemcpyAsync(op.t_start_ns, dts, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if (td_host && (e = cudaMemcpyAsync(op.t_done_ns, dtd, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if (!any_host) {
        if ((ts_host || td_host) && (e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        return MQCT_OK;
    }
    if (final_pop && !pop_dev &&
        (e = cudaMemcpyAsync(final_pop, dpop, sizeof(double) * (size_t)n * nmax, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if (final_amp && !amp_dev &&
        (e = cudaMemcpyAsync(final_amp, damp, sizeof(double) * 2 * (size_t)n * nmax, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    std::vector<mqct_diag> hd(n);
    mqct_diag *dst = (diag && !diag_dev) ? diag : hd.data();
    if ((e = cudaMemcpyAsync(dst, ddiag, sizeof(mqct_diag) * (size_t)n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int i = 0; i < n; ++i)
        if (dst[i].status != 0) return fail(MQCT_ERR_TRAJ, "at least one trajectory ended with a non-zero status");
    return MQCT_OK;
}
