// Discrete adjoint of the RK4 trajectory map: gradients of cross sections with respect to
// the PES expansion parameters theta (v_lambda(R) depends on theta through tables of
// d v_lambda / d theta_p given at create time).
//
// L = sum_{g,l} dL/dsigma[g][l] sigma[g][l],  sigma[g][l] = sum_{t in g} w_t sum_{s in l} |a_s|^2,
// so each trajectory starts the reverse sweep from abar_s = 2 w_t dL/dsigma[g_t][level(s)] a_s.
// One CTA per trajectory, FP64, the factorised coupling M(R) = sum_l v_l(R) G^l (Eq. 12):
//   1. forward RK4 (the same map as mqct_propagate), a checkpoint of the state every K steps;
//   2. for each segment, last first: recompute its states from the checkpoint, then reverse
//      every step: recompute the four stage states and apply the vector-Jacobian product of
//      f (Eqs. 5, 7-10) in reverse stage order:
//        kbar4 = dt/6 lam,                 Ybar4 = J4^T kbar4
//        kbar3 = dt/3 lam + dt   Ybar4,    Ybar3 = J3^T kbar3
//        kbar2 = dt/3 lam + dt/2 Ybar3,    Ybar2 = J2^T kbar2
//        kbar1 = dt/6 lam + dt/2 Ybar2,    Ybar1 = J1^T kbar1,   lam <- lam + sum Ybar_i,
//      with theta_bar accumulated from the same stage quantities;
//   3. the initial P_R depends on theta through M_ss(r0): theta_bar += dP_R0/dtheta * P_R_bar.
// The number of steps of each trajectory is held at its forward value.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace mqct {

constexpr int kAdjThreads = 512;
constexpr int kAdjMaxP = 32;
constexpr int kAdjMaxL = 16;
constexpr int kAdjRed = 8 + 3 * kAdjMaxL;  // block-reduced scalars per VJP

struct AdjArgs {
    const DevSys *sys;
    const mqct_traj *trajs;
    int n;
    int *queue;
    const double *weight;
    const int *group;
    int n_groups;
    const double *dLds;       // [n_groups][n_levels]
    int K;                    // checkpoint interval
    int max_ckpt;             // checkpoints that fit in a CTA's scratch
    double *scratch;          // per CTA: (max_ckpt + K) * stride doubles
    size_t stride;            // doubles per stored state (2n + 4, padded)
    double *theta_traj;       // [n][P] per-trajectory gradient
    int *status;              // [n]
};

struct AdjCtl {
    double q[4], qs[4], lacc[4];   // classical state, stage input, accumulated derivatives
    double qk[4][4];               // classical stage states Y1..Y4 (R, PR, Phi, PPhi)
    double lq[4];                  // classical part of k (forward)
    double lam[4], kb[4], yb[4], ynew[4];  // classical cotangents
    double v[kAdjMaxL], dv[kAdjMaxL], d2v[kAdjMaxL];
    double red[kAdjRed];
    double theta[kAdjMaxP];
    double p_r0;
    int steps, status, item, t, kint;
    double x;
};

__device__ __forceinline__ double bsum_warp(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sums of m values held per thread (vals[0..m)); results in c.red[0..m)
__device__ void block_sums(double *vals, int m, AdjCtl &c, double *wred)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int i = 0; i < m; ++i) {
        const double s = bsum_warp(vals[i]);
        if (lane == 0) wred[warp * kAdjRed + i] = s;
    }
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += wred[w * kAdjRed + i];
        c.red[i] = s;
    }
    __syncthreads();
}

// thread 0: interval and v, v', v'' of all terms at R
__device__ void terms_at(const DevSys &S, double R, AdjCtl &c)
{
    int k = (int)floor((R - S.r_min) * S.inv_h);
    k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
    const double x = R - (S.r_min + k * S.h);
    c.kint = k;
    c.x = x;
    for (int l = 0; l < S.L; ++l) {
        const dbl4 q = S.vcoef[(size_t)l * S.n_int + k];
        c.v[l] = q.x + x * (q.y + x * (q.z + x * q.w));
        c.dv[l] = q.y + x * (2.0 * q.z + 3.0 * x * q.w);
        c.d2v[l] = 2.0 * q.z + 6.0 * x * q.w;
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b)  // conj(a) * b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

struct AdjSmem {
    double2 *A, *Y2, *Y3, *Y4, *K, *ACC, *C, *W, *LAM, *KB, *YN, *Z, *DC, *MZ, *MDC, *U, *PH;
};

// Forward right-hand side f(t, Y): K = da/dt, c.lq = classical derivatives.  Needs c.v/c.dv at
// the stage R (terms_at) and writes C = p Y, W = M c.
__device__ void fwd_eval(const DevSys &S, double t, const double2 *Ya, const double *Yq, AdjSmem &m, AdjCtl &c,
                         double *wred)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = S.n;
    for (int l = tid; l < S.n_levels; l += nt) {
        double sn, cs;
        sincos(S.lev_energy[l] * t, &sn, &cs);
        m.PH[l] = make_double2(cs, -sn);
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) m.C[r] = cmul(m.PH[S.lev[r]], Ya[r]);
    __syncthreads();
    double force = 0.0;
    double vid = 0.0, dvid = 0.0;
    for (int l = 0; l < S.L; ++l)
        if ((S.id_mask >> l) & 1ull) { vid += c.v[l]; dvid += c.dv[l]; }
    for (int sl = warp; sl < S.n_slices; sl += nw) {
        const int r = sl * kSlice + lane;
        const double2 c0 = r < n ? m.C[r] : make_double2(0, 0);
        double2 w = make_double2(vid * c0.x, vid * c0.y), u = make_double2(dvid * c0.x, dvid * c0.y);
        for (int f = 0; f < S.n_f; ++f) {
            const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
            const int off = so[sl], width = (so[sl + 1] - off) / kSlice;
            double2 y = make_double2(0, 0);
            for (int k = 0; k < width; ++k) {
                const double gv = S.f_val[off + k * kSlice + lane];
                const double2 z = m.C[S.f_cols[off + k * kSlice + lane]];
                y.x = fma(gv, z.x, y.x);
                y.y = fma(gv, z.y, y.y);
            }
            const int l = S.f_term[f];
            w.x = fma(c.v[l], y.x, w.x); w.y = fma(c.v[l], y.y, w.y);
            u.x = fma(c.dv[l], y.x, u.x); u.y = fma(c.dv[l], y.y, u.y);
        }
        if (r < n) {
            m.W[r] = w;
            force -= c0.x * u.x + c0.y * u.y;
        }
    }
    __syncthreads();
    const double R = Yq[0], PR = Yq[1], PP = Yq[3];
    const double hp = 0.5 * PP / (S.mu * R * R);
    double torque = 0.0;
    for (int r = tid; r < n; r += nt) {
        const int ru = S.up[r], rd = S.dn[r];
        const double au = S.aup[r], ad = S.adn[r];
        const double2 w = m.W[r], wu = m.W[ru], wd = m.W[rd], z = m.C[r];
        const double2 Dw = make_double2(ad * wd.x - au * wu.x, ad * wd.y - au * wu.y);
        torque += z.x * Dw.x + z.y * Dw.y;
        const double2 y = Ya[ru], yd = Ya[rd];
        const double2 Dy = make_double2(ad * yd.x - au * y.x, ad * yd.y - au * y.y);
        const double2 p = m.PH[S.lev[r]];
        double2 k;
        k.x = fma(hp, Dy.x, p.x * w.y - p.y * w.x);
        k.y = fma(hp, Dy.y, -(p.x * w.x + p.y * w.y));
        m.K[r] = k;
    }
    double vals[2] = {force, torque};
    block_sums(vals, 2, c, wred);
    if (tid == 0) {
        c.lq[0] = PR / S.mu;
        c.lq[1] = c.red[0] + PP * PP / (S.mu * R * R * R);
        c.lq[2] = PP / (S.mu * R * R);
        c.lq[3] = c.red[1];
    }
    __syncthreads();
}

// Vector-Jacobian product at stage (t, Y): given the cotangent (KB, c.kb) of f, add J^T kbar
// to (YN, c.ynew) and the parameter cotangent to c.theta.  Needs terms_at(Y_R).
__device__ void vjp_eval(const DevSys &S, double t, const double2 *Ya, const double *Yq, AdjSmem &m, AdjCtl &c,
                         double *wred)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = S.n, L = S.L;
    for (int l = tid; l < S.n_levels; l += nt) {
        double sn, cs;
        sincos(S.lev_energy[l] * t, &sn, &cs);
        m.PH[l] = make_double2(cs, -sn);
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        const double2 p = m.PH[S.lev[r]];
        m.C[r] = cmul(p, Ya[r]);
        m.Z[r] = cmul(p, m.KB[r]);
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        const double au = S.aup[r], ad = S.adn[r];
        const double2 cu = m.C[S.up[r]], cd = m.C[S.dn[r]];
        m.DC[r] = make_double2(ad * cd.x - au * cu.x, ad * cd.y - au * cu.y);
    }
    __syncthreads();
    // per-row contractions with every term: w = M c, u = M' c, u2 = M'' c, M z, M Dc, and the
    // per-term sums alpha_l = Re(kbar^dag (-i conj(p) G^l c)), beta_l = -Re(c^dag G^l c),
    // gamma_l = -Re((Dc)^dag G^l c)
    double *wt = wred + warp * kAdjRed;  // this warp's per-term sums (alpha, beta, gamma)
    if (lane < 3 * L) wt[4 + lane] = 0.0;
    __syncwarp();
    // warp-reduce one term's three row contributions and add them to the warp's sums
    auto add_term = [&](int l, double a1, double b1, double g1) {
        a1 = bsum_warp(a1); b1 = bsum_warp(b1); g1 = bsum_warp(g1);
        if (lane == 0) { wt[4 + 3 * l] += a1; wt[5 + 3 * l] += b1; wt[6 + 3 * l] += g1; }
    };
    double s3 = 0.0;  // Re(c^dag M'' c)
    for (int sl = warp; sl < S.n_slices; sl += nw) {
        const int r = sl * kSlice + lane;
        const bool in = r < n;
        const double2 c0 = in ? m.C[r] : make_double2(0, 0), z0 = in ? m.Z[r] : make_double2(0, 0);
        const double2 d0 = in ? m.DC[r] : make_double2(0, 0), kb = in ? m.KB[r] : make_double2(0, 0);
        const double2 p = in ? m.PH[S.lev[r]] : make_double2(1, 0);
        double2 w = make_double2(0, 0), u = w, u2 = w, mz = w, md = w;
        for (int l = 0; l < L; ++l) {
            if (!((S.id_mask >> l) & 1ull)) continue;
            w.x += c.v[l] * c0.x; w.y += c.v[l] * c0.y;
            u.x += c.dv[l] * c0.x; u.y += c.dv[l] * c0.y;
            u2.x += c.d2v[l] * c0.x; u2.y += c.d2v[l] * c0.y;
            mz.x += c.v[l] * z0.x; mz.y += c.v[l] * z0.y;
            md.x += c.v[l] * d0.x; md.y += c.v[l] * d0.y;
            const double2 py = cconjmul(p, c0);  // conj(p) Y with Y = c
            add_term(l, kb.x * py.y - kb.y * py.x, -(c0.x * c0.x + c0.y * c0.y), -(d0.x * c0.x + d0.y * c0.y));
        }
        for (int f = 0; f < S.n_f; ++f) {
            const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
            const int off = so[sl], width = (so[sl + 1] - off) / kSlice;
            double2 yc = make_double2(0, 0), yz = yc, yd = yc;
            for (int k = 0; k < width; ++k) {
                const int e = off + k * kSlice + lane;
                const double gv = S.f_val[e];
                const int col = S.f_cols[e];
                const double2 a1 = m.C[col], a2 = m.Z[col], a3 = m.DC[col];
                yc.x = fma(gv, a1.x, yc.x); yc.y = fma(gv, a1.y, yc.y);
                yz.x = fma(gv, a2.x, yz.x); yz.y = fma(gv, a2.y, yz.y);
                yd.x = fma(gv, a3.x, yd.x); yd.y = fma(gv, a3.y, yd.y);
            }
            const int l = S.f_term[f];
            w.x = fma(c.v[l], yc.x, w.x); w.y = fma(c.v[l], yc.y, w.y);
            u.x = fma(c.dv[l], yc.x, u.x); u.y = fma(c.dv[l], yc.y, u.y);
            u2.x = fma(c.d2v[l], yc.x, u2.x); u2.y = fma(c.d2v[l], yc.y, u2.y);
            mz.x = fma(c.v[l], yz.x, mz.x); mz.y = fma(c.v[l], yz.y, mz.y);
            md.x = fma(c.v[l], yd.x, md.x); md.y = fma(c.v[l], yd.y, md.y);
            {
                const double2 py = cconjmul(p, yc);  // zero for padding rows (c0, d0, kb are zero)
                add_term(l, kb.x * py.y - kb.y * py.x, -(c0.x * yc.x + c0.y * yc.y), -(d0.x * yc.x + d0.y * yc.y));
            }
        }
        if (in) {
            m.W[r] = w;
            m.U[r] = u;
            m.MZ[r] = mz;
            m.MDC[r] = md;
            s3 += c0.x * u2.x + c0.y * u2.y;
        }
    }
    __syncthreads();
    const double R = Yq[0], PP = Yq[3], mu = S.mu;
    const double h = 0.5 * PP / (mu * R * R);
    const double PRb = c.kb[1], PPb = c.kb[3];
    double s1 = 0.0, s2 = 0.0, s4 = 0.0;
    for (int r = tid; r < n; r += nt) {
        const int ru = S.up[r], rd = S.dn[r];
        const double au = S.aup[r], ad = S.adn[r];
        const double2 p = m.PH[S.lev[r]], kb = m.KB[r];
        const double2 kbu = m.KB[ru], kbd = m.KB[rd];
        const double2 wu = m.W[ru], wd = m.W[rd];
        const double2 Dkb = make_double2(ad * kbd.x - au * kbu.x, ad * kbd.y - au * kbu.y);
        const double2 Dw = make_double2(ad * wd.x - au * wu.x, ad * wd.y - au * wu.y);
        const double2 u = m.U[r], mz = m.MZ[r], md = m.MDC[r], dc = m.DC[r];
        // abar_in = i conj(p) M (p kbar) - h D kbar - 2 PRbar conj(p) u + PPhibar conj(p) (D w - M D c)
        const double2 imz = make_double2(-mz.y, mz.x);
        const double2 t1 = cconjmul(p, imz);
        const double2 t3 = cconjmul(p, u);
        const double2 t4 = cconjmul(p, make_double2(Dw.x - md.x, Dw.y - md.y));
        double2 o = m.YN[r];
        o.x += t1.x - h * Dkb.x - 2.0 * PRb * t3.x + PPb * t4.x;
        o.y += t1.y - h * Dkb.y - 2.0 * PRb * t3.y + PPb * t4.y;
        m.YN[r] = o;
        // s1 = Re(kbar^dag (-i conj(p) u)), s2 = Re(kbar^dag conj(p) Dc) = Re(kbar^dag D a),
        // s4 = -Re((Dc)^dag u)
        s1 += kb.x * t3.y - kb.y * t3.x;
        const double2 da = cconjmul(p, dc);
        s2 += kb.x * da.x + kb.y * da.y;
        s4 -= dc.x * u.x + dc.y * u.y;
    }
    // four scalar sums, then the per-term sums already held per warp in wred[warp][4 + ...]
    {
        double vals[4] = {s1, s2, s3, s4};
        for (int i = 0; i < 4; ++i) {
            const double sw = bsum_warp(vals[i]);
            if (lane == 0) wred[warp * kAdjRed + i] = sw;
        }
        __syncthreads();
        for (int i = tid; i < 4 + 3 * L; i += nt) {
            double sum = 0.0;
            for (int w2 = 0; w2 < nw; ++w2) sum += wred[w2 * kAdjRed + i];
            c.red[i] = sum;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double S1 = c.red[0], S2 = c.red[1], S3 = c.red[2], S4 = c.red[3];
        const double Rb = c.kb[0], Phb = c.kb[2];
        const double ir = 1.0 / R, ir2 = ir * ir, ir3 = ir2 * ir;
        c.ynew[0] += S1 - PP * ir3 / mu * S2 + PRb * (-S3 - 3.0 * PP * PP * ir2 * ir2 / mu) - 2.0 * PP * ir3 / mu * Phb +
                     PPb * S4;
        c.ynew[1] += Rb / mu;
        c.ynew[3] += 0.5 * S2 * ir2 / mu + PRb * 2.0 * PP * ir3 / mu + Phb * ir2 / mu;
        // parameters: sum_l dv_lp (alpha_l + PPhibar gamma_l) + d(dv)_lp PRbar beta_l
        for (int pp = 0; pp < S.P; ++pp) {
            double acc = 0.0;
            for (int l = 0; l < L; ++l) {
                const dbl4 q = S.dvcoef[((size_t)pp * L + l) * S.n_int + c.kint];
                const double x = c.x;
                const double dvl = q.x + x * (q.y + x * (q.z + x * q.w));
                const double ddvl = q.y + x * (2.0 * q.z + 3.0 * x * q.w);
                acc += dvl * (c.red[4 + 3 * l] + PPb * c.red[6 + 3 * l]) + ddvl * PRb * c.red[5 + 3 * l];
            }
            c.theta[pp] += acc;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kAdjThreads) k_adjoint_fp64(AdjArgs a)
{
    extern __shared__ double2 sm2[];
    __shared__ AdjCtl c;
    __shared__ DevSys S;
    __shared__ double wred[(kAdjThreads / 32) * kAdjRed];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) S = *a.sys;
    __syncthreads();
    const int n = S.n;
    AdjSmem m;
    m.A = sm2; m.Y2 = m.A + n; m.Y3 = m.Y2 + n; m.Y4 = m.Y3 + n; m.K = m.Y4 + n; m.ACC = m.K + n; m.C = m.ACC + n;
    m.W = m.C + n;
    m.LAM = m.W + n; m.KB = m.LAM + n; m.YN = m.KB + n; m.Z = m.YN + n; m.DC = m.Z + n; m.MZ = m.DC + n;
    m.MDC = m.MZ + n; m.U = m.MDC + n; m.PH = m.U + n;
    double *scr = a.scratch + (size_t)blockIdx.x * (size_t)(a.max_ckpt + a.K) * a.stride;
    double *ck = scr, *seg = scr + (size_t)a.max_ckpt * a.stride;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};

    for (;;) {
        if (tid == 0) c.item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = c.item;
        if (item >= a.n) break;
        const int t = item;
        const mqct_traj tr = a.trajs[t];
        const double dt = tr.dt;
        const int s0 = S.inv[tr.init_state];
        // ---- initial state
        for (int r = tid; r < n; r += nt) m.A[r] = make_double2(r == s0 ? 1.0 : 0.0, 0.0);
        if (tid == 0) {
            terms_at(S, tr.r0, c);
            double m00 = 0.0;
            for (int l = 0; l < S.L; ++l) m00 += c.v[l] * S.diag_g[(size_t)l * n + s0];
            const double lz = tr.b * sqrt(2.0 * S.mu * tr.e_coll);
            c.q[0] = tr.r0; c.q[2] = 0.0; c.q[3] = lz;
            c.q[1] = -sqrt(2.0 * S.mu * (tr.e_coll - m00) - lz * lz / (tr.r0 * tr.r0));
            c.p_r0 = c.q[1];
            c.steps = 0; c.status = 0;
            for (int pp = 0; pp < S.P; ++pp) c.theta[pp] = 0.0;
        }
        __syncthreads();
        // ---- forward with checkpoints
        auto store_state = [&](double *dst, const double2 *va, const double *q) {
            for (int r = tid; r < n; r += nt) { dst[2 * r] = va[r].x; dst[2 * r + 1] = va[r].y; }
            if (tid < 4) dst[2 * n + tid] = q[tid];
        };
        auto load_state = [&](const double *src, double2 *va, double *q) {
            for (int r = tid; r < n; r += nt) va[r] = make_double2(src[2 * r], src[2 * r + 1]);
            if (tid < 4) q[tid] = src[2 * n + tid];
        };
        // one forward RK4 step of (A, c.q); the stage states are left in Y2..Y4 / c.qk
        auto fwd_step = [&](int step) {
            const double t0 = step * dt;
            for (int s = 0; s < 4; ++s) {
                const double2 *Ya = s == 0 ? m.A : (s == 1 ? m.Y2 : (s == 2 ? m.Y3 : m.Y4));
                if (tid == 0) {
                    for (int i = 0; i < 4; ++i) c.qk[s][i] = s == 0 ? c.q[i] : c.qs[i];
                    terms_at(S, c.qk[s][0], c);
                }
                __syncthreads();
                fwd_eval(S, t0 + cst[s] * dt, Ya, c.qk[s], m, c, wred);
                const double wk = (s == 1 || s == 2) ? 2.0 : 1.0;
                double2 *Yn = s == 0 ? m.Y2 : (s == 1 ? m.Y3 : m.Y4);
                const double bn = s == 2 ? dt : 0.5 * dt;
                for (int r = tid; r < n; r += nt) {
                    const double2 k = m.K[r];
                    double2 acc = s == 0 ? make_double2(0, 0) : m.ACC[r];
                    acc.x = fma(wk, k.x, acc.x); acc.y = fma(wk, k.y, acc.y);
                    if (s < 3) {
                        m.ACC[r] = acc;
                        Yn[r] = make_double2(fma(bn, k.x, m.A[r].x), fma(bn, k.y, m.A[r].y));
                    } else {
                        m.A[r] = make_double2(fma(dt / 6.0, acc.x, m.A[r].x), fma(dt / 6.0, acc.y, m.A[r].y));
                    }
                }
                if (tid == 0) {
                    for (int i = 0; i < 4; ++i) c.lacc[i] = s == 0 ? c.lq[i] : fma(wk, c.lq[i], c.lacc[i]);
                    if (s < 3)
                        for (int i = 0; i < 4; ++i) c.qs[i] = fma(bn, c.lq[i], c.q[i]);
                    else
                        for (int i = 0; i < 4; ++i) c.q[i] = fma(dt / 6.0, c.lacc[i], c.q[i]);
                }
                __syncthreads();
            }
        };
        store_state(ck, m.A, c.q);
        bool done = tr.max_steps <= 0;
        while (!done) {
            fwd_step(c.steps);
            if (tid == 0) {
                c.steps += 1;
                const bool fin = isfinite(c.q[0]) && isfinite(c.q[1]) && isfinite(c.q[2]) && isfinite(c.q[3]);
                if (!fin) c.status |= MQCT_TRAJ_NONFINITE;
                if (c.steps >= tr.max_steps && !(fin && c.q[0] >= tr.r_end && c.q[1] > 0.0)) c.status |= MQCT_TRAJ_MAX_STEPS;
                if (c.steps % a.K == 0 && c.steps / a.K >= a.max_ckpt) c.status |= MQCT_TRAJ_CKPT;
            }
            __syncthreads();
            done = (c.status & (MQCT_TRAJ_NONFINITE | MQCT_TRAJ_MAX_STEPS | MQCT_TRAJ_CKPT)) ||
                   (c.q[0] >= tr.r_end && c.q[1] > 0.0);
            if (!done && c.steps % a.K == 0) store_state(ck + (size_t)(c.steps / a.K) * a.stride, m.A, c.q);
            __syncthreads();
        }
        const int N = c.steps;
        // ---- terminal cotangent: abar = 2 w dL/dsigma[g][level] a
        const int g = a.group[t];
        const double w = a.weight[t];
        const bool counted = g >= 0 && g < a.n_groups &&
                             !(c.status & (MQCT_TRAJ_NONFINITE | MQCT_TRAJ_MAX_STEPS | MQCT_TRAJ_CKPT));
        for (int r = tid; r < n; r += nt) {
            const double cf = counted ? 2.0 * w * a.dLds[(size_t)g * S.n_levels + S.lev[r]] : 0.0;
            m.LAM[r] = make_double2(cf * m.A[r].x, cf * m.A[r].y);
        }
        if (tid == 0) for (int i = 0; i < 4; ++i) c.lam[i] = 0.0;
        __syncthreads();
        // ---- reverse sweep, segment by segment
        if (counted) {
            for (int sg = (N - 1) / a.K; sg >= 0 && N > 0; --sg) {
                const int n0 = sg * a.K, n1 = N < n0 + a.K ? N : n0 + a.K;
                // recompute the segment's states y_n0 .. y_{n1-1} (y_n0 from the checkpoint)
                load_state(ck + (size_t)sg * a.stride, m.A, c.q);
                __syncthreads();
                for (int st = n0; st < n1; ++st) {
                    store_state(seg + (size_t)(st - n0) * a.stride, m.A, c.q);
                    __syncthreads();
                    if (st + 1 < n1) fwd_step(st);
                }
                for (int st = n1 - 1; st >= n0; --st) {
                    // stage states of step st
                    load_state(seg + (size_t)(st - n0) * a.stride, m.A, c.q);
                    __syncthreads();
                    fwd_step(st);  // leaves Y2..Y4 and c.qk; A now holds y_{st+1} (unused)
                    load_state(seg + (size_t)(st - n0) * a.stride, m.A, c.q);
                    __syncthreads();
                    // ynew = lam; kbar4 = dt/6 lam
                    for (int r = tid; r < n; r += nt) {
                        m.YN[r] = m.LAM[r];
                        m.KB[r] = make_double2(dt / 6.0 * m.LAM[r].x, dt / 6.0 * m.LAM[r].y);
                    }
                    if (tid == 0)
                        for (int i = 0; i < 4; ++i) { c.ynew[i] = c.lam[i]; c.kb[i] = dt / 6.0 * c.lam[i]; }
                    __syncthreads();
                    const double t0 = st * dt;
                    for (int s = 3; s >= 0; --s) {
                        const double2 *Ya = s == 0 ? m.A : (s == 1 ? m.Y2 : (s == 2 ? m.Y3 : m.Y4));
                        if (tid == 0) {
                            terms_at(S, c.qk[s][0], c);
                            for (int i = 0; i < 4; ++i) c.yb[i] = c.ynew[i];  // ynew before this stage
                        }
                        // keep ynew before this stage (K is free here) to form Ybar_s = after - before
                        for (int r = tid; r < n; r += nt) m.K[r] = m.YN[r];
                        __syncthreads();
                        vjp_eval(S, t0 + cst[s] * dt, Ya, c.qk[s], m, c, wred);
                        if (s > 0) {
                            // Ybar_s = YN - K(before); next kbar = wprev * lam + bprev * Ybar_s
                            const double wl = (s == 1) ? dt / 6.0 : dt / 3.0;
                            const double bl = (s == 3) ? dt : 0.5 * dt;
                            for (int r = tid; r < n; r += nt) {
                                const double2 yb = make_double2(m.YN[r].x - m.K[r].x, m.YN[r].y - m.K[r].y);
                                m.KB[r] = make_double2(fma(bl, yb.x, wl * m.LAM[r].x), fma(bl, yb.y, wl * m.LAM[r].y));
                            }
                            if (tid == 0)
                                for (int i = 0; i < 4; ++i) c.kb[i] = fma(bl, c.ynew[i] - c.yb[i], wl * c.lam[i]);
                            __syncthreads();
                        }
                    }
                    for (int r = tid; r < n; r += nt) m.LAM[r] = m.YN[r];
                    if (tid == 0) for (int i = 0; i < 4; ++i) c.lam[i] = c.ynew[i];
                    __syncthreads();
                }
            }
            // initial P_R = -sqrt(2 mu (E - M_ss(r0)) - L^2/r0^2): dP_R/dtheta = -mu dM_ss/dtheta / P_R
            if (tid == 0) {
                int k = (int)floor((tr.r0 - S.r_min) * S.inv_h);
                k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
                const double x = tr.r0 - (S.r_min + k * S.h);
                for (int pp = 0; pp < S.P; ++pp) {
                    double dm = 0.0;
                    for (int l = 0; l < S.L; ++l) {
                        const dbl4 q = S.dvcoef[((size_t)pp * S.L + l) * S.n_int + k];
                        dm += (q.x + x * (q.y + x * (q.z + x * q.w))) * S.diag_g[(size_t)l * n + s0];
                    }
                    c.theta[pp] += -S.mu * dm / c.p_r0 * c.lam[1];
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            for (int pp = 0; pp < S.P; ++pp) a.theta_traj[(size_t)t * S.P + pp] = counted ? c.theta[pp] : 0.0;
            a.status[t] = c.status;
        }
        __syncthreads();
    }
}

__global__ void k_sum_theta(const double *theta_traj, int n, int P, double *out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (int t = 0; t < n; ++t) s += theta_traj[(size_t)t * P + p];
    out[p] = s;
}

}  // namespace mqct

using namespace mqct;

namespace {
bool adj_is_dev(const void *p)
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

extern "C" mqct_status mqct_adjoint(mqct_system sys, const mqct_traj *trajs, int32_t n, const double *weight,
                                    const int32_t *group, int32_t n_groups, const double *dL_dsigma, int32_t ckpt,
                                    double *dL_dparam, void *cuda_stream)
{
    if (!sys || n < 0 || n_groups < 0 || ckpt < 1 || !dL_dparam) return fail(MQCT_ERR_INVALID_ARG, "mqct_adjoint: bad argument");
    const DevSys &h = sys->s.h;
    if (h.P < 1 || !h.dvcoef) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: the system has no parameter tables");
    if (h.P > kAdjMaxP) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: more than 32 parameters");
    if (h.L > kAdjMaxL) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: more than 16 expansion terms");
    if (h.precision != MQCT_FP64) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: FP64 systems only");
    if (n > 0 && (!trajs || !weight || !group || !dL_dsigma)) return fail(MQCT_ERR_INVALID_ARG, "mqct_adjoint: NULL input");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n == 0) {
        std::vector<double> z(h.P, 0.0);
        if (adj_is_dev(dL_dparam)) {
            cudaError_t e = cudaMemcpyAsync(dL_dparam, z.data(), sizeof(double) * h.P, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
            return MQCT_OK;
        }
        std::copy(z.begin(), z.end(), dL_dparam);
        return MQCT_OK;
    }
    const size_t smem = sizeof(double2) * (17 * (size_t)h.n + (size_t)h.n_levels);
    if (smem > 200 * 1024) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: basis too large for the adjoint kernel");
    // host copies of the trajectories (they also size the checkpoint storage)
    std::vector<mqct_traj> ht(n);
    cudaError_t e;
    if (adj_is_dev(trajs)) {
        if ((e = cudaMemcpy(ht.data(), trajs, sizeof(mqct_traj) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy");
    } else {
        std::copy(trajs, trajs + n, ht.begin());
    }
    for (int i = 0; i < n; ++i) {
        const mqct_traj &t = ht[i];
        if (t.system_idx != 0 || t.init_state < 0 || t.init_state >= h.n || !(t.dt > 0) || !(t.e_coll > 0) ||
            !(t.b >= 0) || !(t.r0 > t.b) || t.max_steps < 0 || !std::isfinite(t.r_end))
            return fail(MQCT_ERR_INVALID_ARG, "mqct_adjoint: invalid trajectory");
    }
    // forward step counts bound the checkpoint storage
    std::vector<mqct_diag> dg(n);
    {
        mqct_system one = sys;
        mqct_status s2 = mqct_propagate(&one, 1, ht.data(), n, nullptr, nullptr, dg.data(), cuda_stream);
        if (s2 != MQCT_OK && s2 != MQCT_ERR_TRAJ) return s2;
    }
    int max_steps = 1;
    for (auto &d : dg) max_steps = std::max(max_steps, d.steps);
    const int max_ckpt = max_steps / ckpt + 2;
    const size_t stride = (2 * (size_t)h.n + 4 + 3) & ~(size_t)3;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaFuncSetAttribute(k_adjoint_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_fp64, kAdjThreads, smem)) != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    const int grid = std::max(1, std::min(n, sms * std::max(per_sm, 1)));
    std::vector<void *> tmp;
    auto get = [&](void **p, size_t b) {
        cudaError_t r = cudaMallocAsync(p, b ? b : 16, st);
        if (r == cudaSuccess) tmp.push_back(*p);
        return r;
    };
    auto cleanup = [&]() { for (void *p : tmp) cudaFreeAsync(p, st); };
    auto stage = [&](const void *src, size_t bytes, const void **dst) -> cudaError_t {
        if (adj_is_dev(src)) { *dst = src; return cudaSuccess; }
        void *p = nullptr;
        cudaError_t r = get(&p, bytes);
        if (r != cudaSuccess) return r;
        r = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st);
        *dst = p;
        return r;
    };
    AdjArgs aa;
    const void *ptr = nullptr;
    aa.sys = sys->s.d;
    if ((e = stage(ht.data(), sizeof(mqct_traj) * n, &ptr)) != cudaSuccess) { cleanup(); return cuda_fail(e, "staging"); }
    aa.trajs = (const mqct_traj *)ptr;
    if ((e = stage(weight, sizeof(double) * n, &ptr)) != cudaSuccess) { cleanup(); return cuda_fail(e, "staging"); }
    aa.weight = (const double *)ptr;
    if ((e = stage(group, sizeof(int) * n, &ptr)) != cudaSuccess) { cleanup(); return cuda_fail(e, "staging"); }
    aa.group = (const int *)ptr;
    if ((e = stage(dL_dsigma, sizeof(double) * (size_t)std::max(n_groups, 1) * h.n_levels, &ptr)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "staging");
    }
    aa.dLds = (const double *)ptr;
    aa.n = n; aa.n_groups = n_groups; aa.K = ckpt; aa.max_ckpt = max_ckpt; aa.stride = stride;
    int *queue = nullptr;
    double *scratch = nullptr, *theta = nullptr, *out = nullptr;
    int *status = nullptr;
    if ((e = get((void **)&queue, sizeof(int))) != cudaSuccess ||
        (e = get((void **)&scratch, sizeof(double) * (size_t)grid * (max_ckpt + ckpt) * stride)) != cudaSuccess ||
        (e = get((void **)&theta, sizeof(double) * (size_t)n * h.P)) != cudaSuccess ||
        (e = get((void **)&status, sizeof(int) * (size_t)n)) != cudaSuccess ||
        (e = get((void **)&out, sizeof(double) * h.P)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync (adjoint scratch)");
    }
    aa.queue = queue; aa.scratch = scratch; aa.theta_traj = theta; aa.status = status;
    cudaMemsetAsync(queue, 0, sizeof(int), st);
    k_adjoint_fp64<<<grid, kAdjThreads, smem, st>>>(aa);
    k_sum_theta<<<1, 64, 0, st>>>(theta, n, h.P, out);
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_fail(e, "adjoint kernels"); }
    std::vector<int> hst(n);
    e = cudaMemcpyAsync(dL_dparam, out, sizeof(double) * h.P, adj_is_dev(dL_dparam) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), status, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int i = 0; i < n; ++i)
        if (hst[i] != 0 && hst[i] != MQCT_TRAJ_TABLE_RANGE)
            return fail(MQCT_ERR_TRAJ, "mqct_adjoint: a trajectory did not end normally (excluded from the gradient)");
    return MQCT_OK;
}
