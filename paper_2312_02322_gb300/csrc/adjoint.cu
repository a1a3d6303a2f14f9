// Discrete adjoint of the RK4 trajectory map: gradients of cross sections with respect to
// the PES expansion parameters theta (v_lambda(R) depends on theta through tables of
// d v_lambda / d theta_p given at create time).
//
// L = sum_{g,l} dL/dsigma[g][l] sigma[g][l],  sigma[g][l] = sum_{t in g} w_t sum_{s in l} |a_s|^2,
// so each trajectory starts the reverse sweep from abar_s = 2 w_t dL/dsigma[g_t][level(s)] a_s.
// One CTA per trajectory, the factorised coupling M(R) = sum_l v_l(R) G^l (Eq. 12):
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
//
// Two precisions of the amplitudes and cotangents (template parameter R): FP64 (FP64 systems;
// phase factors from FP64 sine and cosine, the same arithmetic as the FP64 forward kernel) and
// FP32 (mixed-precision systems: FP32 amplitudes, contraction and cotangents, phase arguments as
// 64-bit fixed-point turn counts, the step update of the amplitudes compensated as in the batched
// forward kernel; the classical variables, their cotangents and the parameter gradient stay FP64).
// The FP64 work that is not per element -- spline values of every term, the parameter
// gradient of each stage -- is spread over the lanes of a warp (one term or parameter per lane),
// since on this GPU one FP64 instruction holds its sub-partition's FP64 pipe for tens of cycles
// whatever the number of active lanes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "traj_common.cuh"

namespace mqct {

constexpr int kAdjThreads = 512;
constexpr int kAdjMaxP = 128;
constexpr int kAdjMaxL = 64;
constexpr int kAdjRed = 8 + 3 * kAdjMaxL;  // block-reduced scalars per VJP
constexpr int kAdjWarps = kAdjThreads / 32;

// complex numbers of the amplitude precision
template <class R>
struct Cx;
template <>
struct Cx<double> {
    using T = double2;
    static __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
};
template <>
struct Cx<float> {
    using T = float2;
    static __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
};

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
    unsigned char *scratch;   // per CTA: (max_ckpt + K) * stride bytes
    size_t stride;            // bytes per stored state
    unsigned char *vec;       // per CTA: vec_bytes of global memory for the work vectors when they do
    size_t vec_bytes;         //   not fit in shared memory (nullptr: shared memory)
    double *theta_traj;       // [n][P] per-trajectory gradient
    int *status;              // [n]
};

template <class R>
struct AdjCtl {
    double q[4], qs[4], lacc[4];   // classical state, stage input, accumulated derivatives
    double qk[4][4];               // classical stage states Y1..Y4 (R, PR, Phi, PPhi)
    double lq[4];                  // classical part of k (forward)
    double lam[4], kb[4], yb[4], ynew[4];  // classical cotangents
    R v[kAdjMaxL], dv[kAdjMaxL], d2v[kAdjMaxL];
    R vid, dvid;                   // sums of the identity terms' v and v'
    R hp, prb, ppb;                // dPhi/dt / 2 of the stage; P_R and P_Phi cotangents (amplitude precision)
    R ab[2][kAdjMaxL];             // per-term weights of the parameter gradient of one VJP
    double red[kAdjRed];
    double theta[kAdjMaxP];
    double p_r0;
    double x;                      // offset of R in its spline interval
    int steps, status, item, t, kint;
};

template <class R>
__device__ __forceinline__ R wsum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the warps of per-warp values wred[w * kAdjRed + i] (i < m) into c.red[i] (FP64); the
// FP32 variant sums compensated and converts once
template <class R>
__device__ void cross_warp(int m, AdjCtl<R> &c, const R *wred)
{
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    for (int i = tid; i < m; i += blockDim.x) {
        if constexpr (sizeof(R) == 8) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += wred[w * kAdjRed + i];
            c.red[i] = s;
        } else {
            float hi = 0.f, lo = 0.f;
            for (int w = 0; w < nw; ++w) {
                float e;
                two_sum(hi, wred[w * kAdjRed + i], hi, e);
                lo += e;
            }
            c.red[i] = (double)hi + (double)lo;
        }
    }
    __syncthreads();
}

// block-wide sums of m values held per thread (vals[0..m)); results in c.red[0..m)
template <class R>
__device__ void block_sums(const R *vals, int m, AdjCtl<R> &c, R *wred)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < m; ++i) {
        const R s = wsum(vals[i]);
        if (lane == 0) wred[warp * kAdjRed + i] = s;
    }
    __syncthreads();
    cross_warp(m, c, wred);
}

// warp 0: interval of R and v, v', v'' of every term (one term per lane), identity-term sums
template <class R>
__device__ void terms_at(const DevSys &S, double R_, AdjCtl<R> &c)
{
    const int lane = threadIdx.x & 31;
    int k;
    double x;
    bool below;
    locate_interval(S, R_, k, x, below);
    R vi = 0, dvi = 0;
    for (int l = lane; l < S.L; l += 32) {
        R v, dv, d2v;
        if constexpr (sizeof(R) == 8) {
            const dbl4 q = S.vcoef[(size_t)l * S.n_int + k];
            v = q.x + x * (q.y + x * (q.z + x * q.w));
            dv = q.y + x * (2.0 * q.z + 3.0 * x * q.w);
            d2v = 2.0 * q.z + 6.0 * x * q.w;
        } else {
            const float4 q = S.vcoef_f[(size_t)l * S.n_int + k];
            const float xf = (float)x;
            v = fmaf(xf, fmaf(xf, fmaf(xf, q.w, q.z), q.y), q.x);
            dv = fmaf(xf, fmaf(3.0f * xf, q.w, 2.0f * q.z), q.y);
            d2v = fmaf(6.0f * xf, q.w, 2.0f * q.z);
        }
        c.v[l] = v;
        c.dv[l] = dv;
        c.d2v[l] = d2v;
        if ((S.id_mask >> l) & 1ull) { vi += v; dvi += dv; }
    }
    vi = wsum(vi);
    dvi = wsum(dvi);
    if (lane == 0) {
        c.kint = k;
        c.x = x;
        c.vid = vi;
        c.dvid = dvi;
    }
    __syncwarp();
}

template <class R>
__device__ __forceinline__ typename Cx<R>::T cmul(typename Cx<R>::T a, typename Cx<R>::T b)
{
    return Cx<R>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R>
__device__ __forceinline__ typename Cx<R>::T cconjmul(typename Cx<R>::T a, typename Cx<R>::T b)  // conj(a) b
{
    return Cx<R>::mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

template <class R>
struct AdjSmem {
    using V = typename Cx<R>::T;
    V *A, *E, *Y2, *Y3, *Y4, *K, *ACC, *C, *W, *LAM, *KB, *YN, *Z, *DC, *MZ, *MDC, *U, *PH;
    unsigned long long *inc;  // FP32 variant: fixed-point phase increments per level
};

// phase factors exp(-i E_l t) of every level at stage time t = n_half dt / 2
template <class R>
__device__ void phases(const DevSys &S, double t, unsigned n_half, AdjSmem<R> &m)
{
    for (int l = threadIdx.x; l < S.n_levels; l += blockDim.x) {
        if constexpr (sizeof(R) == 8) {
            double sn, cs;
            sincos(S.lev_energy[l] * t, &sn, &cs);
            m.PH[l] = make_double2(cs, -sn);
        } else {
            m.PH[l] = phase_factor(m.inc[l], n_half);
        }
    }
}

// Forward right-hand side f(t, Y): K = da/dt, c.lq = classical derivatives.  Needs c.v/c.dv at
// the stage R (terms_at) and writes C = p Y, W = M c.
template <class R>
__device__ void fwd_eval(const DevSys &S, double t, unsigned n_half, const typename Cx<R>::T *Ya, const double *Yq,
                         AdjSmem<R> &m, AdjCtl<R> &c, R *wred)
{
    using V = typename Cx<R>::T;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = S.n;
    const double R_ = Yq[0], PR = Yq[1], PP = Yq[3];
    if (tid == 0) c.hp = (R)(0.5 * PP / (S.mu * R_ * R_));
    phases<R>(S, t, n_half, m);
    __syncthreads();
    for (int r = tid; r < n; r += nt) m.C[r] = cmul<R>(m.PH[S.lev[r]], Ya[r]);
    __syncthreads();
    R force = 0;
    const R vid = c.vid, dvid = c.dvid;
    for (int sl = warp; sl < S.n_slices; sl += nw) {
        const int r = sl * kSlice + lane;
        const V c0 = r < n ? m.C[r] : Cx<R>::mk(0, 0);
        V w = Cx<R>::mk(vid * c0.x, vid * c0.y), u = Cx<R>::mk(dvid * c0.x, dvid * c0.y);
        for (int f = 0; f < S.n_f; ++f) {
            const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
            const int off = so[sl], width = (so[sl + 1] - off) / kSlice;
            V y = Cx<R>::mk(0, 0);
            for (int k = 0; k < width; ++k) {
                R gv;
                if constexpr (sizeof(R) == 8) gv = S.f_val[off + k * kSlice + lane];
                else gv = S.f_valf[off + k * kSlice + lane];
                const V z = m.C[S.f_cols[off + k * kSlice + lane]];
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
    const R hp = c.hp;
    R torque = 0;
    for (int r = tid; r < n; r += nt) {
        const int ru = S.up[r], rd = S.dn[r];
        R au, ad;
        if constexpr (sizeof(R) == 8) { au = S.aup[r]; ad = S.adn[r]; }
        else { au = S.aupf[r]; ad = S.adnf[r]; }
        const V w = m.W[r], wu = m.W[ru], wd = m.W[rd], z = m.C[r];
        const V Dw = Cx<R>::mk(ad * wd.x - au * wu.x, ad * wd.y - au * wu.y);
        torque += z.x * Dw.x + z.y * Dw.y;
        const V y = Ya[ru], yd = Ya[rd];
        const V Dy = Cx<R>::mk(ad * yd.x - au * y.x, ad * yd.y - au * y.y);
        const V p = m.PH[S.lev[r]];
        V k;
        k.x = fma(hp, Dy.x, p.x * w.y - p.y * w.x);
        k.y = fma(hp, Dy.y, -(p.x * w.x + p.y * w.y));
        m.K[r] = k;
    }
    const R vals[2] = {force, torque};
    block_sums<R>(vals, 2, c, wred);
    if (tid == 0) {
        c.lq[0] = PR / S.mu;
        c.lq[1] = c.red[0] + PP * PP / (S.mu * R_ * R_ * R_);
        c.lq[2] = PP / (S.mu * R_ * R_);
        c.lq[3] = c.red[1];
    }
    __syncthreads();
}

// Vector-Jacobian product at stage (t, Y): given the cotangent (KB, c.kb) of f, add J^T kbar
// to (YN, c.ynew) and the parameter cotangent to c.theta.  Needs terms_at(Y_R).
template <class R>
__device__ void vjp_eval(const DevSys &S, double t, unsigned n_half, const typename Cx<R>::T *Ya, const double *Yq,
                         AdjSmem<R> &m, AdjCtl<R> &c, R *wred)
{
    using V = typename Cx<R>::T;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = S.n, L = S.L;
    const double R_ = Yq[0], PP = Yq[3], mu = S.mu;
    if (tid == 0) {
        c.hp = (R)(0.5 * PP / (mu * R_ * R_));
        c.prb = (R)c.kb[1];
        c.ppb = (R)c.kb[3];
    }
    phases<R>(S, t, n_half, m);
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        const V p = m.PH[S.lev[r]];
        m.C[r] = cmul<R>(p, Ya[r]);
        m.Z[r] = cmul<R>(p, m.KB[r]);
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        R au, ad;
        if constexpr (sizeof(R) == 8) { au = S.aup[r]; ad = S.adn[r]; }
        else { au = S.aupf[r]; ad = S.adnf[r]; }
        const V cu = m.C[S.up[r]], cd = m.C[S.dn[r]];
        m.DC[r] = Cx<R>::mk(ad * cd.x - au * cu.x, ad * cd.y - au * cu.y);
    }
    __syncthreads();
    // per-row contractions with every term: w = M c, u = M' c, u2 = M'' c, M z, M Dc, and the
    // per-term sums alpha_l = Re(kbar^dag (-i conj(p) G^l c)), beta_l = -Re(c^dag G^l c),
    // gamma_l = -Re((Dc)^dag G^l c)
    R *wt = wred + warp * kAdjRed;  // this warp's per-term sums (alpha, beta, gamma)
    for (int i = lane; i < 3 * L; i += 32) wt[4 + i] = 0;
    __syncwarp();
    // warp-reduce one term's three row contributions and add them to the warp's sums
    auto add_term = [&](int l, R a1, R b1, R g1) {
        a1 = wsum(a1); b1 = wsum(b1); g1 = wsum(g1);
        if (lane == 0) { wt[4 + 3 * l] += a1; wt[5 + 3 * l] += b1; wt[6 + 3 * l] += g1; }
    };
    R s3 = 0;  // Re(c^dag M'' c)
    for (int sl = warp; sl < S.n_slices; sl += nw) {
        const int r = sl * kSlice + lane;
        const bool in = r < n;
        const V c0 = in ? m.C[r] : Cx<R>::mk(0, 0), z0 = in ? m.Z[r] : Cx<R>::mk(0, 0);
        const V d0 = in ? m.DC[r] : Cx<R>::mk(0, 0), kb = in ? m.KB[r] : Cx<R>::mk(0, 0);
        const V p = in ? m.PH[S.lev[r]] : Cx<R>::mk(1, 0);
        V w = Cx<R>::mk(0, 0), u = w, u2 = w, mz = w, md = w;
        for (int l = 0; l < L; ++l) {
            if (!((S.id_mask >> l) & 1ull)) continue;
            w.x += c.v[l] * c0.x; w.y += c.v[l] * c0.y;
            u.x += c.dv[l] * c0.x; u.y += c.dv[l] * c0.y;
            u2.x += c.d2v[l] * c0.x; u2.y += c.d2v[l] * c0.y;
            mz.x += c.v[l] * z0.x; mz.y += c.v[l] * z0.y;
            md.x += c.v[l] * d0.x; md.y += c.v[l] * d0.y;
            const V py = cconjmul<R>(p, c0);  // conj(p) Y with Y = c
            add_term(l, kb.x * py.y - kb.y * py.x, -(c0.x * c0.x + c0.y * c0.y), -(d0.x * c0.x + d0.y * c0.y));
        }
        for (int f = 0; f < S.n_f; ++f) {
            const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
            const int off = so[sl], width = (so[sl + 1] - off) / kSlice;
            V yc = Cx<R>::mk(0, 0), yz = yc, yd = yc;
            for (int k = 0; k < width; ++k) {
                const int e = off + k * kSlice + lane;
                R gv;
                if constexpr (sizeof(R) == 8) gv = S.f_val[e];
                else gv = S.f_valf[e];
                const int col = S.f_cols[e];
                const V a1 = m.C[col], a2 = m.Z[col], a3 = m.DC[col];
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
                const V py = cconjmul<R>(p, yc);  // zero for padding rows (c0, d0, kb are zero)
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
    const R h = c.hp, PRb = c.prb, PPb = c.ppb;
    R s1 = 0, s2 = 0, s4 = 0;
    for (int r = tid; r < n; r += nt) {
        const int ru = S.up[r], rd = S.dn[r];
        R au, ad;
        if constexpr (sizeof(R) == 8) { au = S.aup[r]; ad = S.adn[r]; }
        else { au = S.aupf[r]; ad = S.adnf[r]; }
        const V p = m.PH[S.lev[r]], kb = m.KB[r];
        const V kbu = m.KB[ru], kbd = m.KB[rd];
        const V wu = m.W[ru], wd = m.W[rd];
        const V Dkb = Cx<R>::mk(ad * kbd.x - au * kbu.x, ad * kbd.y - au * kbu.y);
        const V Dw = Cx<R>::mk(ad * wd.x - au * wu.x, ad * wd.y - au * wu.y);
        const V u = m.U[r], mz = m.MZ[r], md = m.MDC[r], dc = m.DC[r];
        // abar_in = i conj(p) M (p kbar) - h D kbar - 2 PRbar conj(p) u + PPhibar conj(p) (D w - M D c)
        const V imz = Cx<R>::mk(-mz.y, mz.x);
        const V t1 = cconjmul<R>(p, imz);
        const V t3 = cconjmul<R>(p, u);
        const V t4 = cconjmul<R>(p, Cx<R>::mk(Dw.x - md.x, Dw.y - md.y));
        V o = m.YN[r];
        o.x += t1.x - h * Dkb.x - 2 * PRb * t3.x + PPb * t4.x;
        o.y += t1.y - h * Dkb.y - 2 * PRb * t3.y + PPb * t4.y;
        m.YN[r] = o;
        // s1 = Re(kbar^dag (-i conj(p) u)), s2 = Re(kbar^dag conj(p) Dc) = Re(kbar^dag D a),
        // s4 = -Re((Dc)^dag u)
        s1 += kb.x * t3.y - kb.y * t3.x;
        const V da = cconjmul<R>(p, dc);
        s2 += kb.x * da.x + kb.y * da.y;
        s4 -= dc.x * u.x + dc.y * u.y;
    }
    // four scalar sums, then the per-term sums already held per warp in wred[warp][4 + ...]
    {
        const R vals[4] = {s1, s2, s3, s4};
        for (int i = 0; i < 4; ++i) {
            const R sw = wsum(vals[i]);
            if (lane == 0) wred[warp * kAdjRed + i] = sw;
        }
        __syncthreads();
        cross_warp(4 + 3 * L, c, wred);
    }
    if (tid == 0) {
        const double S1 = c.red[0], S2 = c.red[1], S3 = c.red[2], S4 = c.red[3];
        const double Rb = c.kb[0], Phb = c.kb[2], PRbd = c.kb[1], PPbd = c.kb[3];
        const double ir = 1.0 / R_, ir2 = ir * ir, ir3 = ir2 * ir;
        c.ynew[0] += S1 - PP * ir3 / mu * S2 + PRbd * (-S3 - 3.0 * PP * PP * ir2 * ir2 / mu) - 2.0 * PP * ir3 / mu * Phb +
                     PPbd * S4;
        c.ynew[1] += Rb / mu;
        c.ynew[3] += 0.5 * S2 * ir2 / mu + PRbd * 2.0 * PP * ir3 / mu + Phb * ir2 / mu;
    }
    // parameters: sum_l dv_lp (alpha_l + PPhibar gamma_l) + d(dv)_lp PRbar beta_l, with the per-term
    // weights formed once (one term per thread), then one parameter per warp, one term per lane
    for (int l = tid; l < L; l += nt) {
        c.ab[0][l] = (R)(c.red[4 + 3 * l] + c.kb[3] * c.red[6 + 3 * l]);
        c.ab[1][l] = (R)(c.kb[1] * c.red[5 + 3 * l]);
    }
    __syncthreads();
    {
        const int k = c.kint;
        const double x = c.x;
        for (int pp = warp; pp < S.P; pp += nw) {
            R acc = 0;
            for (int l = lane; l < L; l += 32) {
                if constexpr (sizeof(R) == 8) {
                    const dbl4 q = S.dvcoef[((size_t)pp * L + l) * S.n_int + k];
                    const double dvl = q.x + x * (q.y + x * (q.z + x * q.w));
                    const double ddvl = q.y + x * (2.0 * q.z + 3.0 * x * q.w);
                    acc += dvl * c.ab[0][l] + ddvl * c.ab[1][l];
                } else {
                    const float4 q = S.dvcoef_f[((size_t)pp * L + l) * S.n_int + k];
                    const float xf = (float)x;
                    const float dvl = fmaf(xf, fmaf(xf, fmaf(xf, q.w, q.z), q.y), q.x);
                    const float ddvl = fmaf(xf, fmaf(3.0f * xf, q.w, 2.0f * q.z), q.y);
                    acc += dvl * c.ab[0][l] + ddvl * c.ab[1][l];
                }
            }
            acc = wsum(acc);
            if (lane == 0) c.theta[pp] += (double)acc;
        }
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint(AdjArgs a)
{
    using V = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ AdjCtl<R> c;
    __shared__ DevSys S;
    __shared__ R wred[kAdjWarps * kAdjRed];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) S = *a.sys;
    __syncthreads();
    const int n = S.n;
    AdjSmem<R> m;
    m.inc = reinterpret_cast<unsigned long long *>(smraw);
    V *base = a.vec ? reinterpret_cast<V *>(a.vec + (size_t)blockIdx.x * a.vec_bytes)
                    : reinterpret_cast<V *>(m.inc + (sizeof(R) == 4 ? ((S.n_levels + 1) & ~1) : 0));
    m.A = base; m.E = m.A + n; m.Y2 = m.E + n; m.Y3 = m.Y2 + n; m.Y4 = m.Y3 + n; m.K = m.Y4 + n; m.ACC = m.K + n;
    m.C = m.ACC + n; m.W = m.C + n; m.LAM = m.W + n; m.KB = m.LAM + n; m.YN = m.KB + n; m.Z = m.YN + n;
    m.DC = m.Z + n; m.MZ = m.DC + n; m.MDC = m.MZ + n; m.U = m.MDC + n; m.PH = m.U + n;
    unsigned char *scr = a.scratch + (size_t)blockIdx.x * (size_t)(a.max_ckpt + a.K) * a.stride;
    unsigned char *ck = scr, *seg = scr + (size_t)a.max_ckpt * a.stride;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    const unsigned hst[4] = {0u, 1u, 1u, 2u};
    constexpr bool fp32 = sizeof(R) == 4;
    // stored state: amplitudes A (and, FP32, the compensation E) then the classical q (FP64)
    const size_t amp_bytes = ((fp32 ? 2 : 1) * 2 * (size_t)n * sizeof(R) + 15) & ~(size_t)15;

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
        for (int r = tid; r < n; r += nt) {
            m.A[r] = Cx<R>::mk(r == s0 ? 1 : 0, 0);
            m.E[r] = Cx<R>::mk(0, 0);
        }
        if (fp32)
            for (int l = tid; l < S.n_levels; l += nt) m.inc[l] = phase_increment(S.lev_energy[l], dt);
        if (tid == 0) {
            int k;
            double x;
            bool below;
            locate_interval(S, tr.r0, k, x, below);
            double m00 = 0.0;
            for (int l = 0; l < S.L; ++l) m00 += spline_fp64(S, l, k, x) * S.diag_g[(size_t)l * n + s0];
            initial_state(S, tr, m00, c.q);
            c.p_r0 = c.q[1];
            c.steps = 0; c.status = 0;
            for (int pp = 0; pp < S.P; ++pp) c.theta[pp] = 0.0;
        }
        __syncthreads();
        // ---- forward with checkpoints
        auto store_state = [&](unsigned char *dst, const double *q) {
            R *da = reinterpret_cast<R *>(dst);
            for (int r = tid; r < n; r += nt) {
                da[2 * r] = m.A[r].x; da[2 * r + 1] = m.A[r].y;
                if (fp32) { da[2 * n + 2 * r] = m.E[r].x; da[2 * n + 2 * r + 1] = m.E[r].y; }
            }
            if (tid < 4) reinterpret_cast<double *>(dst + amp_bytes)[tid] = q[tid];
        };
        auto load_state = [&](const unsigned char *src, double *q) {
            const R *sa = reinterpret_cast<const R *>(src);
            for (int r = tid; r < n; r += nt) {
                m.A[r] = Cx<R>::mk(sa[2 * r], sa[2 * r + 1]);
                m.E[r] = fp32 ? Cx<R>::mk(sa[2 * n + 2 * r], sa[2 * n + 2 * r + 1]) : Cx<R>::mk(0, 0);
            }
            if (tid < 4) q[tid] = reinterpret_cast<const double *>(src + amp_bytes)[tid];
        };
        // one forward RK4 step of (A, c.q); the stage states are left in Y2..Y4 / c.qk
        auto fwd_step = [&](int step) {
            const double t0 = step * dt;
            for (int s = 0; s < 4; ++s) {
                const V *Ya = s == 0 ? m.A : (s == 1 ? m.Y2 : (s == 2 ? m.Y3 : m.Y4));
                if (warp == 0) {
                    if (lane == 0)
                        for (int i = 0; i < 4; ++i) c.qk[s][i] = s == 0 ? c.q[i] : c.qs[i];
                    __syncwarp();
                    terms_at<R>(S, c.qk[s][0], c);
                }
                __syncthreads();
                fwd_eval<R>(S, t0 + cst[s] * dt, 2u * step + hst[s], Ya, c.qk[s], m, c, wred);
                const R wk = (s == 1 || s == 2) ? 2 : 1;
                V *Yn = s == 0 ? m.Y2 : (s == 1 ? m.Y3 : m.Y4);
                const R bn = s == 2 ? (R)dt : (R)(0.5 * dt);
                for (int r = tid; r < n; r += nt) {
                    const V k = m.K[r];
                    V acc = s == 0 ? Cx<R>::mk(0, 0) : m.ACC[r];
                    acc.x = fma(wk, k.x, acc.x); acc.y = fma(wk, k.y, acc.y);
                    if (s < 3) {
                        m.ACC[r] = acc;
                        Yn[r] = Cx<R>::mk(fma(bn, k.x, m.A[r].x), fma(bn, k.y, m.A[r].y));
                    } else if constexpr (fp32) {
                        // compensated a + (dt/6) acc: the rounding error of each update is carried
                        // in E into the next one
                        const float h6 = (float)(dt / 6.0);
                        const V a0 = m.A[r], e0 = m.E[r];
                        float sx, sy, ex, ey;
                        two_sum(a0.x, fmaf(h6, acc.x, e0.x), sx, ex);
                        two_sum(a0.y, fmaf(h6, acc.y, e0.y), sy, ey);
                        m.A[r] = make_float2(sx, sy);
                        m.E[r] = make_float2(ex, ey);
                    } else {
                        m.A[r] = Cx<R>::mk(fma(dt / 6.0, acc.x, m.A[r].x), fma(dt / 6.0, acc.y, m.A[r].y));
                    }
                }
                if (tid == 0) {
                    for (int i = 0; i < 4; ++i) c.lacc[i] = s == 0 ? c.lq[i] : fma((double)wk, c.lq[i], c.lacc[i]);
                    if (s < 3)
                        for (int i = 0; i < 4; ++i) c.qs[i] = fma(s == 2 ? dt : 0.5 * dt, c.lq[i], c.q[i]);
                    else
                        for (int i = 0; i < 4; ++i) c.q[i] = fma(dt / 6.0, c.lacc[i], c.q[i]);
                }
                __syncthreads();
            }
        };
        store_state(ck, c.q);
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
            if (!done && c.steps % a.K == 0) store_state(ck + (size_t)(c.steps / a.K) * a.stride, c.q);
            __syncthreads();
        }
        const int N = c.steps;
        // ---- terminal cotangent: abar = 2 w dL/dsigma[g][level] a
        const int g = a.group[t];
        const double w = a.weight[t];
        const bool counted = g >= 0 && g < a.n_groups &&
                             !(c.status & (MQCT_TRAJ_NONFINITE | MQCT_TRAJ_MAX_STEPS | MQCT_TRAJ_CKPT));
        for (int r = tid; r < n; r += nt) {
            const R cf = counted ? (R)(2.0 * w * a.dLds[(size_t)g * S.n_levels + S.lev[r]]) : (R)0;
            m.LAM[r] = Cx<R>::mk(cf * m.A[r].x, cf * m.A[r].y);
        }
        if (tid == 0) for (int i = 0; i < 4; ++i) c.lam[i] = 0.0;
        __syncthreads();
        // ---- reverse sweep, segment by segment
        if (counted) {
            for (int sg = (N - 1) / a.K; sg >= 0 && N > 0; --sg) {
                const int n0 = sg * a.K, n1 = N < n0 + a.K ? N : n0 + a.K;
                // recompute the segment's states y_n0 .. y_{n1-1} (y_n0 from the checkpoint)
                load_state(ck + (size_t)sg * a.stride, c.q);
                __syncthreads();
                for (int st = n0; st < n1; ++st) {
                    store_state(seg + (size_t)(st - n0) * a.stride, c.q);
                    __syncthreads();
                    if (st + 1 < n1) fwd_step(st);
                }
                for (int st = n1 - 1; st >= n0; --st) {
                    // stage states of step st
                    load_state(seg + (size_t)(st - n0) * a.stride, c.q);
                    __syncthreads();
                    fwd_step(st);  // leaves Y2..Y4 and c.qk; A now holds y_{st+1} (unused)
                    load_state(seg + (size_t)(st - n0) * a.stride, c.q);
                    __syncthreads();
                    // ynew = lam; kbar4 = dt/6 lam
                    const R h6 = (R)(dt / 6.0);
                    for (int r = tid; r < n; r += nt) {
                        m.YN[r] = m.LAM[r];
                        m.KB[r] = Cx<R>::mk(h6 * m.LAM[r].x, h6 * m.LAM[r].y);
                    }
                    if (tid == 0)
                        for (int i = 0; i < 4; ++i) { c.ynew[i] = c.lam[i]; c.kb[i] = dt / 6.0 * c.lam[i]; }
                    __syncthreads();
                    const double t0 = st * dt;
                    for (int s = 3; s >= 0; --s) {
                        const V *Ya = s == 0 ? m.A : (s == 1 ? m.Y2 : (s == 2 ? m.Y3 : m.Y4));
                        if (warp == 0) {
                            terms_at<R>(S, c.qk[s][0], c);
                            if (lane == 0)
                                for (int i = 0; i < 4; ++i) c.yb[i] = c.ynew[i];  // ynew before this stage
                        }
                        // keep ynew before this stage (K is free here) to form Ybar_s = after - before
                        for (int r = tid; r < n; r += nt) m.K[r] = m.YN[r];
                        __syncthreads();
                        vjp_eval<R>(S, t0 + cst[s] * dt, 2u * st + hst[s], Ya, c.qk[s], m, c, wred);
                        if (s > 0) {
                            // Ybar_s = YN - K(before); next kbar = wprev * lam + bprev * Ybar_s
                            const double wl = (s == 1) ? dt / 6.0 : dt / 3.0;
                            const double bl = (s == 3) ? dt : 0.5 * dt;
                            const R wlr = (R)wl, blr = (R)bl;
                            for (int r = tid; r < n; r += nt) {
                                const V yb = Cx<R>::mk(m.YN[r].x - m.K[r].x, m.YN[r].y - m.K[r].y);
                                m.KB[r] = Cx<R>::mk(fma(blr, yb.x, wlr * m.LAM[r].x), fma(blr, yb.y, wlr * m.LAM[r].y));
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
                int k;
                double x;
                bool below;
                locate_interval(S, tr.r0, k, x, below);
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
        for (int pp = tid; pp < S.P; pp += nt) a.theta_traj[(size_t)t * S.P + pp] = counted ? c.theta[pp] : 0.0;
        if (tid == 0) a.status[t] = c.status;
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
    reset_launches();
    if (sys && sys->s.h.grid_log) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: the logarithmic grid is not supported");
    if (!sys || n < 0 || n_groups < 0 || ckpt < 1 || !dL_dparam) return fail(MQCT_ERR_INVALID_ARG, "mqct_adjoint: bad argument");
    const DevSys &h = sys->s.h;
    if (h.P < 1 || !h.dvcoef) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: the system has no parameter tables");
    if (h.P > kAdjMaxP) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: more than 128 parameters");
    if (h.L > kAdjMaxL) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: more than 64 expansion terms");
    if (h.path != MQCT_PATH_FACTORISED)
        return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: the system must use the factorised path");
    if (h.adapt_tol > 0.0) return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: fixed steps only (adapt_tol > 0)");
    if (h.flags & (MQCT_PRESCRIBED_TRAJ | MQCT_DECOUPLED_TRAJ))
        return fail(MQCT_ERR_UNSUPPORTED, "mqct_adjoint: not defined for prescribed or decoupled trajectories");
    const bool fp32 = h.precision != MQCT_FP64;
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
    // a stored state: amplitudes (FP32: and their compensation terms), then 4 classical doubles
    const size_t rsz = fp32 ? sizeof(float) : sizeof(double);
    const size_t amp_bytes = ((fp32 ? 4 : 2) * (size_t)h.n * rsz + 15) & ~(size_t)15;
    const size_t stride = amp_bytes + 32;
    // work vectors: 17 of length N and the phase factors of every level, in shared memory when
    // they fit, else in a global-memory region per CTA
    const size_t vsz = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t inc_bytes = fp32 ? 8 * (size_t)((h.n_levels + 1) & ~1) : 0;
    const size_t vec_bytes = ((17 * (size_t)h.n + h.n_levels) * vsz + 255) & ~(size_t)255;
    const void *kern = fp32 ? (const void *)k_adjoint<float> : (const void *)k_adjoint<double>;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    int dev = 0, sms = 0, per_sm = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool vec_global = fa.sharedSizeBytes + inc_bytes + vec_bytes > (size_t)smem_optin;
    const size_t smem = inc_bytes + (vec_global ? 0 : vec_bytes);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, smem)) != cudaSuccess)
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
    unsigned char *scratch = nullptr, *vec = nullptr;
    double *theta = nullptr, *out = nullptr;
    int *status = nullptr;
    if ((e = get((void **)&queue, sizeof(int))) != cudaSuccess ||
        (e = get((void **)&scratch, (size_t)grid * (max_ckpt + ckpt) * stride)) != cudaSuccess ||
        (vec_global && (e = get((void **)&vec, (size_t)grid * vec_bytes)) != cudaSuccess) ||
        (e = get((void **)&theta, sizeof(double) * (size_t)n * h.P)) != cudaSuccess ||
        (e = get((void **)&status, sizeof(int) * (size_t)n)) != cudaSuccess ||
        (e = get((void **)&out, sizeof(double) * h.P)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync (adjoint scratch)");
    }
    aa.queue = queue; aa.scratch = scratch; aa.theta_traj = theta; aa.status = status;
    aa.vec = vec; aa.vec_bytes = vec_bytes;
    cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (fp32) k_adjoint<float><<<grid, kAdjThreads, smem, st>>>(aa);
    else k_adjoint<double><<<grid, kAdjThreads, smem, st>>>(aa);
    k_sum_theta<<<(h.P + 63) / 64, 64, 0, st>>>(theta, n, h.P, out);
    count_launches(2);
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
