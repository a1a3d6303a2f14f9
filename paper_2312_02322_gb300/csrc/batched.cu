// Batched mixed-precision trajectory kernel (factorised path, FP32 amplitudes).
//
// One CTA integrates B trajectories at once: their phase-rotated stage amplitudes form the
// N x B block C (one column per trajectory, FP32 complex, shared memory, row-major so that a
// row of four columns is 32 contiguous bytes).  A thread owns units (row r, 4 columns); the
// sparse G entries of a row are loaded once and applied to the four columns.  Per RK4 stage:
//   P3  contraction: for every stored term lambda, Y_lambda = G^lambda C, combined per column
//       with the FP32 spline values v_lambda(R_b), v_lambda'(R_b):  w = M(R_b) c_b and
//       u = M'(R_b) c_b   (Eq. 12); Coriolis stencil Dc_b = (J+ - J-) c_b; partial sums of
//       the force -Re(c^dag u), the torque Re(c^dag D w) = -Re((Dc)^dag w) and (stage 0)
//       Re(c^dag w);
//   P4  derivative assembly da/dt = -i exp(iEt) w + (dPhi/dt/2) exp(iEt) Dc   (Eq. 5, using
//       that Coriolis partners share the level energy), RK4 accumulation and next stage input;
//       the step update a + (dt/6) acc is compensated (two-sum), its rounding error carried
//       into the next step's accumulator;
//   C   one lane per trajectory: FP64 classical stage update (Eqs. 7-10), FP64 bookkeeping of
//       norm, total energy and P_Phi + <J_y>, termination, and refill of the slot from the
//       device work queue (trajectories of uneven length share a CTA).
// Phase factors exp(-i E_l t) per level and slot: argument E_l t and its reduction modulo
// 2 pi in FP64, sine and cosine of the reduced angle in FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace mqct {

constexpr int kUpt = 4;  // (row, 4-column) units per thread

enum { SLOT_IDLE = 0, SLOT_ACTIVE = 1, SLOT_FINAL = 2, SLOT_WAIT = 3 };

struct Slot {
    double q[4], qs[4], lacc[4];
    double dt, r_end, e0, j0, ndev, edev, jdev, x, phidot, inv_mu;
    int kint, status, steps, max_steps, traj, state, s0;
};

__device__ __forceinline__ float2 phase_of(double e, double t)
{
    const double two_pi_hi = 6.283185307179586232, two_pi_lo = 2.4492935982947064e-16;
    double th = e * t;
    double k = rint(th * 0.15915494309189535);
    double r = fma(-k, two_pi_hi, th);
    r = fma(-k, two_pi_lo, r);
    float s, c;
    sincosf((float)r, &s, &c);
    return make_float2(c, -s);
}

__device__ __forceinline__ void locate_slot(const DevSys &S, Slot &sl)
{
    const double R = sl.qs[0];
    int k = (int)floor((R - S.r_min) * S.inv_h);
    k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
    sl.kint = k;
    sl.x = R - (S.r_min + k * S.h);
    const double ir = 1.0 / R;
    sl.phidot = sl.qs[3] * sl.inv_mu * ir * ir;
    if (R < S.r_min) sl.status |= MQCT_TRAJ_TABLE_RANGE;
}

// slot lane: claim the next valid trajectory (FP64 initial conditions)
__device__ void claim(const BatchArgs &a, const DevSys &S, Slot &sl)
{
    for (;;) {
        const int item = atomicAdd(a.queue, 1);
        if (item >= a.n) {
            sl.state = SLOT_IDLE;
            return;
        }
        const int t = a.order ? a.order[item] : item;
        const mqct_traj tr = a.trajs[t];
        const bool ok = tr.system_idx == a.sys_idx && tr.dt > 0.0 && tr.e_coll > 0.0 && tr.b >= 0.0 && tr.r0 > 0.0 &&
                        tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0 && tr.init_state >= 0 &&
                        tr.init_state < S.n;
        if (!ok) {
            if (a.diag) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                a.diag[t] = d;
            }
            continue;
        }
        if (a.t_start) a.t_start[t] = mqct_clock_ns();
        const int s0 = S.inv[tr.init_state];
        int k = (int)floor((tr.r0 - S.r_min) * S.inv_h);
        k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
        const double x = tr.r0 - (S.r_min + k * S.h);
        double m00 = 0.0;
        for (int l = 0; l < S.L; ++l) {
            const dbl4 c = S.vcoef[(size_t)l * S.n_int + k];
            m00 += (c.x + x * (c.y + x * (c.z + x * c.w))) * S.diag_g[(size_t)l * S.n + s0];
        }
        const double lz = tr.b * sqrt(2.0 * S.mu * tr.e_coll);
        sl.q[0] = tr.r0; sl.q[2] = 0.0; sl.q[3] = lz;
        sl.q[1] = -sqrt(2.0 * S.mu * (tr.e_coll - m00) - lz * lz / (tr.r0 * tr.r0));
        for (int i = 0; i < 4; ++i) sl.qs[i] = sl.q[i];
        sl.dt = tr.dt; sl.r_end = tr.r_end; sl.max_steps = tr.max_steps;
        sl.ndev = sl.edev = sl.jdev = 0.0;
        sl.inv_mu = 1.0 / S.mu;
        sl.status = 0; sl.steps = 0; sl.traj = t; sl.s0 = s0;
        sl.state = SLOT_WAIT;
        sl.kint = k; sl.x = x; sl.phidot = 0.0;
        return;
    }
}

struct F4x2 {  // four complex FP32 values (one unit row of four columns)
    float2 v[4];
};

__device__ __forceinline__ F4x2 ld4(const float2 *p)
{
    const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    F4x2 r;
    r.v[0] = make_float2(a.x, a.y); r.v[1] = make_float2(a.z, a.w);
    r.v[2] = make_float2(b.x, b.y); r.v[3] = make_float2(b.z, b.w);
    return r;
}

__device__ __forceinline__ void st4(float2 *p, const F4x2 &r)
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(r.v[0].x, r.v[0].y, r.v[1].x, r.v[1].y);
    reinterpret_cast<float4 *>(p)[1] = make_float4(r.v[2].x, r.v[2].y, r.v[3].x, r.v[3].y);
}

template <int B, int T>
__global__ void __launch_bounds__(T, 512 / T) k_batched_f32(BatchArgs a)
{
    static_assert(B % 4 == 0 && B <= 32, "batch width");
    constexpr int G4 = B / 4;  // four-column groups per row
    constexpr int NW = T / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ DevSys S;
    __shared__ Slot sl[B];
    __shared__ __align__(16) float vid[B];
    __shared__ __align__(16) float dvid[B];
    __shared__ __align__(16) float s_hp[B];
    __shared__ __align__(16) float s_dt[B];
    __shared__ int s_state[B], s_traj[B], s_s0[B];
    __shared__ double red2[B][6];
    __shared__ int s_live;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid % G4;
    if (tid == 0) S = *a.sys;
    __syncthreads();
    const int n = S.n, NL = S.n_levels, L = S.L;
    float2 *C = reinterpret_cast<float2 *>(smraw);
    float2 *A = C + (size_t)n * B, *ACC = A + (size_t)n * B;
    float2 *PHa = ACC + (size_t)n * B, *PHb = PHa + (size_t)NL * B;
    float *vv = reinterpret_cast<float *>(PHb + (size_t)NL * B), *dvv = vv + (size_t)L * B;
    double *red = reinterpret_cast<double *>(dvv + (size_t)L * B);  // [NW][B][6]
    const int upt = (n * G4 + T - 1) / T;

    // per-column views written by the slot lanes after every update
    auto publish = [&](int b) {
        const Slot &m = sl[b];
        s_hp[b] = (float)(0.5 * m.phidot);
        s_dt[b] = (float)m.dt;
        s_state[b] = m.state;
        s_traj[b] = m.traj;
        s_s0[b] = m.s0;
    };
    // v_lambda, v_lambda' at every running slot's stage R (FP32 spline, FP64-located interval)
    auto terms = [&]() {
        for (int i = tid; i < L * B; i += T) {
            const int l = i / B, bb = i % B;
            const Slot &s = sl[bb];
            if (s.state == SLOT_IDLE || s.state == SLOT_WAIT) { vv[i] = 0.f; dvv[i] = 0.f; continue; }
            const float4 c = S.vcoef_f[(size_t)l * S.n_int + s.kint];
            const float x = (float)s.x;
            vv[i] = fmaf(x, fmaf(x, fmaf(x, c.w, c.z), c.y), c.x);
            dvv[i] = fmaf(x, fmaf(3.0f * x, c.w, 2.0f * c.z), c.y);
        }
        __syncthreads();
        if (tid < B) {
            float v0 = 0.f, d0 = 0.f;
            for (int l = 0; l < L; ++l)
                if ((S.id_mask >> l) & 1ull) { v0 += vv[l * B + tid]; d0 += dvv[l * B + tid]; }
            vid[tid] = v0;
            dvid[tid] = d0;
        }
    };

    // ---- start: every slot claims a trajectory; columns e_s0, accumulators 0, phases 1
    if (tid < B) {
        claim(a, S, sl[tid]);
        publish(tid);
    }
    __syncthreads();
    for (int i = tid; i < n * B; i += T) {
        const int r = i / B, bb = i % B;
        if (s_state[bb] != SLOT_WAIT) continue;
        const float2 v = make_float2(r == s_s0[bb] ? 1.0f : 0.0f, 0.0f);
        A[i] = v; ACC[i] = make_float2(0.f, 0.f); C[i] = v;
    }
    for (int i = tid; i < NL * B; i += T) PHa[i] = make_float2(1.f, 0.f);
    __syncthreads();
    if (tid < B) {
        Slot &m = sl[tid];
        if (m.state == SLOT_WAIT) {
            m.state = m.max_steps > 0 ? SLOT_ACTIVE : SLOT_FINAL;
            if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
            locate_slot(S, m);
        }
        publish(tid);
    }
    if (tid == 0) s_live = 1;
    __syncthreads();
    terms();
    __syncthreads();

    while (s_live) {
        for (int s = 0; s < 4; ++s) {
            const float2 *PHc = (s == 0 || s == 3) ? PHa : PHb;
            const float2 *PHn = (s == 0 || s == 1) ? PHb : PHa;
            if (s == 0 || s == 2) {
                float2 *dst = s == 0 ? PHb : PHa;
                for (int i = tid; i < NL * B; i += T) {
                    const Slot &q = sl[i % B];
                    if (q.state != SLOT_ACTIVE) continue;
                    const double t = q.steps * q.dt + (s == 0 ? 0.5 * q.dt : q.dt);
                    dst[i] = phase_of(S.lev_energy[i / B], t);
                }
            }
            // column states of my group
            int cst[4];
            bool any = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cst[j] = s_state[4 * g + j];
                any |= cst[j] == SLOT_ACTIVE || cst[j] == SLOT_FINAL;
            }
            // ---- P3
            F4x2 kq[kUpt];  // derivative da/dt of the unit's four columns (Eq. 5)
            float fp[4] = {0, 0, 0, 0}, tp[4] = {0, 0, 0, 0}, vp[4] = {0, 0, 0, 0};
            float np_[4] = {0, 0, 0, 0}, ep[4] = {0, 0, 0, 0}, jp[4] = {0, 0, 0, 0};
            const float4 hp4 = reinterpret_cast<const float4 *>(s_hp)[g];
            const float hp[4] = {hp4.x, hp4.y, hp4.z, hp4.w};
#pragma unroll
            for (int k = 0; k < kUpt; ++k) {
                const int r = (tid + k * T) / G4;
                if (k >= upt || r >= n || !any) continue;
                const F4x2 c = ld4(C + (size_t)r * B + 4 * g);
                const float4 vi = reinterpret_cast<const float4 *>(vid)[g], dvi = reinterpret_cast<const float4 *>(dvid)[g];
                const float vi_[4] = {vi.x, vi.y, vi.z, vi.w}, dvi_[4] = {dvi.x, dvi.y, dvi.z, dvi.w};
                F4x2 w, u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    w.v[j] = make_float2(vi_[j] * c.v[j].x, vi_[j] * c.v[j].y);
                    u.v[j] = make_float2(dvi_[j] * c.v[j].x, dvi_[j] * c.v[j].y);
                }
                for (int f = 0; f < S.n_f; ++f) {
                    const int *ptr = S.csr_ptr + (size_t)f * (n + 1);
                    const int q0 = __ldg(ptr + r), q1 = __ldg(ptr + r + 1);
                    float2 y[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
                    // two entries per iteration: their loads are in flight together (same sum order)
#pragma unroll 2
                    for (int q = q0; q < q1; ++q) {
                        const int col = __ldg(S.csr_col + q);
                        const float gv = __ldg(S.csr_val + q);
                        const F4x2 z = ld4(C + (size_t)col * B + 4 * g);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            y[j].x = fmaf(gv, z.v[j].x, y[j].x);
                            y[j].y = fmaf(gv, z.v[j].y, y[j].y);
                        }
                    }
                    const int l = S.f_term[f];
                    const float4 v4 = reinterpret_cast<const float4 *>(vv + l * B)[g];
                    const float4 d4 = reinterpret_cast<const float4 *>(dvv + l * B)[g];
                    const float vl[4] = {v4.x, v4.y, v4.z, v4.w}, dl[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        w.v[j].x = fmaf(vl[j], y[j].x, w.v[j].x); w.v[j].y = fmaf(vl[j], y[j].y, w.v[j].y);
                        u.v[j].x = fmaf(dl[j], y[j].x, u.v[j].x); u.v[j].y = fmaf(dl[j], y[j].y, u.v[j].y);
                    }
                }
                const float au = __ldg(S.aupf + r), ad = __ldg(S.adnf + r);
                const F4x2 cu = ld4(C + (size_t)__ldg(S.up + r) * B + 4 * g);
                const F4x2 cd = ld4(C + (size_t)__ldg(S.dn + r) * B + 4 * g);
                const int lev = S.lev[r];
                const F4x2 p = ld4(PHc + (size_t)lev * B + 4 * g);
                F4x2 a0;
                if (s == 0) a0 = ld4(A + (size_t)r * B + 4 * g);
                const float elev = (float)S.lev_energy[lev];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 dc = make_float2(ad * cd.v[j].x - au * cu.v[j].x, ad * cd.v[j].y - au * cu.v[j].y);
                    const float2 wj = w.v[j], pj = p.v[j];
                    fp[j] -= c.v[j].x * u.v[j].x + c.v[j].y * u.v[j].y;
                    tp[j] -= dc.x * wj.x + dc.y * wj.y;
                    vp[j] += c.v[j].x * wj.x + c.v[j].y * wj.y;
                    // conj(p) Dc = (J+ - J-) a at this stage (partners share the level energy)
                    const float2 da = make_float2(pj.x * dc.x + pj.y * dc.y, pj.x * dc.y - pj.y * dc.x);
                    kq[k].v[j].x = fmaf(hp[j], da.x, pj.x * wj.y - pj.y * wj.x);
                    kq[k].v[j].y = fmaf(hp[j], da.y, -(pj.x * wj.x + pj.y * wj.y));
                    if (s == 0) {
                        const float2 aj = a0.v[j];
                        const float pp = aj.x * aj.x + aj.y * aj.y;
                        np_[j] += pp;
                        ep[j] += elev * pp;
                        jp[j] += aj.x * da.y - aj.y * da.x;
                    }
                }
            }
            __syncthreads();
            // ---- P4 (own units only)
            const float4 dt4 = reinterpret_cast<const float4 *>(s_dt)[g];
            const float dtj[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
            const float wgt = (s == 1 || s == 2) ? 2.0f : 1.0f;
#pragma unroll
            for (int k = 0; k < kUpt; ++k) {
                const int r = (tid + k * T) / G4;
                if (k >= upt || r >= n) continue;
                const size_t o = (size_t)r * B + 4 * g;
                const int lev = S.lev[r];
                F4x2 a0 = ld4(A + o), acc = ld4(ACC + o), cn = ld4(C + o);
                const F4x2 pn = ld4(PHn + (size_t)lev * B + 4 * g);
                bool wr_a = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int stj = cst[j];
                    if (stj == SLOT_WAIT) {
                        if (s == 3) {
                            const float2 v = make_float2(r == s_s0[4 * g + j] ? 1.0f : 0.0f, 0.0f);
                            a0.v[j] = v; acc.v[j] = make_float2(0.f, 0.f); cn.v[j] = v;
                            wr_a = true;
                        }
                        continue;
                    }
                    if (stj != SLOT_ACTIVE && stj != SLOT_FINAL) continue;
                    const float2 kk = kq[k].v[j];
                    const float2 aj = a0.v[j];
                    if (s == 0) {
                        if (stj == SLOT_FINAL) {
                            const float pp = aj.x * aj.x + aj.y * aj.y;
                            const size_t oo = (size_t)s_traj[4 * g + j] * a.nmax + S.perm[r];
                            if (a.pop) a.pop[oo] = (double)pp;
                            if (a.amp) { a.amp[2 * oo] = aj.x; a.amp[2 * oo + 1] = aj.y; }
                            continue;
                        }
                        // the accumulator enters the step holding the rounding error of the last update
                        acc.v[j] = make_float2(kk.x + acc.v[j].x, kk.y + acc.v[j].y);
                    } else {
                        acc.v[j].x = fmaf(wgt, kk.x, acc.v[j].x);
                        acc.v[j].y = fmaf(wgt, kk.y, acc.v[j].y);
                        if (s == 3) {
                            // compensated a + (dt/6) acc (two-sum): far from the collision the
                            // interaction-picture amplitudes change by increments a plain FP32 add
                            // would round away; the error is carried to the next accumulator
                            const float h6 = dtj[j] * (1.0f / 6.0f), ih6 = 6.0f / dtj[j];
                            const float ix = h6 * acc.v[j].x, iy = h6 * acc.v[j].y;
                            const float sx = __fadd_rn(aj.x, ix), sy = __fadd_rn(aj.y, iy);
                            const float bx = __fsub_rn(sx, aj.x), by = __fsub_rn(sy, aj.y);
                            const float ex = __fadd_rn(__fsub_rn(aj.x, __fsub_rn(sx, bx)), __fsub_rn(ix, bx));
                            const float ey = __fadd_rn(__fsub_rn(aj.y, __fsub_rn(sy, by)), __fsub_rn(iy, by));
                            a0.v[j] = make_float2(sx, sy);
                            acc.v[j] = make_float2(ex * ih6, ey * ih6);
                            const float2 q = pn.v[j];
                            cn.v[j] = make_float2(q.x * sx - q.y * sy, q.x * sy + q.y * sx);
                            wr_a = true;
                            continue;
                        }
                    }
                    const float bn = s == 2 ? dtj[j] : 0.5f * dtj[j];
                    const float2 yn = make_float2(fmaf(bn, kk.x, aj.x), fmaf(bn, kk.y, aj.y));
                    const float2 q = pn.v[j];
                    cn.v[j] = make_float2(q.x * yn.x - q.y * yn.y, q.x * yn.y + q.y * yn.x);
                }
                if (wr_a) st4(A + o, a0);
                st4(ACC + o, acc);
                st4(C + o, cn);
            }
            // ---- per-column reduction: lanes of one group inside the warp, then warps in FP64
            const int nq = s == 0 ? 6 : 2;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float part[6] = {fp[j], tp[j], vp[j], np_[j], ep[j], jp[j]};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    if (q >= nq) break;
                    float v = part[q];
#pragma unroll
                    for (int off = G4; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    part[q] = v;
                }
                if (lane < G4)
                    for (int q = 0; q < nq; ++q) red[((size_t)warp * B + 4 * lane + j) * 6 + q] = (double)part[q];
            }
            __syncthreads();
            if (tid < B * 6) {
                const int bb = tid / 6, q = tid % 6;
                double sum = 0.0;
                if (q < nq)
                    for (int w2 = 0; w2 < NW; ++w2) sum += red[((size_t)w2 * B + bb) * 6 + q];
                red2[bb][q] = sum;
            }
            __syncthreads();
            // ---- C: one lane per slot, FP64
            if (tid < B) {
                Slot &m = sl[tid];
                const double F = red2[tid][0], Tq = red2[tid][1];
                if (m.state == SLOT_ACTIVE || m.state == SLOT_FINAL) {
                    const double R = m.qs[0], PR = m.qs[1], PP = m.qs[3], imu = m.inv_mu;
                    const double ir = 1.0 / R, ir2 = ir * ir;
                    if (s == 0) {
                        const double V = red2[tid][2], NR = red2[tid][3], ER = red2[tid][4], JY = red2[tid][5];
                        const double et = 0.5 * imu * (PR * PR + PP * PP * ir2) + ER + V;
                        const double jt = PP + 0.5 * JY;
                        if (m.steps == 0) { m.e0 = et; m.j0 = jt; }
                        m.ndev = fmax(m.ndev, fabs(NR - 1.0));
                        m.edev = fmax(m.edev, fabs(et - m.e0));
                        m.jdev = fmax(m.jdev, fabs(jt - m.j0));
                    }
                    if (m.state == SLOT_FINAL) {
                        if (s == 0) {
                            if (a.diag) {
                                mqct_diag d;
                                d.steps = m.steps; d.status = m.status;
                                d.norm_dev = m.ndev; d.energy_dev = m.edev; d.angmom_dev = m.jdev;
                                d.t_final = m.steps * m.dt;
                                a.diag[m.traj] = d;
                            }
                            if (a.t_done) a.t_done[m.traj] = mqct_clock_ns();
                            claim(a, S, m);
                        }
                    } else {
                        const double l4[4] = {PR * imu, F + PP * PP * imu * ir2 * ir, m.phidot, Tq};
                        const double wg = (s == 1 || s == 2) ? 2.0 : 1.0;
                        for (int i = 0; i < 4; ++i) m.lacc[i] = s == 0 ? l4[i] : fma(wg, l4[i], m.lacc[i]);
                        if (s < 3) {
                            const double bnd = s == 2 ? m.dt : 0.5 * m.dt;
                            for (int i = 0; i < 4; ++i) m.qs[i] = fma(bnd, l4[i], m.q[i]);
                        } else {
                            for (int i = 0; i < 4; ++i) { m.q[i] = fma(m.dt / 6.0, m.lacc[i], m.q[i]); m.qs[i] = m.q[i]; }
                            m.steps += 1;
                            const bool fin = isfinite(m.q[0]) && isfinite(m.q[1]) && isfinite(m.q[2]) && isfinite(m.q[3]);
                            if (!fin) m.status |= MQCT_TRAJ_NONFINITE;
                            if (!fin || (m.q[0] >= m.r_end && m.q[1] > 0.0)) m.state = SLOT_FINAL;
                            else if (m.steps >= m.max_steps) { m.status |= MQCT_TRAJ_MAX_STEPS; m.state = SLOT_FINAL; }
                        }
                        if (!(m.status & MQCT_TRAJ_NONFINITE)) locate_slot(S, m);
                    }
                } else if (m.state == SLOT_WAIT && s == 3) {
                    m.state = m.max_steps > 0 ? SLOT_ACTIVE : SLOT_FINAL;
                    if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
                    locate_slot(S, m);
                }
                publish(tid);
            }
            __syncthreads();
            if (s == 3) {
                if (tid == 0) {
                    int live_n = 0;
                    for (int q = 0; q < B; ++q) live_n += sl[q].state != SLOT_IDLE;
                    s_live = live_n;
                }
                // slots that start a trajectory at the next stage: phases of t = 0 (their columns
                // were initialised in P4 of this stage)
                for (int i = tid; i < NL * B; i += T) {
                    const Slot &q = sl[i % B];
                    if ((q.state == SLOT_ACTIVE || q.state == SLOT_FINAL) && q.steps == 0) PHa[i] = make_float2(1.f, 0.f);
                }
            }
            terms();
            __syncthreads();
        }
    }
}

template <int B, int T>
size_t batched_smem(const DevSys &h)
{
    return sizeof(float2) * (3 * (size_t)h.n * B + 2 * (size_t)h.n_levels * B) + sizeof(float) * 2 * (size_t)h.L * B +
           sizeof(double) * (T / 32) * B * 6;
}

template <int B, int T>
bool batched_fits(const DevSys &h, size_t cap)
{
    return (size_t)h.n * (B / 4) <= (size_t)kUpt * T && batched_smem<B, T>(h) <= cap;
}

template <int B, int T>
cudaError_t launch_batched(const BatchArgs &a, const DevSys &h, int sms, cudaStream_t st)
{
    if (a.sm_limit > 0) sms = std::min(sms, a.sm_limit);
    const size_t smem = batched_smem<B, T>(h);
    cudaError_t e = cudaFuncSetAttribute(k_batched_f32<B, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_f32<B, T>, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = std::min(sms * per_sm, (a.n + B - 1) / B);
    grid = std::max(grid, 1);
    k_batched_f32<B, T><<<grid, T, smem, st>>>(a);
    return cudaGetLastError();
}

// Batch shape: 256-thread CTAs, two per SM, when a CTA's block fits in half the shared
// memory; otherwise 512-thread CTAs, one per SM.  Widest batch first.
bool batched_shape_fits(const DevSys &h, int i)
{
    const size_t half = 110 * 1024, full = 220 * 1024;
    switch (i) {
        case 0: return batched_fits<32, 256>(h, half);
        case 1: return batched_fits<16, 256>(h, half);
        case 2: return batched_fits<8, 256>(h, half);
        case 3: return batched_fits<16, 512>(h, full);
        case 4: return batched_fits<8, 512>(h, full);
        case 5: return batched_fits<4, 512>(h, full);
        case 6: return batched_fits<4, 256>(h, half);
        default: return false;
    }
}

int batched_width(const DevSys &h)
{
    for (int i = 0; i < 6; ++i)  // automatic choice: the first six, widest first
        if (batched_shape_fits(h, i)) return kBatchShapes[i][0] * 1000 + kBatchShapes[i][1];
    return 0;
}

// launch with the requested shape (a.shape = index + 1) or the automatic one
cudaError_t run_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st, int *width)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int idx = -1;
    if (a.shape > 0) {
        if (a.shape > 7 || !batched_shape_fits(h, a.shape - 1)) return cudaErrorInvalidConfiguration;
        idx = a.shape - 1;
    } else {
        for (int i = 0; i < 6 && idx < 0; ++i)
            if (batched_shape_fits(h, i)) idx = i;
    }
    if (idx < 0) return cudaErrorInvalidConfiguration;
    if (width) *width = kBatchShapes[idx][0];
    switch (idx) {
        case 0: return launch_batched<32, 256>(a, h, sms, st);
        case 1: return launch_batched<16, 256>(a, h, sms, st);
        case 2: return launch_batched<8, 256>(a, h, sms, st);
        case 3: return launch_batched<16, 512>(a, h, sms, st);
        case 4: return launch_batched<8, 512>(a, h, sms, st);
        case 5: return launch_batched<4, 512>(a, h, sms, st);
        case 6: return launch_batched<4, 256>(a, h, sms, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace mqct
