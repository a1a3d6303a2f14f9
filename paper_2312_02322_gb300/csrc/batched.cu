// Batched mixed-precision trajectory kernel (factorised path, FP32 amplitudes).
//
// One CTA integrates B trajectories at once: their phase-rotated stage amplitudes form the
// N x B block C (one column per trajectory, FP32 complex, shared memory).  Per RK4 stage:
//   P3  contraction: for every stored term lambda, Y_lambda = G^lambda C (sparse G, the same
//       row entries applied to all B columns), combined per column with the FP32 spline
//       values v_lambda(R_b), v_lambda'(R_b):  w = M(R_b) c_b, u = M'(R_b) c_b   (Eq. 12);
//       Coriolis stencil Dc_b = (J+ - J-) c_b; partial sums of the force -Re(c^dag u), the
//       torque Re(c^dag D w) = -Re((Dc)^dag w) and (stage 0) Re(c^dag w);
//   P4  derivative assembly da/dt = -i exp(iEt) w + (dPhi/dt/2) exp(iEt) Dc   (Eq. 5, using
//       that Coriolis partners share the level energy), RK4 accumulation and next stage input;
//   C   one lane per trajectory: FP64 classical stage update (Eqs. 7-10), FP64 bookkeeping of
//       norm, total energy and P_Phi + <J_y>, termination, and refill of the slot from the
//       device work queue (trajectories of uneven length share a CTA).
// Phase factors exp(-i E_l t) per level and slot: argument E_l t and its reduction modulo
// 2 pi in FP64, sine and cosine of the reduced angle in FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace mqct {

constexpr int kBThreads = 512;
constexpr int kEptMax = 16;  // elements (row, column) owned by one thread

enum { SLOT_IDLE = 0, SLOT_ACTIVE = 1, SLOT_FINAL = 2, SLOT_WAIT = 3 };

struct Slot {
    double q[4], qs[4], lacc[4];
    double dt, r_end, e0, j0, ndev, edev, jdev, x, phidot;
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

// slot thread: claim the next valid trajectory for slot b (FP64 initial conditions)
__device__ void claim(const BatchArgs &a, const DevSys &S, Slot &sl)
{
    for (;;) {
        int item = atomicAdd(a.queue, 1);
        if (item >= a.n) {
            sl.state = SLOT_IDLE;
            return;
        }
        const int t = a.order ? a.order[item] : item;
        const mqct_traj tr = a.trajs[t];
        bool ok = tr.system_idx == a.sys_idx && tr.dt > 0.0 && tr.e_coll > 0.0 && tr.b >= 0.0 && tr.r0 > 0.0 &&
                  tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0 && tr.init_state >= 0 &&
                  tr.init_state < S.n;
        if (!ok) {
            if (a.diag) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                a.diag[t] = d;
            }
            continue;
        }
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
        sl.status = 0; sl.steps = 0; sl.traj = t; sl.s0 = s0;
        sl.state = SLOT_WAIT;
        sl.kint = k; sl.x = x; sl.phidot = 0.0;
        return;
    }
}

__device__ __forceinline__ void locate_slot(const DevSys &S, Slot &sl)
{
    const double R = sl.qs[0];
    int k = (int)floor((R - S.r_min) * S.inv_h);
    k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
    sl.kint = k;
    sl.x = R - (S.r_min + k * S.h);
    sl.phidot = sl.qs[3] / (S.mu * R * R);
    if (R < S.r_min) sl.status |= MQCT_TRAJ_TABLE_RANGE;
}

template <int B>
__global__ void __launch_bounds__(kBThreads, 1) k_batched_f32(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ DevSys S;
    __shared__ Slot sl[B];
    __shared__ float vid[B], dvid[B];
    __shared__ int s_live;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBThreads / 32;
    const int b = tid & (B - 1);
    if (tid == 0) S = *a.sys;
    __syncthreads();
    const int n = S.n, NL = S.n_levels, L = S.L;
    float2 *C = reinterpret_cast<float2 *>(smraw);
    float2 *A = C + (size_t)n * B, *ACC = A + (size_t)n * B;
    float2 *PHa = ACC + (size_t)n * B, *PHb = PHa + (size_t)NL * B;
    float *vv = reinterpret_cast<float *>(PHb + (size_t)NL * B), *dvv = vv + (size_t)L * B;
    double *red = reinterpret_cast<double *>(dvv + (size_t)L * B);  // [NW][B][6], 8-byte aligned (B >= 4)
    const int ept = (n * B + kBThreads - 1) / kBThreads;

    // v_lambda, v_lambda' at every slot's stage R (FP32 spline of the FP64-located interval)
    auto terms = [&]() {
        for (int i = tid; i < L * B; i += kBThreads) {
            const int l = i / B, bb = i % B;
            const Slot &s = sl[bb];
            if (s.state == SLOT_IDLE || s.state == SLOT_WAIT) continue;
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
    // column initialisation of slots waiting to start (A = e_s0, ACC = 0, C = A, phases 1)
    auto init_columns = [&]() {
        for (int k = 0; k < ept; ++k) {
            const int e = tid + k * kBThreads, r = e / B;
            if (r >= n || sl[b].state != SLOT_WAIT) continue;
            const float2 v = make_float2(r == sl[b].s0 ? 1.0f : 0.0f, 0.0f);
            A[e] = v; ACC[e] = make_float2(0.f, 0.f); C[e] = v;
        }
        for (int i = tid; i < NL * B; i += kBThreads)
            if (sl[i % B].state == SLOT_WAIT) PHa[i] = make_float2(1.f, 0.f);
    };

    if (tid < B) claim(a, S, sl[tid]);
    __syncthreads();
    init_columns();
    __syncthreads();
    if (tid < B && sl[tid].state == SLOT_WAIT) {
        sl[tid].state = sl[tid].max_steps > 0 ? SLOT_ACTIVE : SLOT_FINAL;
        if (sl[tid].max_steps <= 0) sl[tid].status |= MQCT_TRAJ_MAX_STEPS;
        locate_slot(S, sl[tid]);
    }
    if (tid == 0) s_live = 1;
    __syncthreads();
    terms();
    __syncthreads();

    while (s_live) {
        for (int s = 0; s < 4; ++s) {
            const float2 *PHc = (s == 0 || s == 3) ? PHa : PHb;
            const float2 *PHn = (s == 0 || s == 1) ? PHb : PHa;
            // phases of the next distinct stage time for the running slots
            if (s == 0 || s == 2) {
                float2 *dst = s == 0 ? PHb : PHa;
                for (int i = tid; i < NL * B; i += kBThreads) {
                    const Slot &q = sl[i % B];
                    if (q.state != SLOT_ACTIVE) continue;
                    const double t = q.steps * q.dt + (s == 0 ? 0.5 * q.dt : q.dt);
                    dst[i] = phase_of(S.lev_energy[i / B], t);
                }
            }
            // ---- P3: contraction, Coriolis stencil, partial sums
            const int st_b = sl[b].state;
            const bool live = st_b == SLOT_ACTIVE || st_b == SLOT_FINAL;
            float2 wk[kEptMax], dck[kEptMax];
            float fpart = 0.f, tpart = 0.f, vpart = 0.f;
#pragma unroll
            for (int k = 0; k < kEptMax; ++k) {
                wk[k] = make_float2(0.f, 0.f);
                dck[k] = make_float2(0.f, 0.f);
                const int e = tid + k * kBThreads, r = e / B;
                if (k >= ept || r >= n || !live) continue;
                const float2 c = C[e];
                float2 w = make_float2(vid[b] * c.x, vid[b] * c.y);
                float2 u = make_float2(dvid[b] * c.x, dvid[b] * c.y);
                for (int f = 0; f < S.n_f; ++f) {
                    const int *ptr = S.csr_ptr + (size_t)f * (n + 1);
                    const int e0 = __ldg(ptr + r), e1 = __ldg(ptr + r + 1);
                    float2 y = make_float2(0.f, 0.f);
                    for (int q = e0; q < e1; ++q) {
                        const float g = __ldg(S.csr_val + q);
                        const float2 z = C[__ldg(S.csr_col + q) * B + b];
                        y.x = fmaf(g, z.x, y.x);
                        y.y = fmaf(g, z.y, y.y);
                    }
                    const int l = S.f_term[f];
                    const float v = vv[l * B + b], dv = dvv[l * B + b];
                    w.x = fmaf(v, y.x, w.x); w.y = fmaf(v, y.y, w.y);
                    u.x = fmaf(dv, y.x, u.x); u.y = fmaf(dv, y.y, u.y);
                }
                const float au = (float)S.aup[r], ad = (float)S.adn[r];
                const float2 cu = C[S.up[r] * B + b], cd = C[S.dn[r] * B + b];
                const float2 dc = make_float2(ad * cd.x - au * cu.x, ad * cd.y - au * cu.y);
                fpart -= c.x * u.x + c.y * u.y;
                tpart -= dc.x * w.x + dc.y * w.y;
                vpart += c.x * w.x + c.y * w.y;
                wk[k] = w;
                dck[k] = dc;
            }
            __syncthreads();
            // ---- P4: derivatives, RK4 accumulation, next stage input (own elements only)
            const Slot &me = sl[b];
            const float hp = 0.5f * (float)me.phidot;
            const float dtf = (float)me.dt;
            const float wgt = (s == 1 || s == 2) ? 2.0f : 1.0f;
            const float bn = s == 2 ? dtf : 0.5f * dtf;
            float npart = 0.f, epart = 0.f, jpart = 0.f;
#pragma unroll
            for (int k = 0; k < kEptMax; ++k) {
                const int e = tid + k * kBThreads, r = e / B;
                if (k >= ept || r >= n) continue;
                if (st_b == SLOT_WAIT && s == 3) {
                    const float2 v = make_float2(r == me.s0 ? 1.0f : 0.0f, 0.0f);
                    A[e] = v; ACC[e] = make_float2(0.f, 0.f); C[e] = v;
                    continue;
                }
                if (!live) continue;
                const int lev = S.lev[r];
                const float2 p = PHc[lev * B + b], w = wk[k], dc = dck[k];
                // conj(p) Dc = (J+ - J-) a at this stage (partners share the level energy)
                const float2 da = make_float2(p.x * dc.x + p.y * dc.y, p.x * dc.y - p.y * dc.x);
                float2 kk;
                kk.x = fmaf(hp, da.x, p.x * w.y - p.y * w.x);
                kk.y = fmaf(hp, da.y, -(p.x * w.x + p.y * w.y));
                const float2 a0 = A[e];
                if (s == 0) {
                    const float pp = a0.x * a0.x + a0.y * a0.y;
                    npart += pp;
                    epart += (float)S.lev_energy[lev] * pp;
                    jpart += a0.x * da.y - a0.y * da.x;
                    if (st_b == SLOT_FINAL) {
                        const size_t o = (size_t)me.traj * a.nmax + S.perm[r];
                        if (a.pop) a.pop[o] = (double)pp;
                        if (a.amp) { a.amp[2 * o] = a0.x; a.amp[2 * o + 1] = a0.y; }
                        continue;
                    }
                    // the accumulator enters the step holding the rounding error of the last update
                    const float2 cmp = ACC[e];
                    ACC[e] = make_float2(kk.x + cmp.x, kk.y + cmp.y);
                } else {
                    float2 acc = ACC[e];
                    acc.x = fmaf(wgt, kk.x, acc.x);
                    acc.y = fmaf(wgt, kk.y, acc.y);
                    if (s == 3) {
                        // compensated update a + (dt/6) acc (two-sum): in the interaction picture a
                        // changes by tiny increments far from the collision, which a plain FP32 add
                        // would round away; the error is carried to the next step's accumulator
                        const float h6 = dtf / 6.0f, ih6 = 6.0f / dtf;
                        const float ix = h6 * acc.x, iy = h6 * acc.y;
                        const float sx = __fadd_rn(a0.x, ix), sy = __fadd_rn(a0.y, iy);
                        const float bx = __fsub_rn(sx, a0.x), by = __fsub_rn(sy, a0.y);
                        const float ex = __fadd_rn(__fsub_rn(a0.x, __fsub_rn(sx, bx)), __fsub_rn(ix, bx));
                        const float ey = __fadd_rn(__fsub_rn(a0.y, __fsub_rn(sy, by)), __fsub_rn(iy, by));
                        const float2 an = make_float2(sx, sy);
                        A[e] = an;
                        ACC[e] = make_float2(ex * ih6, ey * ih6);
                        const float2 pn = PHn[lev * B + b];
                        C[e] = make_float2(pn.x * an.x - pn.y * an.y, pn.x * an.y + pn.y * an.x);
                        continue;
                    }
                    ACC[e] = acc;
                }
                const float2 yn = make_float2(fmaf(bn, kk.x, a0.x), fmaf(bn, kk.y, a0.y));
                const float2 pn = PHn[lev * B + b];
                C[e] = make_float2(pn.x * yn.x - pn.y * yn.y, pn.x * yn.y + pn.y * yn.x);
            }
            // per-column reduction: lanes of one column inside the warp, then warps in FP64
            float part[6] = {fpart, tpart, vpart, npart, epart, jpart};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float v = part[q];
                for (int o = B; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                part[q] = v;
            }
            if (lane < B) {
#pragma unroll
                for (int q = 0; q < 6; ++q) red[((size_t)warp * B + lane) * 6 + q] = (double)part[q];
            }
            __syncthreads();
            // ---- C: one lane per slot, FP64
            if (tid < B) {
                Slot &m = sl[tid];
                double F = 0, T = 0, V = 0, NR = 0, ER = 0, JY = 0;
                for (int w2 = 0; w2 < NW; ++w2) {
                    const double *r6 = red + ((size_t)w2 * B + tid) * 6;
                    F += r6[0]; T += r6[1]; V += r6[2]; NR += r6[3]; ER += r6[4]; JY += r6[5];
                }
                const double mu = S.mu;
                if (m.state == SLOT_ACTIVE || m.state == SLOT_FINAL) {
                    const double R = m.qs[0], PR = m.qs[1], PP = m.qs[3];
                    if (s == 0) {
                        const double et = PR * PR / (2.0 * mu) + PP * PP / (2.0 * mu * R * R) + ER + V;
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
                            claim(a, S, m);
                        }
                    } else {
                        const double l4[4] = {PR / mu, F + PP * PP / (mu * R * R * R), m.phidot, T};
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
            }
            __syncthreads();
            if (tid == 0 && s == 3) {
                int live_n = 0;
                for (int q = 0; q < B; ++q) live_n += sl[q].state != SLOT_IDLE;
                s_live = live_n;
            }
            // phases of slots that start a trajectory at the next stage (t = 0); their columns were
            // initialised in P4 of this stage
            if (s == 3)
                for (int i = tid; i < NL * B; i += kBThreads) {
                    const Slot &q = sl[i % B];
                    if ((q.state == SLOT_ACTIVE || q.state == SLOT_FINAL) && q.steps == 0) PHa[i] = make_float2(1.f, 0.f);
                }
            terms();
            __syncthreads();
        }
    }
}

template <int B>
size_t batched_smem(const DevSys &h)
{
    return sizeof(float2) * (3 * (size_t)h.n * B + 2 * (size_t)h.n_levels * B) + sizeof(float) * 2 * (size_t)h.L * B +
           sizeof(double) * (kBThreads / 32) * B * 6;
}

template <int B>
cudaError_t launch_batched(const BatchArgs &a, const DevSys &h, int sms, cudaStream_t st)
{
    const size_t smem = batched_smem<B>(h);
    cudaError_t e = cudaFuncSetAttribute(k_batched_f32<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_f32<B>, kBThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = std::min(sms * per_sm, (a.n + B - 1) / B);
    grid = std::max(grid, 1);
    k_batched_f32<B><<<grid, kBThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// pick the widest batch whose shared-memory block and per-thread element count fit
int batched_width(const DevSys &h)
{
    const size_t cap = 220 * 1024;
    if ((size_t)h.n * 32 <= (size_t)kEptMax * kBThreads && batched_smem<32>(h) <= cap) return 32;
    if ((size_t)h.n * 16 <= (size_t)kEptMax * kBThreads && batched_smem<16>(h) <= cap) return 16;
    if ((size_t)h.n * 8 <= (size_t)kEptMax * kBThreads && batched_smem<8>(h) <= cap) return 8;
    if ((size_t)h.n * 4 <= (size_t)kEptMax * kBThreads && batched_smem<4>(h) <= cap) return 4;
    return 0;
}

cudaError_t run_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st, int *width)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int B = batched_width(h);
    if (width) *width = B;
    switch (B) {
        case 32: return launch_batched<32>(a, h, sms, st);
        case 16: return launch_batched<16>(a, h, sms, st);
        case 8: return launch_batched<8>(a, h, sms, st);
        case 4: return launch_batched<4>(a, h, sms, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace mqct
