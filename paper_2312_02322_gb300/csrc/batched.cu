// Batched mixed-precision trajectory kernel (factorised path, FP32 amplitudes).
//
// One CTA integrates B trajectories ("slots") at once; finished slots are refilled from the
// device work queue, so trajectories of uneven length share a CTA.  Their phase-rotated stage
// amplitudes form the N x B block C (one column per trajectory, FP32 complex, shared memory,
// row-major: a row of four columns is 32 contiguous bytes).  The warps have two roles:
//
//   element warps  own units (row r, 4 columns); per RK4 stage
//     P3  contraction (Eq. 12): for every stored term l, Y_l = G^l C over the coalesced
//         32-row sliced-ELL copy of G^l, combined per column with the FP32 spline values:
//         w = M(R_b) c_b and u = M'(R_b) c_b; Coriolis stencil Dc = (J+ - J-) c; the stage
//         derivative da/dt = -i exp(iEt) w + (dPhi/dt / 2) exp(iEt) Dc (Eq. 5) and the partial
//         sums of the force -Re(c^dag u) (Eq. 9), the torque Re(c^dag D w) = -Re((Dc)^dag w)
//         (Eq. 10) and, at stage 0, Re(c^dag w), |a|^2, E|a|^2, <J_y>;
//     P4  RK4 accumulation and the next stage's input c (phase-rotated); the step update
//         a + (dt/6) acc is compensated (two-sum), its rounding error carried into the next
//         step's accumulator;
//   slot warps     hold the FP64 classical state of the slots in registers, one lane per
//     (component, slot): lane 8 c + j carries component c of (R, P_R, Phi, P_Phi) of slot j, so
//     one FP64 instruction advances all four components of eight trajectories.  While the
//     element warps contract stage s they look ahead: R of stage s+1 depends only on P_R of
//     stage s, so its spline interval, 1/R and the spline values v_l, v_l' of stage s+1 are
//     ready before stage s's force is known.  After the force and torque reductions only the
//     RK4 update of (R, P_R, Phi, P_Phi) and dPhi/dt of the next stage remain (a handful of
//     FP64 instructions); the bookkeeping of norm, total energy and P_Phi + <J_y>, the stop
//     rule's outputs and the refill of a finished slot run during the next contraction.
//
// Uneven batches (trajectories of several systems, i.e. basis sizes, in one call) run in this one
// persistent launch: a CTA binds to a system (its share of the grid at the start is proportional
// to the systems' estimated work), takes trajectories from that system's work list (longest
// first) with as many slots as the system's basis allows in the CTA's shared memory, and when the
// list is exhausted and its slots have drained it binds to the system with the most estimated
// work left.
//
// On this GPU an FP64 instruction holds its sub-partition's FP64 pipe for tens of cycles
// whatever the number of active lanes, so the kernel keeps FP64 off the per-element work:
// the phase arguments are 64-bit fixed-point turn counts (traj_common.cuh), the partial sums
// are FP32 within a warp and compensated FP32 (two-sum) across warps, converted to FP64 once per
// trajectory and stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "traj_common.cuh"

namespace mqct {


enum { SLOT_IDLE = 0, SLOT_ACTIVE = 1, SLOT_FINAL = 2, SLOT_WAIT = 3 };

// slot warps for B slots (eight slots per warp, four component lanes per slot)
__host__ __device__ constexpr int batch_slot_warps(int B) { return B > 8 ? B / 8 : 1; }

struct F4x2 {  // four complex FP32 values (one unit row of four columns)
    float2 v[4];
};

// Shared-memory layout of the [rows][B] float2 arrays (C, A, ACC, PHa, PHb): element e = row B + col
// is stored at swz(e), which swaps the two 16-byte halves of a four-column unit when bit 3 of its
// 16-byte chunk index is set.  Warps access units of consecutive rows (their own rows, and the
// gathered neighbours of a banded coupling), whose 16-byte chunks would otherwise fall on only
// half of the eight bank groups of a 128-byte line.
__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 4) & 1) << 1); }

// the four columns e0 .. e0 + 3 (e0 a multiple of 4)
__device__ __forceinline__ F4x2 ld4(const float2 *p, int e0)
{
    const float4 a = *reinterpret_cast<const float4 *>(p + swz(e0));
    const float4 b = *reinterpret_cast<const float4 *>(p + swz(e0 + 2));
    F4x2 r;
    r.v[0] = make_float2(a.x, a.y); r.v[1] = make_float2(a.z, a.w);
    r.v[2] = make_float2(b.x, b.y); r.v[3] = make_float2(b.z, b.w);
    return r;
}

__device__ __forceinline__ void st4(float2 *p, int e0, const F4x2 &r)
{
    *reinterpret_cast<float4 *>(p + swz(e0)) = make_float4(r.v[0].x, r.v[0].y, r.v[1].x, r.v[1].y);
    *reinterpret_cast<float4 *>(p + swz(e0 + 2)) = make_float4(r.v[2].x, r.v[2].y, r.v[3].x, r.v[3].y);
}

// per-slot values the element warps read during one stage, written by the slot warps during the
// stage before (double-buffered by stage parity, so that writer and readers never overlap)
template <int B>
struct SlotView {
    __align__(16) float hp[B];    // dPhi/dt / 2 (FP32 view)
    __align__(16) float dtf[B];   // dt (FP32 view)
    __align__(16) float vid[B];   // sum of the identity terms' v_l (FP32 spline)
    __align__(16) float dvid[B];  // and of their v_l'
    int state[B], traj[B], s0[B], steps[B];
};

// per-slot values of the slot warps that are not needed at every stage (shared memory keeps
// them out of the registers the element warps' stage derivatives need)
struct SlotCold {
    double e0, j0, ndev, edev, jdev;  // initial E_tot and P_Phi + <J_y>, running deviations
    double last_dt, r_end, i2m0;      // dt of the phase increments; stop radius; (1/mu)/R^2 at stage 0
    int status, max_steps, traj, s0;
    float dtf;
};

// shared state of one CTA besides the big per-element arrays
template <int B>
struct BatchShared {
    DevSys S;
    SlotView<B> view[2];
    SlotCold cold[B];
    float2 sum[6][B];  // cross-warp sums (hi, lo) of the six partial sums of the last phase B
    int live;
    int cur;           // system the CTA is bound to (-1: no work left)
};

// dynamic shared memory of a CTA bound to a system with B slots: inc [NL][B] (u64), C, A, ACC [n][B]
// float2, PHa, PHb [NL][B] float2, vv, dvv [2][L][B] float, elev [NL] float, red [NE][B][8] float
template <int BMAX, int T>
size_t batched_smem(const DevSys &h, int B)
{
    constexpr int NE = T / 32 - batch_slot_warps(BMAX);
    const size_t nl = h.n_levels, n = h.n, L = h.L;
    return 8 * nl * B + 8 * (3 * n * B + 2 * nl * B) + 4 * (4 * L * B + nl) + 4 * (size_t)NE * B * 8 + 16;
}

template <int T>
constexpr int batched_min_blocks() { return T >= 512 ? 1 : (T >= 256 ? 2 : 4); }

// the system a CTA binds to next: at the start, the CTA's share of the grid by estimated work;
// afterwards the system with the most estimated work left (-1: none)
__device__ int pick_system(const BatchMultiArgs &a, bool first)
{
    const int ns = a.n_systems;
    auto count_of = [&](int s) { return a.counts ? a.counts[s] : a.n; };
    if (first && ns > 1 && a.work) {
        double tot = 0.0;
        for (int s = 0; s < ns; ++s) tot += a.work[s];
        const double target = (blockIdx.x + 0.5) / gridDim.x * tot;
        double acc = 0.0;
        for (int s = 0; s < ns; ++s) {
            acc += a.work[s];
            if (acc >= target && count_of(s) > 0) return s;
        }
    }
    int best = -1;
    double best_score = -1.0;
    for (int s = 0; s < ns; ++s) {
        const int c = count_of(s);
        const int q = *((volatile const int *)(a.queues + s));
        const int rem = c - (q < c ? q : c);
        if (rem <= 0) continue;
        const double score = rem * (a.work ? a.work[s] / c : 1.0);
        if (score > best_score) {
            best_score = score;
            best = s;
        }
    }
    return best;
}

// everything a CTA does while bound to system `cur`: with BC > 0 its slot count is the compile-time
// constant BC, with BC = 0 the system's entry of a.slots
template <int BC, int BMAX, int T, int kUpt>
__device__ __forceinline__ void batched_system(const BatchMultiArgs &a, BatchShared<BMAX> &sh, int cur,
                                               unsigned char *smraw)
{
    static_assert(BC % 4 == 0 && BC <= BMAX, "slots per CTA");
    constexpr int NS = batch_slot_warps(BMAX);  // slot warps (the last NS warps)
    constexpr int NW = T / 32, NE = NW - NS;    // element warps
    constexpr int TE = NE * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool slot_warp = warp >= NE;
    const int sc = lane >> 3, sj = lane & 7;
    const int sb = slot_warp ? 8 * (warp - NE) + sj : 0;
    const unsigned full = 0xffffffffu;
    const unsigned m4 = 0x01010101u << sj;  // the four component lanes of this slot
    const DevSys &S = sh.S;
    const int B = BC > 0 ? BC : a.slots[cur];    // slots (4, 8, 16 or 32)
    const int G4 = B / 4;                        // four-column groups per row
    const int lg4 = G4 == 1 ? 0 : (G4 == 2 ? 1 : (G4 == 4 ? 2 : 3));
    const int n = S.n, NL = S.n_levels, L = S.L;
    const int *order = a.lists + (size_t)cur * a.n;
    int *queue = a.queues + cur;
    const int count = a.counts ? a.counts[cur] : a.n;
    unsigned long long *inc = reinterpret_cast<unsigned long long *>(smraw);
    float2 *C = reinterpret_cast<float2 *>(inc + (size_t)NL * B);
    float2 *A = C + (size_t)n * B, *ACC = A + (size_t)n * B;
    float2 *PHa = ACC + (size_t)n * B, *PHb = PHa + (size_t)NL * B;
    float *vv = reinterpret_cast<float *>(PHb + (size_t)NL * B), *dvv = vv + 2 * (size_t)L * B;
    float *elev = dvv + 2 * (size_t)L * B;
    float *red = elev + NL;  // [NE][B][8]
    for (int l = tid; l < NL; l += T) elev[l] = (float)S.lev_energy[l];
    // columns of the slots that start at the first stage 0: e_s0, accumulators 0, phases of t = 0
    // and t = dt/2 (after the slot warps' first claims; both roles share the work)
    auto init_columns = [&]() {
        for (int i = tid; i < n * B; i += T) {
            const int r = i / B, bb = i % B;
            const int st = sh.view[0].state[bb];
            if (st != SLOT_ACTIVE && st != SLOT_FINAL) continue;
            const float2 v = make_float2(r == sh.view[0].s0[bb] ? 1.0f : 0.0f, 0.0f);
            A[swz(i)] = v; ACC[swz(i)] = make_float2(0.f, 0.f); C[swz(i)] = v;
        }
        for (int i = tid; i < NL * B; i += T) {
            PHa[swz(i)] = make_float2(1.f, 0.f);
            const int st = sh.view[0].state[i % B];
            if (st == SLOT_ACTIVE || st == SLOT_FINAL) PHb[swz(i)] = phase_factor(inc[i], 1u);
        }
    };
    if (tid == 0) sh.live = 1;

    // The two roles run separate code with the same barriers (two per stage), so that the
    // registers of one role are not kept alive in the other.
    if (slot_warp) {
    // slot-warp registers (lane 8 c + j: component c of (R, P_R, Phi, P_Phi) of slot 8 (warp - NE) + j)
    double q = 0.0, qs = 0.0, lacc = 0.0;
    double imu = 1.0 / S.mu, dtd = 1.0, hdt = 0.5, h6 = 1.0 / 6.0;
    double ir = 0.0, i2m = 0.0, phid = 0.0, t1 = 0.0;  // 1/R, (1/mu)/R^2, dPhi/dt, P_Phi^2/(mu R^3)
    double ir_n = 0.1, i2m_n = 0.0;                   // look-ahead
    int steps = 0, state = SLOT_IDLE;
    bool below_n = false;

    // Every lane of a slot warp runs the same instructions (lanes of slots >= B compute on copies
    // and store nothing), so that the shuffles between the four component lanes of a slot are
    // warp-uniform.
    const bool slot_lane = slot_warp && sb < B;
    const int sbc = sb < B ? sb : B - 1;   // a valid index for reads of the lanes past B
    SlotCold &cs = sh.cold[sbc];
    if (slot_lane && sc == 0) {
        cs.last_dt = -1.0;
        cs.status = 0;
    }
    __syncwarp();

    auto comp = [&](double v, int c2) { return __shfl_sync(full, v, 8 * c2 + sj); };

    // publish this slot's view for stage `stage`
    auto publish = [&](int stage) {
        if (slot_lane && sc == 0) {
            SlotView<BMAX> &vw = sh.view[stage & 1];
            vw.state[sb] = state;
            vw.traj[sb] = cs.traj;
            vw.s0[sb] = cs.s0;
            vw.steps[sb] = steps;
            vw.dtf[sb] = cs.dtf;
            vw.hp[sb] = (float)phid * 0.5f;
        }
    };

    // claim the next valid trajectory for this slot (its four lanes together, shuffles over m4);
    // on return the slot is WAIT (column to be initialised at the next stage 3) or IDLE
    auto claim = [&]() {
        for (;;) {
            int item = 0;
            if (sc == 0) item = atomicAdd(queue, 1);
            item = __shfl_sync(m4, item, sj);
            if (item >= count) {
                state = SLOT_IDLE;
                return;
            }
            const int t = order ? order[item] : item;
            const mqct_traj tr = a.trajs[t];
            if (!traj_valid(tr, S, a.sys_base + cur)) {
                if (a.diag && sc == 0) {
                    mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                    a.diag[t] = d;
                }
                __syncwarp(m4);
                continue;
            }
            if (a.t_start && sc == 0) a.t_start[t] = mqct_clock_ns();
            const int s0 = S.inv[tr.init_state];
            int k0;
            double x0;
            bool bl;
            locate_interval(S, tr.r0, k0, x0, bl);
            // initial mean field M_ss(r0): the four lanes split the terms
            double m = 0.0;
            for (int l = sc; l < L; l += 4) m += spline_fp64(S, l, k0, x0) * S.diag_g[(size_t)l * n + s0];
            m += __shfl_xor_sync(m4, m, 8);
            m += __shfl_xor_sync(m4, m, 16);
            double q4[4];
            initial_state(S, tr, m, q4);
            q = q4[sc];
            qs = q;
            lacc = 0.0;
            dtd = tr.dt;
            hdt = 0.5 * tr.dt;
            h6 = tr.dt / 6.0;
            steps = 0;
            state = SLOT_WAIT;
            const bool new_dt = tr.dt != cs.last_dt;
            __syncwarp(m4);
            if (sc == 0) {
                cs.traj = t;
                cs.s0 = s0;
                cs.dtf = (float)tr.dt;
                cs.r_end = tr.r_end;
                cs.max_steps = tr.max_steps;
                cs.status = 0;
                cs.ndev = cs.edev = cs.jdev = 0.0;
                cs.last_dt = tr.dt;
            }
            // fixed-point phase increments of every level for this dt (kept while dt repeats)
            if (new_dt)
                for (int l = sc; l < NL; l += 4) inc[(size_t)l * B + sb] = phase_increment(S.lev_energy[l], tr.dt);
            __syncwarp(m4);
            return;
        }
    };

    // look-ahead for stage s+1 (s = -1: a slot that starts at the next stage 0): R, its interval,
    // 1/R and the spline values of every term, written to vv / dvv [(s+1) & 1]
    auto look_ahead = [&](int s) {
        const int par = (s + 1) & 1;
        const bool act = slot_lane && state == SLOT_ACTIVE;
        const bool start = slot_lane && state == SLOT_WAIT && (s == 3 || s == -1);
        const double q0 = comp(q, 0), pr = comp(qs, 1), la0 = comp(lacc, 0);
        double qs0 = 0.0, lacc0 = la0;
        stage_component(s < 0 ? 0 : s, imu, pr, 0.0, hdt, dtd, h6, q0, qs0, lacc0);
        double Rn = act ? qs0 : (start ? q0 : 10.0);  // any finite R for slots not running
        int k;
        double x;
        locate_interval(S, Rn, k, x, below_n);
        ir_n = 1.0 / Rn;
        i2m_n = imu * ir_n * ir_n;
        const float xf = (float)x;
        float v0 = 0.f, d0 = 0.f;
        for (int l = sc; l < L; l += 4) {
            float v = 0.f, dv = 0.f;
            if (act || start) {
                const float4 c = S.vcoef_f[(size_t)l * S.n_int + k];
                v = fmaf(xf, fmaf(xf, fmaf(xf, c.w, c.z), c.y), c.x);
                dv = fmaf(xf, fmaf(3.0f * xf, c.w, 2.0f * c.z), c.y);
            }
            if (slot_lane) {
                vv[((size_t)par * L + l) * B + sb] = v;
                dvv[((size_t)par * L + l) * B + sb] = dv;
            }
            if ((S.id_mask >> l) & 1ull) { v0 += v; d0 += dv; }
        }
        v0 += __shfl_xor_sync(full, v0, 8);
        v0 += __shfl_xor_sync(full, v0, 16);
        d0 += __shfl_xor_sync(full, d0, 8);
        d0 += __shfl_xor_sync(full, d0, 16);
        if (slot_lane && sc == 0) {
            sh.view[par].vid[sb] = v0;
            sh.view[par].dvid[sb] = d0;
        }
    };

    // total energy, P_Phi + <J_y> and norm of the state at the start of a step (or of the final
    // state) from its stage-0 sums (sh.sum[2..5]): running maxima of their deviations, for the
    // slots where `apply` holds
    auto bookkeeping = [&](bool apply) {
        const float2 pv = sh.sum[2 + sc][sbc];  // lane c converts V, |a|^2, E|a|^2, <J_y>
        const double val = (double)pv.x + (double)pv.y;
        const double V = comp(val, 0), NR = comp(val, 1), ER = comp(val, 2), JY = comp(val, 3);
        const double PR = comp(q, 1), PP = comp(q, 3);
        const double et = 0.5 * (imu * PR * PR + PP * PP * cs.i2m0) + ER + V;
        const double jt = PP + 0.5 * JY;
        const double e0 = steps == 0 ? et : cs.e0, j0 = steps == 0 ? jt : cs.j0;
        const double nd = fmax(cs.ndev, fabs(NR - 1.0));
        const double ed = fmax(cs.edev, fabs(et - e0));
        const double jd = fmax(cs.jdev, fabs(jt - j0));
        __syncwarp();
        if (apply && sc == 0) {
            cs.e0 = e0; cs.j0 = j0;
            cs.ndev = nd; cs.edev = ed; cs.jdev = jd;
        }
        __syncwarp();
    };

    // ---------------------------------------------------------------- start
    {
        if (slot_lane) claim();
        look_ahead(-1);
        if (slot_lane && state == SLOT_WAIT) {
            const int ms = cs.max_steps;
            state = ms > 0 ? SLOT_ACTIVE : SLOT_FINAL;
            __syncwarp(m4);
            if (sc == 0) cs.status |= (ms <= 0 ? MQCT_TRAJ_MAX_STEPS : 0) | (below_n ? MQCT_TRAJ_TABLE_RANGE : 0);
            ir = ir_n;
            i2m = i2m_n;
        }
        const double pp3 = comp(q, 3);
        if (slot_lane && state != SLOT_IDLE) phid = pp3 * i2m;
        publish(0);
    }
    __syncthreads();
    init_columns();
    __syncthreads();
    {
        while (sh.live) {
            for (int s = 0; s < 4; ++s) {
                // ================================================================ phase A
                {
                // ---- slot warps during the contraction: bookkeeping of stage 0 (a finished slot
                // at stage 1, before its refill; running slots at stage 2), the diagnostics and
                // refill of a finished slot, then the look-ahead for stage s+1
                const bool fin_any = __any_sync(full, slot_lane && state == SLOT_FINAL);
                if (s == 1 && fin_any) {
                    bookkeeping(slot_lane && state == SLOT_FINAL);
                    if (slot_lane && state == SLOT_FINAL) {
                        if (sc == 0) {
                            if (a.diag) {
                                mqct_diag d;
                                d.steps = steps; d.status = cs.status;
                                d.norm_dev = cs.ndev; d.energy_dev = cs.edev; d.angmom_dev = cs.jdev;
                                d.t_final = steps * dtd;
                                a.diag[cs.traj] = d;
                            }
                            if (a.t_done) a.t_done[cs.traj] = mqct_clock_ns();
                        }
                        __syncwarp(m4);
                        claim();  // WAIT or IDLE: phases at stage 2, column at stage 3
                    }
                }
                if (s == 2) bookkeeping(slot_lane && state == SLOT_ACTIVE);
                const double pp3 = comp(qs, 3);
                if (slot_lane && state == SLOT_ACTIVE) t1 = pp3 * phid * ir;  // P_Phi^2 / (mu R^3)
                look_ahead(s);
                }
                __syncthreads();
                // ================================================================ phase B
                {
                // ---- slot warps: cross-warp sums (compensated FP32), then the classical stage
                const int nq = s == 0 ? 6 : 2;
                const int sid = tid - TE;
                for (int pidx = sid; pidx < nq * B; pidx += NS * 32) {
                    const int qq = pidx / B, bb = pidx % B;
                    float hi = 0.f, lo = 0.f;
                    for (int w2 = 0; w2 < NE; ++w2) {
                        float e2;
                        two_sum(hi, red[((size_t)w2 * B + bb) * 8 + qq], hi, e2);
                        lo += e2;
                    }
                    sh.sum[qq][bb] = make_float2(hi, lo);
                }
                if (NS > 1) asm volatile("bar.sync 1, %0;" ::"r"(NS * 32) : "memory");
                else __syncwarp();
                // lane c = 1 converts the force, c = 3 the torque (c = 0, 2: unused copies)
                const float2 pv = sh.sum[sc == 3 ? 1 : 0][sbc];
                const double X2 = (double)pv.x + (double)pv.y;
                const double pr = comp(qs, 1);
                if (s == 0 && slot_lane && sc == 0) cs.i2m0 = i2m;
                const bool act = slot_lane && state == SLOT_ACTIVE;
                const bool start = slot_lane && state == SLOT_WAIT && s == 3;
                {
                    // derivative l_c: (P_R / mu, F + P_Phi^2/(mu R^3), dPhi/dt, torque) (Eqs. 7-10)
                    const double X = sc == 0 ? pr : (sc == 2 ? phid : X2);
                    const double alpha = sc == 0 ? imu : 1.0, beta = sc == 1 ? t1 : 0.0;
                    double qs2 = qs, lacc2 = lacc;
                    stage_component(s, alpha, X, beta, hdt, dtd, h6, q, qs2, lacc2);
                    if (act) { qs = qs2; lacc = lacc2; }
                }
                int add_status = 0;
                if (s == 3) {
                    const unsigned bad = __ballot_sync(full, act && !finite64(qs));
                    const double R = comp(qs, 0), PR = comp(qs, 1);
                    if (act) {
                        q = qs;
                        steps += 1;
                        if ((bad >> sj) & 0x01010101u) {
                            add_status |= MQCT_TRAJ_NONFINITE;
                            state = SLOT_FINAL;
                        } else if (ge_pos(R, cs.r_end) && __double_as_longlong(PR) > 0) {
                            state = SLOT_FINAL;
                        } else if (steps >= cs.max_steps) {
                            add_status |= MQCT_TRAJ_MAX_STEPS;
                            state = SLOT_FINAL;
                        }
                    }
                }
                const double pp3 = comp(qs, 3);
                if ((act && !(add_status & MQCT_TRAJ_NONFINITE)) || start) {
                    if (below_n) add_status |= MQCT_TRAJ_TABLE_RANGE;
                    ir = ir_n;
                    i2m = i2m_n;
                    phid = pp3 * i2m_n;
                }
                if (start) {
                    const int ms = cs.max_steps;
                    state = ms > 0 ? SLOT_ACTIVE : SLOT_FINAL;
                    if (ms <= 0) add_status |= MQCT_TRAJ_MAX_STEPS;
                }
                __syncwarp();
                if (slot_lane && sc == 0 && add_status) cs.status |= add_status;
                publish(s + 1);
                if (s == 3) {
                    const unsigned live = __ballot_sync(full, slot_lane && state != SLOT_IDLE);
                    if (warp == NE && lane == 0) sh.live = 0;
                    if (NS > 1) asm volatile("bar.sync 1, %0;" ::"r"(NS * 32) : "memory");
                    if (lane == 0 && live) atomicOr(&sh.live, 1);
                }
                }
                __syncthreads();
            }
        }
    }
    } else {
    __syncthreads();
    init_columns();
    __syncthreads();
    const int g = tid & (G4 - 1);
    float2 kq[kUpt][4];  // stage derivative da/dt of the unit's four columns (Eq. 5)
    while (sh.live) {
        for (int s = 0; s < 4; ++s) {
            const int par = s & 1;
            const SlotView<BMAX> &vw = sh.view[par];
            // ================================================================ phase A
            {
                // phase factors of the next distinct stage time: t + dt/2 (after stage 0) and
                // t + dt (after stage 2); a slot that starts at the next stage 0 gets t = 0
                if (s == 0 || s == 2) {
                    float2 *dst = s == 0 ? PHb : PHa;
                    for (int i = tid; i < NL * B; i += TE) {
                        const int bb = i % B, st = vw.state[bb];
                        if (st == SLOT_ACTIVE)
                            dst[swz(i)] = phase_factor(inc[i], 2u * (unsigned)vw.steps[bb] + (s == 0 ? 1u : 2u));
                        else if (st == SLOT_WAIT && s == 2)
                            dst[swz(i)] = make_float2(1.f, 0.f);
                    }
                }
                // ---- P3: contraction, derivative, partial sums
                const float2 *PHc = (s == 0 || s == 3) ? PHa : PHb;
                const float *vvs = vv + (size_t)par * L * B, *dvvs = dvv + (size_t)par * L * B;
                int cst[4];
                bool any = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cst[j] = vw.state[4 * g + j];
                    any |= cst[j] == SLOT_ACTIVE || cst[j] == SLOT_FINAL;
                }
                float fp[4] = {0, 0, 0, 0}, tp[4] = {0, 0, 0, 0}, vp[4] = {0, 0, 0, 0};
                float np_[4] = {0, 0, 0, 0}, ep[4] = {0, 0, 0, 0}, jp[4] = {0, 0, 0, 0};
                const float4 hp4 = *reinterpret_cast<const float4 *>(vw.hp + 4 * g);
                const float hp[4] = {hp4.x, hp4.y, hp4.z, hp4.w};
                const float4 vi = *reinterpret_cast<const float4 *>(vw.vid + 4 * g);
                const float4 dvi = *reinterpret_cast<const float4 *>(vw.dvid + 4 * g);
                const float vi_[4] = {vi.x, vi.y, vi.z, vi.w}, dvi_[4] = {dvi.x, dvi.y, dvi.z, dvi.w};
#pragma unroll
                for (int k = 0; k < kUpt; ++k) {
                    const int u = tid + k * TE, r = u >> lg4;
                    if (r >= n || !any) continue;
                    const F4x2 c = ld4(C, r * B + 4 * g);
                    F4x2 w, uu;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        w.v[j] = make_float2(vi_[j] * c.v[j].x, vi_[j] * c.v[j].y);
                        uu.v[j] = make_float2(dvi_[j] * c.v[j].x, dvi_[j] * c.v[j].y);
                    }
                    const int sl = r >> 5, rl = r & 31;
                    for (int f = 0; f < S.n_f; ++f) {
                        const int *so = S.f_sl_off + (size_t)f * (S.n_slices + 1);
                        const int o0 = __ldg(so + sl), o1 = __ldg(so + sl + 1);
                        const int2 *pe = S.f_cvf + o0 + rl;
                        const int width = (o1 - o0) >> 5;
                        float2 y[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll 2
                        for (int e = 0; e < width; ++e, pe += kSlice) {
                            const int2 cv = __ldg(pe);
                            const int col = cv.x;
                            const float gv = __int_as_float(cv.y);
                            const F4x2 z = ld4(C, col * B + 4 * g);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                y[j].x = fmaf(gv, z.v[j].x, y[j].x);
                                y[j].y = fmaf(gv, z.v[j].y, y[j].y);
                            }
                        }
                        const int l = __ldg(S.f_term + f);
                        const float4 v4 = *reinterpret_cast<const float4 *>(vvs + l * B + 4 * g);
                        const float4 d4 = *reinterpret_cast<const float4 *>(dvvs + l * B + 4 * g);
                        const float vl[4] = {v4.x, v4.y, v4.z, v4.w}, dl[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            w.v[j].x = fmaf(vl[j], y[j].x, w.v[j].x); w.v[j].y = fmaf(vl[j], y[j].y, w.v[j].y);
                            uu.v[j].x = fmaf(dl[j], y[j].x, uu.v[j].x); uu.v[j].y = fmaf(dl[j], y[j].y, uu.v[j].y);
                        }
                    }
                    const float au = __ldg(S.aupf + r), ad = __ldg(S.adnf + r);
                    const F4x2 cu = ld4(C, __ldg(S.up + r) * B + 4 * g);
                    const F4x2 cd = ld4(C, __ldg(S.dn + r) * B + 4 * g);
                    const int lev = __ldg(S.lev + r);
                    const F4x2 p = ld4(PHc, lev * B + 4 * g);
                    F4x2 a0;
                    if (s == 0) a0 = ld4(A, r * B + 4 * g);
                    const float el = elev[lev];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float2 dc = make_float2(ad * cd.v[j].x - au * cu.v[j].x, ad * cd.v[j].y - au * cu.v[j].y);
                        const float2 wj = w.v[j], pj = p.v[j];
                        fp[j] -= c.v[j].x * uu.v[j].x + c.v[j].y * uu.v[j].y;
                        tp[j] -= dc.x * wj.x + dc.y * wj.y;
                        // conj(p) Dc = (J+ - J-) a at this stage (partners share the level energy)
                        const float2 da = make_float2(pj.x * dc.x + pj.y * dc.y, pj.x * dc.y - pj.y * dc.x);
                        kq[k][j].x = fmaf(hp[j], da.x, pj.x * wj.y - pj.y * wj.x);
                        kq[k][j].y = fmaf(hp[j], da.y, -(pj.x * wj.x + pj.y * wj.y));
                        if (s == 0) {
                            const float2 aj = a0.v[j];
                            const float pp = aj.x * aj.x + aj.y * aj.y;
                            vp[j] += c.v[j].x * wj.x + c.v[j].y * wj.y;
                            np_[j] += pp;
                            ep[j] += el * pp;
                            jp[j] += aj.x * da.y - aj.y * da.x;
                        }
                    }
                }
                // per-column sums over the warp (lanes of one column group), FP32; six quantities
                // at stage 0, two (force, torque) at the others
                auto warp_sums = [&](auto nqc) {
                    constexpr int NQ = decltype(nqc)::value;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float part[NQ];
                        part[0] = fp[j];
                        part[1] = tp[j];
                        if constexpr (NQ == 6) {
                            part[2] = vp[j]; part[3] = np_[j]; part[4] = ep[j]; part[5] = jp[j];
                        }
#pragma unroll
                        for (int qq = 0; qq < NQ; ++qq) {
                            float v = part[qq];
#pragma unroll
                            for (int off = G4; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                            part[qq] = v;
                        }
                        if (lane < G4)
#pragma unroll
                            for (int qq = 0; qq < NQ; ++qq) red[((size_t)warp * B + 4 * lane + j) * 8 + qq] = part[qq];
                    }
                };
                if (s == 0) warp_sums(std::integral_constant<int, 6>{});
                else warp_sums(std::integral_constant<int, 2>{});
            }
            __syncthreads();
            // ================================================================ phase B
            {
                // ---- P4: RK4 accumulation and the next stage's input (own units only)
                const float2 *PHn = (s == 0 || s == 1) ? PHb : PHa;
                const float4 dt4 = *reinterpret_cast<const float4 *>(vw.dtf + 4 * g);
                const float dtj[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
                int cst[4];
                bool all_act = true;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cst[j] = vw.state[4 * g + j];
                    all_act &= cst[j] == SLOT_ACTIVE;
                }
                const float wgt = (s == 1 || s == 2) ? 2.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < kUpt; ++k) {
                    const int u = tid + k * TE, r = u >> lg4;
                    if (r >= n) continue;
                    const int o = r * B + 4 * g;
                    const int lev = __ldg(S.lev + r);
                    F4x2 a0 = ld4(A, o), acc = ld4(ACC, o), cn;
                    // the columns not updated below keep their input; when all four are running,
                    // every column is written and the old row is not needed
                    if (!all_act) cn = ld4(C, o);
                    const F4x2 pn = ld4(PHn, lev * B + 4 * g);
                    bool wr_a = false;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int stj = cst[j];
                        if (stj == SLOT_WAIT) {
                            if (s == 3) {
                                const float2 v = make_float2(r == vw.s0[4 * g + j] ? 1.0f : 0.0f, 0.0f);
                                a0.v[j] = v; acc.v[j] = make_float2(0.f, 0.f); cn.v[j] = v;
                                wr_a = true;
                            }
                            continue;
                        }
                        if (stj != SLOT_ACTIVE && stj != SLOT_FINAL) continue;
                        if (stj == SLOT_FINAL && s != 0) continue;
                        const float2 kk = kq[k][j];
                        const float2 aj = a0.v[j];
                        if (s == 0) {
                            if (stj == SLOT_FINAL) {
                                const float pp = aj.x * aj.x + aj.y * aj.y;
                                const size_t oo = (size_t)vw.traj[4 * g + j] * a.nmax + __ldg(S.perm + r);
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
                                const float h6f = dtj[j] * (1.0f / 6.0f), ih6 = 6.0f / dtj[j];
                                const float ix = h6f * acc.v[j].x, iy = h6f * acc.v[j].y;
                                float sx, sy, ex, ey;
                                two_sum(aj.x, ix, sx, ex);
                                two_sum(aj.y, iy, sy, ey);
                                a0.v[j] = make_float2(sx, sy);
                                acc.v[j] = make_float2(ex * ih6, ey * ih6);
                                const float2 qn = pn.v[j];
                                cn.v[j] = make_float2(qn.x * sx - qn.y * sy, qn.x * sy + qn.y * sx);
                                wr_a = true;
                                continue;
                            }
                        }
                        const float bn = s == 2 ? dtj[j] : 0.5f * dtj[j];
                        const float2 yn = make_float2(fmaf(bn, kk.x, aj.x), fmaf(bn, kk.y, aj.y));
                        const float2 qn = pn.v[j];
                        cn.v[j] = make_float2(qn.x * yn.x - qn.y * yn.y, qn.x * yn.y + qn.y * yn.x);
                    }
                    if (wr_a) st4(A, o, a0);
                    st4(ACC, o, acc);
                    st4(C, o, cn);
                }
            }
            __syncthreads();
        }
    }
    }
}

// EXACT: every system of the launch runs BMAX slots per CTA (compile-time slot count); otherwise
// each system runs the slot count of a.slots
template <int BMAX, int T, int kUpt, bool EXACT>  // kUpt: (row, 4-column) units per element thread at most
__global__ void __launch_bounds__(T, batched_min_blocks<T>()) k_batched_f32(BatchMultiArgs a)
{
    static_assert(BMAX % 4 == 0 && BMAX <= 32, "batch width");
    static_assert(T / 32 - batch_slot_warps(BMAX) >= 1, "no element warps");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ BatchShared<BMAX> sh;
    bool first = true;
    for (;;) {
        // bind to a system
        if (threadIdx.x == 0) {
            const int s = pick_system(a, first);
            sh.cur = s;
            if (s >= 0) sh.S = a.sys[s];
        }
        __syncthreads();
        first = false;
        const int cur = sh.cur;
        if (cur < 0) break;
        batched_system<EXACT ? BMAX : 0, BMAX, T, kUpt>(a, sh, cur, smraw);
        __syncthreads();  // both roles are done with this system before the CTA binds to the next
    }
}

// the largest slot count (4, 8, 16 or 32, at most BMAX) with which a system fits a CTA of the shape
// in `cap` bytes of shared memory; 0 if none
template <int BMAX, int T, int kUpt>
int batched_slots(const DevSys &h, size_t cap)
{
    constexpr int TE = (T / 32 - batch_slot_warps(BMAX)) * 32;
    for (int b = BMAX; b >= 4; b >>= 1)
        if ((size_t)h.n * (b / 4) <= (size_t)kUpt * TE && batched_smem<BMAX, T>(h, b) + sizeof(BatchShared<BMAX>) <= cap)
            return b;
    return 0;
}

template <int BMAX, int T, int kUpt>
cudaError_t launch_batched(BatchMultiArgs a, const std::vector<const DevSys *> &hs, size_t cap, int sms,
                           cudaStream_t st)
{
    size_t smem = 0;
    int minb = BMAX;
    for (size_t i = 0; i < hs.size(); ++i) {
        const int b = batched_slots<BMAX, T, kUpt>(*hs[i], cap);
        if (b == 0) return cudaErrorInvalidConfiguration;
        a.slots[i] = b;
        minb = std::min(minb, b);
        smem = std::max(smem, batched_smem<BMAX, T>(*hs[i], b));
    }
    const bool exact = minb == BMAX;
    const void *kern = exact ? (const void *)k_batched_f32<BMAX, T, kUpt, true>
                             : (const void *)k_batched_f32<BMAX, T, kUpt, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(sms * per_sm, (a.n + minb - 1) / minb));
    if (exact) k_batched_f32<BMAX, T, kUpt, true><<<grid, T, smem, st>>>(a);
    else k_batched_f32<BMAX, T, kUpt, false><<<grid, T, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// Shapes (slots per CTA at most, threads), kBatchShapes; a CTA of 256 threads leaves room for two
// per SM (half the shared memory each).
static size_t shape_cap(int i) { return (i == 2 || i == 6) ? 110 * 1024 : 220 * 1024; }

// slot count of shape index i for the system (0: does not fit) and the shared memory it takes
template <int BMAX, int T, int kUpt>
static int shape_slots_of(const DevSys &h, size_t cap, size_t *smem)
{
    const int b = batched_slots<BMAX, T, kUpt>(h, cap);
    if (smem) *smem = b ? batched_smem<BMAX, T>(h, b) + sizeof(BatchShared<BMAX>) : 0;
    return b;
}

static int shape_slots(const DevSys &h, int i, size_t *smem = nullptr)
{
    const size_t cap = shape_cap(i);
    switch (i) {
        case 0: return shape_slots_of<32, 512, 4>(h, cap, smem);
        case 1: return shape_slots_of<16, 512, 4>(h, cap, smem);
        case 2: return shape_slots_of<8, 256, 4>(h, cap, smem);
        case 3: return shape_slots_of<8, 512, 2>(h, cap, smem);
        case 4: return shape_slots_of<4, 512, 4>(h, cap, smem);
        case 5: return shape_slots_of<16, 256, 4>(h, cap, smem);
        case 6: return shape_slots_of<4, 256, 2>(h, cap, smem);
        default: return 0;
    }
}

bool batched_shape_fits(const DevSys &h, int i) { return shape_slots(h, i) > 0; }

int batched_width(const DevSys &h)
{
    for (int i = 0; i < 6; ++i)
        if (batched_shape_fits(h, i)) return kBatchShapes[i][0] * 1000 + kBatchShapes[i][1];
    return 0;
}

// The automatic shape for n trajectories over the systems hs.  A CTA steps its slots in lockstep,
// so its step time grows with its slot count while the throughput of an SM levels off from about
// eight slots on: the longest trajectories, which start first from the longest-first work list,
// then set the end of the launch when there are too many slots, and the refill order of the list
// cannot balance the slots when there are too few.  The rule: the shape with the most slots on
// the GPU (slots per CTA x CTAs per SM x SMs, the slot count of the narrowest system) that still
// leaves two trajectories per slot, else the one with the fewest slots; ties go to the earlier
// entry of kAutoOrder, which puts the eight-slots-per-SM shapes first.  -1: no shape fits.
int batched_auto_shape(const std::vector<const DevSys *> &hs, int n, int sms)
{
    static const int kAutoOrder[7] = {3, 6, 4, 0, 1, 5, 2};
    int best = -1, fewest = -1;
    long long best_slots = -1, fewest_slots = 0;
    for (int k = 0; k < 7; ++k) {
        const int i = kAutoOrder[k];
        int b = 1 << 30;
        size_t smem = 0;
        for (const DevSys *h : hs) {
            size_t sm = 0;
            b = std::min(b, shape_slots(*h, i, &sm));
            smem = std::max(smem, sm);
        }
        if (hs.empty() || b <= 0) continue;
        // two CTAs of 256 threads share an SM's registers when their shared memory allows
        const int per_sm = (kBatchShapes[i][1] == 256 && smem <= 113 * 1024) ? 2 : 1;
        const long long slots = (long long)b * per_sm * sms;
        if (2 * slots <= n && slots > best_slots) {
            best_slots = slots;
            best = i;
        }
        if (fewest < 0 || slots < fewest_slots) {
            fewest_slots = slots;
            fewest = i;
        }
    }
    return best >= 0 ? best : fewest;
}

// one persistent launch over every system of the call, with the requested shape (index + 1) or
// the automatic one (batched_auto_shape)
cudaError_t run_batched(BatchMultiArgs a, const std::vector<const DevSys *> &hs, int shape, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (hs.empty() || (int)hs.size() > kBatchMaxSystems) return cudaErrorInvalidValue;
    auto all_fit = [&](int i) {
        for (const DevSys *h : hs)
            if (!batched_shape_fits(*h, i)) return false;
        return true;
    };
    int idx = -1;
    if (shape > 0) {
        if (shape > 7 || !all_fit(shape - 1)) return cudaErrorInvalidConfiguration;
        idx = shape - 1;
    } else {
        idx = batched_auto_shape(hs, a.n, sms);
    }
    if (idx < 0) return cudaErrorInvalidConfiguration;
    const size_t cap = shape_cap(idx);
    switch (idx) {
        case 0: return launch_batched<32, 512, 4>(a, hs, cap, sms, st);
        case 1: return launch_batched<16, 512, 4>(a, hs, cap, sms, st);
        case 2: return launch_batched<8, 256, 4>(a, hs, cap, sms, st);
        case 3: return launch_batched<8, 512, 2>(a, hs, cap, sms, st);
        case 4: return launch_batched<4, 512, 4>(a, hs, cap, sms, st);
        case 5: return launch_batched<16, 256, 4>(a, hs, cap, sms, st);
        case 6: return launch_batched<4, 256, 2>(a, hs, cap, sms, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace mqct
