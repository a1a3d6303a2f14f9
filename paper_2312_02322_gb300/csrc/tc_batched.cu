// Stage-synchronous tensor-core trajectory path (factorised coupling, BF16x3 contraction).
//
// All trajectories in flight form one N x S block of amplitudes in global memory (S slots,
// one column per trajectory; finished slots are refilled from the device work queue).  Every
// RK4 stage runs three kernels:
//   k_tc_contract  tcgen05 GEMMs: for every row tile (packed m-blocks, <= 128 rows) and tile of
//                  64 slots (128 real columns = Re, Im), the two accumulators
//                      w = sum_l G^l (v_l(R_b) c_b)    u = sum_l G^l (v_l'(R_b) c_b)
//                  (Eq. 12 with the spline values folded into the B operand) are built in tensor
//                  memory from BF16 hi/lo splits, three MMAs per K step (hi.hi + hi.lo + lo.hi),
//                  FP32 accumulation; identity terms are added in the epilogue;
//   k_tc_update    per element: Coriolis stencil, derivative da/dt = -i exp(iEt) w +
//                  (dPhi/dt/2) exp(iEt) D c (Eq. 5), compensated RK4 accumulation, next stage
//                  input; per-slot partial sums of force, torque and (stage 0) diagnostics;
//   k_tc_slots     one thread per slot, FP64: classical stage update (Eqs. 7-10), bookkeeping,
//                  stop rule, refill, the spline values and phase factors of the next stage.
// The host runs chunks of steps as one CUDA graph and checks the number of live slots between
// chunks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mqct {

namespace {

constexpr int kTcSlotsPerTile = 64;  // 128 real columns
constexpr int kTcRows = 8;           // rows per k_tc_update block (x 32 slots)
constexpr long long kTcWait = 1ll << 24;

enum { TS_IDLE = 0, TS_ACTIVE = 1, TS_FINAL = 2, TS_WAIT = 3 };

struct TSlot {
    double q[4], qs[4], lacc[4];
    double dt, r_end, e0, j0, ndev, edev, jdev, x, phidot, inv_mu;
    int kint, status, steps, max_steps, traj, state, s0;
};

struct TcState {
    const DevSys *sys;
    const mqct_traj *trajs;
    const int *order;
    int n, S;                 // trajectories, slots
    int *queue;
    int *live;                // live slots after the last step
    double *pop, *amp;
    mqct_diag *diag;
    int nmax;
    float2 *C[2];             // [n][S] stage amplitudes (phase rotated), double buffered
    float2 *A, *ACC;          // [n][S]
    float2 *W, *U;            // [n][S] contraction results
    float *coef;              // [2][L][S] v_l and v_l' at each slot's stage R
    float *vid;               // [2][S] identity-term sums of v and v'
    float *hp, *dtf;          // [S] dPhi/dt / 2 and dt (FP32 views)
    int *state;               // [S]
    float2 *PHa, *PHb;        // [n_levels][S]
    double *part;             // [n_rowblocks][S][6]
    TSlot *slot;              // [S]
};

__device__ __forceinline__ float2 tc_phase(double e, double t)
{
    const double two_pi_hi = 6.283185307179586232, two_pi_lo = 2.4492935982947064e-16;
    const double th = e * t;
    const double k = rint(th * 0.15915494309189535);
    double r = fma(-k, two_pi_hi, th);
    r = fma(-k, two_pi_lo, r);
    float s, c;
    sincosf((float)r, &s, &c);
    return make_float2(c, -s);
}

__device__ __forceinline__ uint16_t bf16_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// ---------------------------------------------------------------------------------------------
// contraction: one CTA per (row tile, slot tile), 4 warps; one thread issues the MMAs
__global__ void __launch_bounds__(128) k_tc_contract(TcState T, int cur)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int any_live;
    const DevSys &S = *T.sys;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = S.n_tiles;
    const int rt = blockIdx.x % nt, ct = blockIdx.x / nt;
    const int r0 = S.tile_r0[rt], R = S.tile_r0[rt + 1] - r0;
    const int s0 = ct * kTcSlotsPerTile;
    if (tid == 0) any_live = 0;
    __syncthreads();
    if (tid < kTcSlotsPerTile && s0 + tid < T.S) {
        const int st = T.state[s0 + tid];
        if (st == TS_ACTIVE || st == TS_FINAL) any_live = 1;
    }
    __syncthreads();
    if (!any_live) return;
    // shared memory: C tile FP32 [128][64] complex (64 KB), B operand hi/lo (2 x 32 KB),
    // A operand hi/lo (2 x 32 KB)
    float2 *Ct = reinterpret_cast<float2 *>(sm);
    unsigned char *Bhi = sm + 65536, *Blo = Bhi + 32768, *Ahi = Blo + 32768, *Alo = Ahi + 32768;
    const float2 *Cg = T.C[cur];
    for (int i = tid; i < 128 * kTcSlotsPerTile; i += blockDim.x) {
        const int k = i / kTcSlotsPerTile, j = i % kTcSlotsPerTile;
        float2 v = make_float2(0.f, 0.f);
        if (k < R && s0 + j < T.S) v = Cg[(size_t)(r0 + k) * T.S + s0 + j];
        Ct[i] = v;
    }
    if (warp == 0) {
        tc_tmem_alloc(&tmem_base, 256);
        tc_tmem_relinquish();
    }
    if (tid == 0) tc_mbar_init(&mbar, 1);
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tw = tmem_base, tu = tmem_base + 128;
    const uint32_t idesc = tc_idesc_bf16_f32(128, 128);
    uint32_t phase = 0;
    bool ok = true, first_w = true, first_u = true;
    for (int f = 0; f < S.n_f && ok; ++f) {
        const int l = S.f_term[f];
        // A operand: the G^l tile (hi, lo), 16-byte copies
        const uint4 *src = reinterpret_cast<const uint4 *>(S.g_tiles + ((size_t)f * nt + rt) * 2 * 16384);
        uint4 *dst = reinterpret_cast<uint4 *>(Ahi);
        for (int i = tid; i < 2 * 32768 / 16; i += blockDim.x) dst[i] = __ldg(src + i);
        for (int which = 0; which < 2 && ok; ++which) {
            const float *cf = T.coef + ((size_t)which * S.L + l) * T.S + s0;
            // B operand: real column n = 2j + (Re, Im) of slot j, K = row k; coef_l(slot) * c
            for (int i = tid; i < 128 * 128; i += blockDim.x) {
                const int k = i / 128, nn = i % 128, j = nn >> 1;
                const float2 c = Ct[k * kTcSlotsPerTile + j];
                const float cv = (s0 + j < T.S) ? cf[j] : 0.f;
                const float x = cv * ((nn & 1) ? c.y : c.x);
                const uint16_t h = bf16_rn(x);
                const uint16_t lo = bf16_rn(x - bf16_f(h));
                const uint32_t off = tc_kmajor_offset(nn, k, 16);
                *reinterpret_cast<uint16_t *>(Bhi + off) = h;
                *reinterpret_cast<uint16_t *>(Blo + off) = lo;
            }
            tc_fence_proxy_async();
            __syncthreads();
            tc_fence_after_sync();
            if (tid == 0) {
                const uint32_t acc = which ? tu : tw;
                bool fst = which ? first_u : first_w;
                const uint32_t a_hi = tc_smem_addr(Ahi), a_lo = tc_smem_addr(Alo);
                const uint32_t b_hi = tc_smem_addr(Bhi), b_lo = tc_smem_addr(Blo);
                for (int ks = 0; ks < 8; ++ks) {
                    const uint32_t o = ks * 256;
                    tc_mma_bf16(acc, tc_sdesc(a_hi + o, 128, 2048), tc_sdesc(b_hi + o, 128, 2048), idesc, !fst);
                    tc_mma_bf16(acc, tc_sdesc(a_hi + o, 128, 2048), tc_sdesc(b_lo + o, 128, 2048), idesc, true);
                    tc_mma_bf16(acc, tc_sdesc(a_lo + o, 128, 2048), tc_sdesc(b_hi + o, 128, 2048), idesc, true);
                    fst = false;
                }
                tc_commit(&mbar);
            }
            if (which) first_u = false; else first_w = false;
            // the B buffers are rewritten next: wait for these MMAs
            ok = tc_mbar_wait(&mbar, phase, kTcWait);
            phase ^= 1u;
            tc_fence_after_sync();
            __syncthreads();
        }
    }
    // epilogue: lane = row of the tile; identity terms added from the FP32 tile
    if (ok && !first_w) {
        const int row = warp * 32 + lane;
        const float *vi = T.vid + s0, *dvi = T.vid + T.S + s0;
        for (int c = 0; c < 128; c += 8) {
            float vw[8], vu[8];
            tc_ld_32x32b_x8(tw + ((uint32_t)(warp * 32) << 16) + c, vw);
            tc_ld_32x32b_x8(tu + ((uint32_t)(warp * 32) << 16) + c, vu);
            tc_wait_ld();
            if (row < R)
                for (int q = 0; q < 4; ++q) {
                    const int j = c / 2 + q;
                    if (s0 + j >= T.S) continue;
                    const float2 cc = Ct[row * kTcSlotsPerTile + j];
                    const size_t o = (size_t)(r0 + row) * T.S + s0 + j;
                    T.W[o] = make_float2(vw[2 * q] + vi[j] * cc.x, vw[2 * q + 1] + vi[j] * cc.y);
                    T.U[o] = make_float2(vu[2 * q] + dvi[j] * cc.x, vu[2 * q + 1] + dvi[j] * cc.y);
                }
        }
    } else if (!ok && tid == 0) {
        atomicOr(T.live + 1, 1);  // error flag: a bounded wait ran out
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc_tmem_dealloc(tmem_base, 256);
}

// contraction for systems whose terms are all identities (no stored G): w = v_id c, u = v'_id c
__global__ void k_tc_identity(TcState T, int cur)
{
    const DevSys &S = *T.sys;
    const size_t tot = (size_t)S.n * T.S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % T.S);
        const float2 c = T.C[cur][i];
        T.W[i] = make_float2(T.vid[s] * c.x, T.vid[s] * c.y);
        T.U[i] = make_float2(T.vid[T.S + s] * c.x, T.vid[T.S + s] * c.y);
    }
}

// ---------------------------------------------------------------------------------------------
// the update of one element (row r, slot sl) from w = M c and u = M' c (Eq. 5, RK4); adds its
// force, torque and (stage 0) diagnostic contributions to part[6]
__device__ __forceinline__ void tc_elem(const TcState &T, const DevSys &S, int s, int cur, int r, int sl, int st,
                                        float2 w, float2 u, double *part)
{
    const int nxt = cur ^ 1;
    const size_t e = (size_t)r * T.S + sl;
    const float2 *PHc = (s == 0 || s == 3) ? T.PHa : T.PHb;
    const float2 *PHn = (s == 0 || s == 1) ? T.PHb : T.PHa;
    if (st == TS_WAIT && s == 3) {
        const float2 v = make_float2(r == T.slot[sl].s0 ? 1.0f : 0.0f, 0.0f);
        T.A[e] = v;
        T.ACC[e] = make_float2(0.f, 0.f);
        T.C[nxt][e] = v;
        return;
    }
    if (st != TS_ACTIVE && st != TS_FINAL) return;
    const float2 *Cc = T.C[cur];
    const float2 c = Cc[e];
    const float au = S.aupf[r], ad = S.adnf[r];
    const float2 cu = Cc[(size_t)S.up[r] * T.S + sl], cd = Cc[(size_t)S.dn[r] * T.S + sl];
    const float2 dc = make_float2(ad * cd.x - au * cu.x, ad * cd.y - au * cu.y);
    const int lev = S.lev[r];
    const float2 p = PHc[(size_t)lev * T.S + sl];
    const float2 da = make_float2(p.x * dc.x + p.y * dc.y, p.x * dc.y - p.y * dc.x);
    const float hp = T.hp[sl];
    float2 kk;
    kk.x = fmaf(hp, da.x, p.x * w.y - p.y * w.x);
    kk.y = fmaf(hp, da.y, -(p.x * w.x + p.y * w.y));
    part[0] -= (double)(c.x * u.x + c.y * u.y);
    part[1] -= (double)(dc.x * w.x + dc.y * w.y);
    const float2 a0 = T.A[e];
    if (s == 0) {
        const float pp = a0.x * a0.x + a0.y * a0.y;
        part[2] += (double)(c.x * w.x + c.y * w.y);
        part[3] += (double)pp;
        part[4] += S.lev_energy[lev] * (double)pp;
        part[5] += (double)(a0.x * da.y - a0.y * da.x);
    }
    if (st == TS_FINAL) {
        if (s == 0) {
            const size_t oo = (size_t)T.slot[sl].traj * T.nmax + S.perm[r];
            if (T.pop) T.pop[oo] = (double)(a0.x * a0.x + a0.y * a0.y);
            if (T.amp) { T.amp[2 * oo] = a0.x; T.amp[2 * oo + 1] = a0.y; }
        }
        return;
    }
    const float dtj = T.dtf[sl];
    float2 acc = T.ACC[e];
    if (s == 0) {
        acc = make_float2(kk.x + acc.x, kk.y + acc.y);  // acc holds the last rounding error
    } else {
        const float wg = (s == 1 || s == 2) ? 2.0f : 1.0f;
        acc.x = fmaf(wg, kk.x, acc.x);
        acc.y = fmaf(wg, kk.y, acc.y);
    }
    if (s == 3) {
        // compensated a + (dt/6) acc (two-sum); the rounding error goes to the accumulator
        const float h6 = dtj * (1.0f / 6.0f), ih6 = 6.0f / dtj;
        const float ix = h6 * acc.x, iy = h6 * acc.y;
        const float sx = __fadd_rn(a0.x, ix), sy = __fadd_rn(a0.y, iy);
        const float bx = __fsub_rn(sx, a0.x), by = __fsub_rn(sy, a0.y);
        const float ex = __fadd_rn(__fsub_rn(a0.x, __fsub_rn(sx, bx)), __fsub_rn(ix, bx));
        const float ey = __fadd_rn(__fsub_rn(a0.y, __fsub_rn(sy, by)), __fsub_rn(iy, by));
        T.A[e] = make_float2(sx, sy);
        T.ACC[e] = make_float2(ex * ih6, ey * ih6);
        const float2 q = PHn[(size_t)lev * T.S + sl];
        T.C[nxt][e] = make_float2(q.x * sx - q.y * sy, q.x * sy + q.y * sx);
    } else {
        T.ACC[e] = acc;
        const float bn = s == 2 ? dtj : 0.5f * dtj;
        const float2 yn = make_float2(fmaf(bn, kk.x, a0.x), fmaf(bn, kk.y, a0.y));
        const float2 q = PHn[(size_t)lev * T.S + sl];
        T.C[nxt][e] = make_float2(q.x * yn.x - q.y * yn.y, q.x * yn.y + q.y * yn.x);
    }
}

// element update after k_tc_contract: block = kTcRows rows x 32 slots
__global__ void __launch_bounds__(256) k_tc_update(TcState T, int s, int cur)
{
    __shared__ double red[kTcRows][32][6];
    const DevSys &S = *T.sys;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int sl = blockIdx.x * 32 + tx, r = blockIdx.y * kTcRows + ty;
    double part[6] = {0, 0, 0, 0, 0, 0};
    if (sl < T.S && r < S.n) {
        const size_t e = (size_t)r * T.S + sl;
        tc_elem(T, S, s, cur, r, sl, T.state[sl], T.W[e], T.U[e], part);
    }
    for (int q = 0; q < 6; ++q) red[ty][tx][q] = part[q];
    __syncthreads();
    if (ty == 0 && sl < T.S) {
        double acc6[6] = {0, 0, 0, 0, 0, 0};
        for (int y = 0; y < kTcRows; ++y)
            for (int q = 0; q < 6; ++q) acc6[q] += red[y][tx][q];
        double *o = T.part + ((size_t)blockIdx.y * T.S + sl) * 6;
        for (int q = 0; q < 6; ++q) o[q] = acc6[q];
    }
}

// ---------------------------------------------------------------------------------------------
// per-slot work, FP64
__device__ void tc_locate(const DevSys &S, TSlot &m)
{
    const double R = m.qs[0];
    int k = (int)floor((R - S.r_min) * S.inv_h);
    k = k < 0 ? 0 : (k > S.n_int - 1 ? S.n_int - 1 : k);
    m.kint = k;
    m.x = R - (S.r_min + k * S.h);
    const double ir = 1.0 / R;
    m.phidot = m.qs[3] * m.inv_mu * ir * ir;
    if (R < S.r_min) m.status |= MQCT_TRAJ_TABLE_RANGE;
}

// spline values of the next stage, FP32 views, identity-term sums
__device__ void tc_publish(const TcState &T, const DevSys &S, int sl)
{
    const TSlot &m = T.slot[sl];
    T.state[sl] = m.state;
    if (m.state == TS_IDLE) {
        for (int l = 0; l < S.L; ++l) T.coef[(size_t)l * T.S + sl] = T.coef[((size_t)S.L + l) * T.S + sl] = 0.f;
        T.vid[sl] = T.vid[T.S + sl] = 0.f;
        T.hp[sl] = 0.f;
        T.dtf[sl] = 1.f;
        return;
    }
    float v0 = 0.f, d0 = 0.f;
    const float x = (float)m.x;
    for (int l = 0; l < S.L; ++l) {
        const float4 c = S.vcoef_f[(size_t)l * S.n_int + m.kint];
        const float v = fmaf(x, fmaf(x, fmaf(x, c.w, c.z), c.y), c.x);
        const float dv = fmaf(x, fmaf(3.0f * x, c.w, 2.0f * c.z), c.y);
        T.coef[(size_t)l * T.S + sl] = v;
        T.coef[((size_t)S.L + l) * T.S + sl] = dv;
        if ((S.id_mask >> l) & 1ull) { v0 += v; d0 += dv; }
    }
    T.vid[sl] = v0;
    T.vid[T.S + sl] = d0;
    T.hp[sl] = (float)(0.5 * m.phidot);
    T.dtf[sl] = (float)m.dt;
}

__device__ void tc_claim(const TcState &T, const DevSys &S, int sl)
{
    TSlot &m = T.slot[sl];
    for (;;) {
        const int item = atomicAdd(T.queue, 1);
        if (item >= T.n) {
            m.state = TS_IDLE;
            return;
        }
        const int t = T.order ? T.order[item] : item;
        const mqct_traj tr = T.trajs[t];
        const bool ok = tr.system_idx == 0 && tr.dt > 0.0 && tr.e_coll > 0.0 && tr.b >= 0.0 && tr.r0 > 0.0 &&
                        tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0 && tr.init_state >= 0 &&
                        tr.init_state < S.n;
        if (!ok) {
            if (T.diag) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                T.diag[t] = d;
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
        m.q[0] = tr.r0; m.q[2] = 0.0; m.q[3] = lz;
        m.q[1] = -sqrt(2.0 * S.mu * (tr.e_coll - m00) - lz * lz / (tr.r0 * tr.r0));
        for (int i = 0; i < 4; ++i) m.qs[i] = m.q[i];
        m.dt = tr.dt; m.r_end = tr.r_end; m.max_steps = tr.max_steps;
        m.ndev = m.edev = m.jdev = 0.0;
        m.inv_mu = 1.0 / S.mu;
        m.status = 0; m.steps = 0; m.traj = t; m.s0 = s0;
        m.state = TS_WAIT;
        m.kint = k; m.x = x; m.phidot = 0.0;
        return;
    }
}

// a slot that starts a trajectory: phases of t = 0 and t = dt/2
__device__ void tc_start_phases(const TcState &T, const DevSys &S, int sl)
{
    const TSlot &m = T.slot[sl];
    for (int l = 0; l < S.n_levels; ++l) {
        T.PHa[(size_t)l * T.S + sl] = make_float2(1.f, 0.f);
        T.PHb[(size_t)l * T.S + sl] = tc_phase(S.lev_energy[l], 0.5 * m.dt);
    }
}

__global__ void k_tc_init(TcState T)
{
    const DevSys &S = *T.sys;
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= T.S) return;
    tc_claim(T, S, sl);
    TSlot &m = T.slot[sl];
    if (m.state == TS_WAIT) {
        for (int r = 0; r < S.n; ++r) {
            const float2 v = make_float2(r == m.s0 ? 1.0f : 0.0f, 0.0f);
            const size_t e = (size_t)r * T.S + sl;
            T.A[e] = v; T.ACC[e] = make_float2(0.f, 0.f); T.C[0][e] = v;
        }
        m.state = m.max_steps > 0 ? TS_ACTIVE : TS_FINAL;
        if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
        tc_locate(S, m);
        tc_start_phases(T, S, sl);
    }
    tc_publish(T, S, sl);
}

__global__ void k_tc_slots(TcState T, int s, int n_rowblocks)
{
    const DevSys &S = *T.sys;
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= T.S) return;
    TSlot &m = T.slot[sl];
    double F = 0, Tq = 0, V = 0, NR = 0, ER = 0, JY = 0;
    for (int b = 0; b < n_rowblocks; ++b) {
        const double *p = T.part + ((size_t)b * T.S + sl) * 6;
        F += p[0]; Tq += p[1];
        if (s == 0) { V += p[2]; NR += p[3]; ER += p[4]; JY += p[5]; }
    }
    if (m.state == TS_ACTIVE || m.state == TS_FINAL) {
        const double R = m.qs[0], PR = m.qs[1], PP = m.qs[3], imu = m.inv_mu;
        const double ir = 1.0 / R, ir2 = ir * ir;
        if (s == 0) {
            const double et = 0.5 * imu * (PR * PR + PP * PP * ir2) + ER + V;
            const double jt = PP + 0.5 * JY;
            if (m.steps == 0) { m.e0 = et; m.j0 = jt; }
            m.ndev = fmax(m.ndev, fabs(NR - 1.0));
            m.edev = fmax(m.edev, fabs(et - m.e0));
            m.jdev = fmax(m.jdev, fabs(jt - m.j0));
        }
        if (m.state == TS_FINAL) {
            if (s == 0) {
                if (T.diag) {
                    mqct_diag d;
                    d.steps = m.steps; d.status = m.status;
                    d.norm_dev = m.ndev; d.energy_dev = m.edev; d.angmom_dev = m.jdev;
                    d.t_final = m.steps * m.dt;
                    T.diag[m.traj] = d;
                }
                tc_claim(T, S, sl);  // WAIT (column initialised at stage 3) or IDLE
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
                if (!fin || (m.q[0] >= m.r_end && m.q[1] > 0.0)) m.state = TS_FINAL;
                else if (m.steps >= m.max_steps) { m.status |= MQCT_TRAJ_MAX_STEPS; m.state = TS_FINAL; }
            }
            if (!(m.status & MQCT_TRAJ_NONFINITE)) tc_locate(S, m);
            // phase factors needed ahead: after stage 1 the integer time t + dt, after stage 3
            // the half time of the next step
            if (s == 1)
                for (int l = 0; l < S.n_levels; ++l)
                    T.PHa[(size_t)l * T.S + sl] = tc_phase(S.lev_energy[l], m.steps * m.dt + m.dt);
            if (s == 3 && m.state == TS_ACTIVE)
                for (int l = 0; l < S.n_levels; ++l)
                    T.PHb[(size_t)l * T.S + sl] = tc_phase(S.lev_energy[l], m.steps * m.dt + 0.5 * m.dt);
        }
    } else if (m.state == TS_WAIT && s == 3) {
        m.state = m.max_steps > 0 ? TS_ACTIVE : TS_FINAL;
        if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
        tc_locate(S, m);
        tc_start_phases(T, S, sl);
    }
    tc_publish(T, S, sl);
    if (s == 3 && m.state != TS_IDLE) atomicAdd(T.live, 1);
}

}  // namespace

mqct_status run_tc_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st)
{
    const int n = h.n;
    int S = std::min(a.n, 8192);
    S = (S + kTcSlotsPerTile - 1) / kTcSlotsPerTile * kTcSlotsPerTile;
    const int n_rowblocks = (n + kTcRows - 1) / kTcRows;
    std::vector<void *> tmp;
    cudaError_t e = cudaSuccess;
    auto get = [&](void **p, size_t b) {
        if (e != cudaSuccess) return;
        e = cudaMallocAsync(p, b ? b : 16, st);
        if (e == cudaSuccess) tmp.push_back(*p);
    };
    auto cleanup = [&]() { for (void *p : tmp) cudaFreeAsync(p, st); };
    TcState T;
    std::memset(&T, 0, sizeof(T));
    T.sys = a.sys; T.trajs = a.trajs; T.order = a.order; T.n = a.n; T.S = S; T.queue = a.queue;
    T.pop = a.pop; T.amp = a.amp; T.diag = a.diag; T.nmax = a.nmax;
    const size_t ns = (size_t)n * S;
    get((void **)&T.live, 2 * sizeof(int));
    get((void **)&T.C[0], sizeof(float2) * ns);
    get((void **)&T.C[1], sizeof(float2) * ns);
    get((void **)&T.A, sizeof(float2) * ns);
    get((void **)&T.ACC, sizeof(float2) * ns);
    get((void **)&T.W, sizeof(float2) * ns);
    get((void **)&T.U, sizeof(float2) * ns);
    get((void **)&T.coef, sizeof(float) * 2 * (size_t)h.L * S);
    get((void **)&T.vid, sizeof(float) * 2 * (size_t)S);
    get((void **)&T.hp, sizeof(float) * S);
    get((void **)&T.dtf, sizeof(float) * S);
    get((void **)&T.state, sizeof(int) * S);
    get((void **)&T.PHa, sizeof(float2) * (size_t)h.n_levels * S);
    get((void **)&T.PHb, sizeof(float2) * (size_t)h.n_levels * S);
    get((void **)&T.part, sizeof(double) * 6 * (size_t)n_rowblocks * S);
    get((void **)&T.slot, sizeof(TSlot) * (size_t)S);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync (tensor-core path scratch)");
    }
    const size_t smem = 65536 + 4 * 32768;
    if ((e = cudaFuncSetAttribute(k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    cudaMemsetAsync(T.live, 0, 2 * sizeof(int), st);
    k_tc_init<<<(S + 127) / 128, 128, 0, st>>>(T);
    const int n_ct = S / kTcSlotsPerTile;
    const dim3 ugrid((S + 31) / 32, n_rowblocks);
    // one chunk of steps, captured once as a graph
    const int chunk = 16;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaStreamCreate");
    }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(T.live, 0, sizeof(int), cap);
        for (int k = 0; k < chunk; ++k)
            for (int s = 0; s < 4; ++s) {
                const int cur = s & 1;
                if (h.n_f > 0) k_tc_contract<<<h.n_tiles * n_ct, 128, smem, cap>>>(T, cur);
                else k_tc_identity<<<4 * 152, 256, 0, cap>>>(T, cur);
                k_tc_update<<<ugrid, 256, 0, cap>>>(T, s, cur);
                k_tc_slots<<<(S + 127) / 128, 128, 0, cap>>>(T, s, n_rowblocks);
            }
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    int live[2] = {1, 0};
    long long chunks = 0;
    while (e == cudaSuccess && live[0] > 0 && !live[1]) {
        e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(live, T.live, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        ++chunks;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core path");
    if (live[1]) return fail(MQCT_ERR_TIMEOUT, "tensor-core path: a bounded MMA completion wait ran out");
    (void)chunks;
    return MQCT_OK;
}

}  // namespace mqct
