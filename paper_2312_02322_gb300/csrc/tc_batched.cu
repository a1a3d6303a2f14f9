// Stage-synchronous tensor-core trajectory path (factorised coupling, BF16x3 contraction).
//
// All trajectories in flight form one N x S block of amplitudes in global memory (S slots,
// one column per trajectory; finished slots are refilled from the device work queue).  Every
// RK4 stage runs two kernels:
//   k_tc_stage  one CTA per row tile (packed m-blocks, <= 128 rows) and tile of 64 slots (128
//               real columns = Re, Im): tcgen05 GEMMs Y_l = G^l C from BF16 hi/lo splits (three
//               MMAs per K chunk: hi.hi + hi.lo + lo.hi, FP32 accumulation in tensor memory),
//               folded per slot into w = sum_l v_l(R_b) Y_l and u = sum_l v_l'(R_b) Y_l (Eq. 12);
//               then per element the Coriolis stencil, da/dt = -i exp(iEt) w + (dPhi/dt/2)
//               exp(iEt) D c (Eq. 5), the compensated RK4 accumulation and the next stage input,
//               with per-slot partial sums of force, torque and (stage 0) diagnostics;
//   k_tc_slots  one warp per eight slots (one lane per classical component and slot), FP64:
//               classical stage update (Eqs. 7-10), bookkeeping, stop rule, refill, the spline
//               values and phase factors of the next stage.
// The classical state lives in global memory with one lane per (component, slot) in k_tc_slots
// (eight slots per warp), phase arguments are 64-bit fixed-point turn counts and the partial sums
// are compensated FP32, so that neither kernel runs FP64 per element or per level.  Chunks of steps
// run inside a CUDA graph's conditional WHILE node whose condition the last kernel of each chunk
// sets from the number of live slots: one graph launch runs every trajectory to its end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"
#include "traj_common.cuh"

namespace mqct {

namespace {

constexpr int kTcSlotsPerTile = 64;  // 128 real columns
constexpr long long kTcWait = 1ll << 24;

enum { TS_IDLE = 0, TS_ACTIVE = 1, TS_FINAL = 2, TS_WAIT = 3 };

// per-slot values that are not per component (the four component lanes of a slot read them)
struct TSlot {
    double dt, h6, r_end, e0, j0, ndev, edev, jdev;
    double ir, i2m, phid, last_dt;  // 1/R, (1/mu)/R^2 and dPhi/dt of the current stage; dt of inc
    int status, steps, max_steps, traj, state, s0;
};

struct TcState {
    const DevSys *sys;
    const mqct_traj *trajs;
    const int *order;
    int n, S;                 // trajectories, slots
    int *queue;
    int *live;                // live slots after the last step; [1]: error flag
    double *pop, *amp;
    mqct_diag *diag;
    long long *t_start, *t_done;  // optional device clock (ns) at start / end of each trajectory
    int nmax, sys_idx;
    double inv_mu;
    float2 *C[2];             // [n][S] stage amplitudes (phase rotated), double buffered
    float2 *A, *ACC;          // [n][S]
    float *coef;              // [2][L][S] v_l and v_l' at each slot's stage R
    float *vid;               // [2][S] identity-term sums of v and v'
    float *hp, *dtf;          // [S] dPhi/dt / 2 and dt (FP32 views)
    int *state;               // [S]
    float2 *PHa, *PHb;        // [n_levels][S]
    unsigned long long *inc;  // [n_levels][S] fixed-point phase increments
    float2 *part;             // [n_tiles][6][S] per-row-tile partial sums (hi, lo)
    double *Q, *QS, *LACC;    // [4][S] classical state, stage input, RK4 accumulator
    TSlot *slot;              // [S]
    // PLAIN path (FP32 spline table): each slot's interval, local coordinate and dx/dR
    int *kint;                // [S]
    float *xs, *dinv;         // [S]
    int plain;
};

__device__ __forceinline__ uint16_t bf16_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// ---------------------------------------------------------------------------------------------
// the inputs of one element update (row r, slot sl) gathered from global memory
struct ElemIn {
    float2 c, cu, cd, p, q, a0, acc;
    float au, ad;
    int lev;
};

// gather: only loads, so that several elements' loads are in flight before any store
__device__ __forceinline__ void tc_elem_gather(const TcState &T, const DevSys &S, int s, int cur, int r, int sl,
                                               ElemIn &in)
{
    const size_t e = (size_t)r * T.S + sl;
    const float2 *Cc = T.C[cur];
    const float2 *PHc = (s == 0 || s == 3) ? T.PHa : T.PHb;
    const float2 *PHn = (s == 0 || s == 1) ? T.PHb : T.PHa;
    in.c = __ldg(Cc + e);
    in.au = __ldg(S.aupf + r);
    in.ad = __ldg(S.adnf + r);
    in.cu = __ldg(Cc + (size_t)__ldg(S.up + r) * T.S + sl);
    in.cd = __ldg(Cc + (size_t)__ldg(S.dn + r) * T.S + sl);
    in.lev = __ldg(S.lev + r);
    in.p = __ldg(PHc + (size_t)in.lev * T.S + sl);
    in.q = __ldg(PHn + (size_t)in.lev * T.S + sl);
    in.a0 = T.A[e];
    in.acc = T.ACC[e];
}

// the update of one element from w = M c and u = M' c (Eq. 5, RK4) and its inputs; adds its force,
// torque and (stage 0) diagnostic contributions to part[6] (FP32: a thread sums a few rows; the
// sums across threads, row tiles and the classical update are FP64 -- the FP64 pipe of this GPU is
// far too narrow for per-element FP64 arithmetic).  Returns what the caller stores: 0 nothing,
// 1 ACC and the next stage input C', 2 A, ACC and C', 3 the final amplitude a0 (a FINAL slot at
// stage 0).  A slot waiting for its first step (WAIT, stage 3) gets e_s0 (is_s0), zero, e_s0.
__device__ __forceinline__ int elem_core(int s, int st, bool is_s0, float2 c, float2 cu, float2 cd, float2 p,
                                         float2 q, float2 a0, float2 acc, float au, float ad, float elev, float hp,
                                         float dtj, float2 w, float2 u, float *part, float2 &a_out,
                                         float2 &acc_out, float2 &c_out)
{
    if (st == TS_WAIT && s == 3) {
        a_out = c_out = make_float2(is_s0 ? 1.0f : 0.0f, 0.0f);
        acc_out = make_float2(0.f, 0.f);
        return 2;
    }
    if (st != TS_ACTIVE && st != TS_FINAL) return 0;
    const float2 dc = make_float2(ad * cd.x - au * cu.x, ad * cd.y - au * cu.y);
    const float2 da = make_float2(p.x * dc.x + p.y * dc.y, p.x * dc.y - p.y * dc.x);
    float2 kk;
    kk.x = fmaf(hp, da.x, p.x * w.y - p.y * w.x);
    kk.y = fmaf(hp, da.y, -(p.x * w.x + p.y * w.y));
    part[0] -= c.x * u.x + c.y * u.y;
    part[1] -= dc.x * w.x + dc.y * w.y;
    if (s == 0) {
        const float pp = a0.x * a0.x + a0.y * a0.y;
        part[2] += c.x * w.x + c.y * w.y;
        part[3] += pp;
        part[4] += elev * pp;
        part[5] += a0.x * da.y - a0.y * da.x;
    }
    if (st == TS_FINAL) {
        a_out = a0;
        return s == 0 ? 3 : 0;
    }
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
        a_out = make_float2(sx, sy);
        acc_out = make_float2(ex * ih6, ey * ih6);
        c_out = make_float2(q.x * sx - q.y * sy, q.x * sy + q.y * sx);
        return 2;
    }
    acc_out = acc;
    const float bn = s == 2 ? dtj : 0.5f * dtj;
    const float2 yn = make_float2(fmaf(bn, kk.x, a0.x), fmaf(bn, kk.y, a0.y));
    c_out = make_float2(q.x * yn.x - q.y * yn.y, q.x * yn.y + q.y * yn.x);
    return 1;
}

// stores of one element's update (elem_core's return value); a FINAL slot's populations and
// amplitudes go to the caller's arrays in the caller's state order
__device__ __forceinline__ void elem_store(const TcState &T, const DevSys &S, int cur, int r, int sl, int mode,
                                           float2 a, float2 acc, float2 c)
{
    const size_t e = (size_t)r * T.S + sl;
    if (mode == 1) {
        T.ACC[e] = acc;
        T.C[cur ^ 1][e] = c;
    } else if (mode == 2) {
        T.A[e] = a;
        T.ACC[e] = acc;
        T.C[cur ^ 1][e] = c;
    } else if (mode == 3) {
        const size_t oo = (size_t)T.slot[sl].traj * T.nmax + S.perm[r];
        if (T.pop) T.pop[oo] = (double)(a.x * a.x + a.y * a.y);
        if (T.amp) { T.amp[2 * oo] = a.x; T.amp[2 * oo + 1] = a.y; }
    }
}

__device__ __forceinline__ void tc_elem_apply(const TcState &T, const DevSys &S, int s, int cur, int r, int sl,
                                              int st, const ElemIn &in, float2 w, float2 u, float *part)
{
    if (st == TS_IDLE) return;
    const bool is_s0 = st == TS_WAIT && s == 3 && r == T.slot[sl].s0;
    const float elev = (st == TS_ACTIVE || st == TS_FINAL) && s == 0 ? S.lev_energy_f[in.lev] : 0.f;
    float2 a, acc, c;
    const int mode = elem_core(s, st, is_s0, in.c, in.cu, in.cd, in.p, in.q, in.a0, in.acc, in.au, in.ad, elev,
                               T.hp[sl], T.dtf[sl], w, u, part, a, acc, c);
    elem_store(T, S, cur, r, sl, mode, a, acc, c);
}

// ---------------------------------------------------------------------------------------------
// one RK4 stage of every element: one CTA per (row tile, 64-slot tile).
//  - B operand: the tile's phase-rotated amplitudes as BF16 hi/lo, built once;
//  - the G^l tiles (BF16 hi/lo) stream through a two-deep shared-memory ring by bulk TMA copies
//    (warp 17); warp 16 issues, per term, the MMAs of the non-zero K chunks (three per chunk:
//    hi.hi + hi.lo + lo.hi) into one of two TMEM accumulators, Y_l = G^l C;
//  - sixteen epilogue warps (four per TMEM lane quadrant, 32 columns each) fold each term into
//    w += v_l Y_l and u += v_l' Y_l with the per-slot spline weights (Eq. 12), in registers;
//  - the element update of Eq. 5 and RK4 (tc_elem_gather / tc_elem_apply, four rows' loads in
//    flight per thread) runs on the staged w, u with the identity
//    terms added, and the per-slot partial sums of force, torque and diagnostics over the
//    tile's rows go to part[row tile][slot].
constexpr int kTcEpiWarps = 16;
constexpr int kTcMmaWarp = kTcEpiWarps, kTcLoadWarp = kTcEpiWarps + 1;
constexpr int kTcThreads = 32 * (kTcEpiWarps + 2);
constexpr uint32_t kTcTileBytes = 2u * 128u * 128u * 2u;  // a G tile or the B operand, hi + lo
constexpr size_t kTcSmemFixed = 3 * (size_t)kTcTileBytes;  // A ring (2) + B operand
constexpr int kTcWs = kTcSlotsPerTile + 1;                  // padded row of the staged w, u

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_stage(TcState T, int s, int cur)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_mma[2], bar_epi[2], bar_drain;
    __shared__ uint32_t tmem_base;
    __shared__ int any_live, err;
    const DevSys &S = *T.sys;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = S.n_tiles, nf = S.n_f;
    const int rt = blockIdx.x % nt, ct = blockIdx.x / nt;
    const int r0 = S.tile_r0[rt], R = S.tile_r0[rt + 1] - r0;
    const int s0 = ct * kTcSlotsPerTile;
    if (tid == 0) { any_live = 0; err = 0; }
    __syncthreads();
    if (tid < kTcSlotsPerTile) {
        const int st = T.state[s0 + tid];
        if (st != TS_IDLE) any_live = 1;
    }
    __syncthreads();
    if (!any_live) return;
    unsigned char *Aring = sm, *Bop = sm + 2 * kTcTileBytes;
    float *s_v = reinterpret_cast<float *>(sm + kTcSmemFixed), *s_dv = s_v + nf * kTcSlotsPerTile;
    const float2 *Cg = T.C[cur];
    // per-term spline weights of the tile's slots
    for (int i = tid; i < nf * kTcSlotsPerTile; i += kTcThreads) {
        const int f = i / kTcSlotsPerTile, j = i % kTcSlotsPerTile, l = S.f_term[f];
        s_v[i] = T.coef[(size_t)l * T.S + s0 + j];
        s_dv[i] = T.coef[((size_t)S.L + l) * T.S + s0 + j];
    }
    // B operand: real column n = 2j + (Re, Im) of slot j, K = row k of the tile; 8 rows of one
    // slot per task, written as 16-byte core-matrix rows
    for (int task = tid; task < kTcSlotsPerTile * 16; task += kTcThreads) {
        const int j = task % kTcSlotsPerTile, o = task / kTcSlotsPerTile;
        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
            const int k = 8 * o + i;
            if (k < R) c0 = Cg[(size_t)(r0 + k) * T.S + s0 + j];
            if (k + 1 < R) c1 = Cg[(size_t)(r0 + k + 1) * T.S + s0 + j];
            const uint16_t h0 = bf16_rn(c0.x), h1 = bf16_rn(c1.x), g0 = bf16_rn(c0.y), g1 = bf16_rn(c1.y);
            rh[i / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            ih[i / 2] = (uint32_t)g0 | ((uint32_t)g1 << 16);
            rl[i / 2] = (uint32_t)bf16_rn(c0.x - bf16_f(h0)) | ((uint32_t)bf16_rn(c1.x - bf16_f(h1)) << 16);
            il[i / 2] = (uint32_t)bf16_rn(c0.y - bf16_f(g0)) | ((uint32_t)bf16_rn(c1.y - bf16_f(g1)) << 16);
        }
        const uint32_t ore = tc_kmajor_offset(2 * j, 8 * o, 16), oim = tc_kmajor_offset(2 * j + 1, 8 * o, 16);
        *reinterpret_cast<uint4 *>(Bop + ore) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<uint4 *>(Bop + kTcTileBytes / 2 + ore) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<uint4 *>(Bop + oim) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<uint4 *>(Bop + kTcTileBytes / 2 + oim) = make_uint4(il[0], il[1], il[2], il[3]);
    }
    if (warp == kTcMmaWarp) {
        tc_tmem_alloc(&tmem_base, 256);
        tc_tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc_mbar_init(&bar_full[b], 1);
            tc_mbar_init(&bar_mma[b], 1);
            tc_mbar_init(&bar_epi[b], kTcEpiWarps);
        }
        tc_mbar_init(&bar_drain, 1);
    }
    tc_fence_proxy_async();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tbase = tmem_base;
    float w[32], u[32];
    if (warp == kTcLoadWarp) {
        // ---- bulk copies of the G tiles into the ring (lane 0); slot f & 1 is free once the
        // MMAs of term f - 2 completed
        if (lane == 0) {
            const unsigned char *gt = reinterpret_cast<const unsigned char *>(S.g_tiles);
            int f = 0;
            for (; f < nf; ++f) {
                const int b = f & 1;
                if (f >= 2 && !tc_mbar_wait(&bar_mma[b], ((f - 2) >> 1) & 1, kTcWait)) {
                    err = 1;
                    break;
                }
                tc_mbar_expect_tx(&bar_full[b], kTcTileBytes);
                tc_bulk_g2s(Aring + b * kTcTileBytes, gt + ((size_t)f * nt + rt) * kTcTileBytes, kTcTileBytes,
                            &bar_full[b]);
            }
            // before the buffers are released: the last copies issued have landed
            for (int k = f - 1; k >= 0 && k >= f - 2; --k) tc_mbar_wait(&bar_full[k & 1], (k >> 1) & 1, kTcWait);
        }
    } else if (warp == kTcMmaWarp) {
        // ---- MMA issue (lane 0)
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_bf16_f32(128, 128);
            const uint32_t b_hi = tc_smem_addr(Bop), b_lo = b_hi + kTcTileBytes / 2;
            for (int f = 0; f < nf; ++f) {
                const int b = f & 1;
                bool ok = tc_mbar_wait(&bar_full[b], (f >> 1) & 1, kTcWait);
                if (ok && f >= 2) ok = tc_mbar_wait(&bar_epi[b], ((f - 2) >> 1) & 1, kTcWait);
                if (!ok) {
                    // the MMAs already issued complete before the accumulators are released
                    err = 1;
                    tc_commit(&bar_drain);
                    tc_mbar_wait(&bar_drain, 0, kTcWait);
                    break;
                }
                tc_fence_after_sync();
                const uint32_t a_hi = tc_smem_addr(Aring + b * kTcTileBytes), a_lo = a_hi + kTcTileBytes / 2;
                const uint32_t d = tbase + 128u * b;
                const uint32_t km = S.g_kmask[(size_t)f * nt + rt];
                bool acc = false;
                for (int ks = 0; ks < 8; ++ks) {
                    if (!((km >> ks) & 1u)) continue;
                    const uint32_t o = ks * 256;
                    tc_mma_bf16(d, tc_sdesc(a_hi + o, 128, 2048), tc_sdesc(b_hi + o, 128, 2048), idesc, acc);
                    tc_mma_bf16(d, tc_sdesc(a_hi + o, 128, 2048), tc_sdesc(b_lo + o, 128, 2048), idesc, true);
                    tc_mma_bf16(d, tc_sdesc(a_lo + o, 128, 2048), tc_sdesc(b_hi + o, 128, 2048), idesc, true);
                    acc = true;
                }
                tc_commit(&bar_mma[b]);
            }
        }
    } else {
        // ---- epilogue warps: lanes of quadrant warp % 4, columns 32 * (warp / 4) .. + 31
        const int q = warp & 3, hcol = 32 * (warp >> 2);
#pragma unroll
        for (int i = 0; i < 32; ++i) { w[i] = 0.f; u[i] = 0.f; }
        for (int f = 0; f < nf; ++f) {
            const int b = f & 1;
            if (!tc_mbar_wait(&bar_mma[b], (f >> 1) & 1, kTcWait)) { err = 1; break; }
            tc_fence_after_sync();
            const float *vf = s_v + f * kTcSlotsPerTile + hcol / 2, *dvf = s_dv + f * kTcSlotsPerTile + hcol / 2;
            const uint32_t ta = tbase + 128u * b + ((uint32_t)(32 * q) << 16) + hcol;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t d[16];
                tc_ld16_raw(ta + 16 * hh, d);
                tc_wait_ld_16(d);
#pragma unroll
                for (int c = 0; c < 16; c += 4) {
                    const float2 v2 = *reinterpret_cast<const float2 *>(vf + 8 * hh + (c >> 1));
                    const float2 dv2 = *reinterpret_cast<const float2 *>(dvf + 8 * hh + (c >> 1));
                    const int o = 16 * hh + c;
                    w[o] = fmaf(v2.x, __uint_as_float(d[c]), w[o]);
                    w[o + 1] = fmaf(v2.x, __uint_as_float(d[c + 1]), w[o + 1]);
                    w[o + 2] = fmaf(v2.y, __uint_as_float(d[c + 2]), w[o + 2]);
                    w[o + 3] = fmaf(v2.y, __uint_as_float(d[c + 3]), w[o + 3]);
                    u[o] = fmaf(dv2.x, __uint_as_float(d[c]), u[o]);
                    u[o + 1] = fmaf(dv2.x, __uint_as_float(d[c + 1]), u[o + 1]);
                    u[o + 2] = fmaf(dv2.y, __uint_as_float(d[c + 2]), u[o + 2]);
                    u[o + 3] = fmaf(dv2.y, __uint_as_float(d[c + 3]), u[o + 3]);
                }
            }
            tc_fence_before_sync();
            __syncwarp();
            if (lane == 0) tc_mbar_arrive(&bar_epi[b]);
        }
    }
    __syncthreads();
    // stage w and u through shared memory (the ring and B buffers are free now)
    float2 *Wst = reinterpret_cast<float2 *>(sm), *Ust = Wst + 128 * kTcWs;
    float *red = reinterpret_cast<float *>(Ust + 128 * kTcWs);  // [8][64][6]
    if (!err && warp < kTcEpiWarps) {
        const int row = 32 * (warp & 3) + lane, j0 = 16 * (warp >> 2);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            Wst[row * kTcWs + j0 + i] = make_float2(w[2 * i], w[2 * i + 1]);
            Ust[row * kTcWs + j0 + i] = make_float2(u[2 * i], u[2 * i + 1]);
        }
    }
    __syncthreads();
    if (!err) {
        // element update: thread (row group g, slot j) takes rows g, g + 8, ... of slot j
        if (tid < 8 * kTcSlotsPerTile) {
            const int j = tid % kTcSlotsPerTile, g = tid / kTcSlotsPerTile, sl = s0 + j;
            const int st = T.state[sl];
            const float vi = T.vid[sl], dvi = T.vid[T.S + sl];
            float part[6] = {0, 0, 0, 0, 0, 0};
            const bool work = st == TS_ACTIVE || st == TS_FINAL;
            constexpr int kB = 4;  // rows gathered before any is updated
            for (int rb = g; rb < R; rb += 8 * kB) {
                ElemIn in[kB];
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const int row = rb + 8 * k;
                    if (work && row < R) tc_elem_gather(T, S, s, cur, r0 + row, sl, in[k]);
                }
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const int row = rb + 8 * k;
                    if (row >= R) continue;
                    float2 wt = make_float2(0.f, 0.f), ut = wt;
                    if (work) {
                        const float2 c = in[k].c, ws = Wst[row * kTcWs + j], us = Ust[row * kTcWs + j];
                        wt = make_float2(fmaf(vi, c.x, ws.x), fmaf(vi, c.y, ws.y));
                        ut = make_float2(fmaf(dvi, c.x, us.x), fmaf(dvi, c.y, us.y));
                    }
                    tc_elem_apply(T, S, s, cur, r0 + row, sl, st, in[k], wt, ut, part);
                }
            }
            for (int k = 0; k < 6; ++k) red[(g * kTcSlotsPerTile + j) * 6 + k] = part[k];
        }
        __syncthreads();
        if (tid < kTcSlotsPerTile) {
            // the eight row groups of the tile, compensated
            for (int k = 0; k < 6; ++k) {
                float hi = 0.f, lo = 0.f;
                for (int g = 0; g < 8; ++g) {
                    float e2;
                    two_sum(hi, red[(g * kTcSlotsPerTile + tid) * 6 + k], hi, e2);
                    lo += e2;
                }
                T.part[((size_t)rt * 6 + k) * T.S + s0 + tid] = make_float2(hi, lo);
            }
        }
    } else if (tid == 0) {
        atomicOr(T.live + 1, 1);  // error flag: a bounded wait ran out
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == kTcMmaWarp) tc_tmem_dealloc(tbase, 256);
}

// ---------------------------------------------------------------------------------------------
// one RK4 stage of every element on the PLAIN path with FP32 spline tables (bases too large for
// shared memory, Sec. III): one CTA per (block of 256 rows, tile of 32 consecutive slots); lane =
// slot, each warp takes one 32-row slice row by row.  Per element of a row's sliced-ELL list the
// column index is one broadcast load, the amplitudes of the 32 slots one 256-byte load, and the
// float4 (c0..c3) of each lane's interval a gather that lanes in the same interval share:
//   w = sum_c M_rc(x) C_c,   u = (dx/dR) sum_c M'_rc(x) C_c,
// then the element update of Eq. 5 and RK4 (every load coalesced over the slots) and the per-slot
// partial sums of force, torque and diagnostics over the 256 rows (compensated FP32 across warps).
constexpr int kSpWarps = 8, kSpTile = 32;

__global__ void __launch_bounds__(32 * kSpWarps, 4) k_sp_stage(TcState T, int s, int cur)
{
    const DevSys &S = *T.sys;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sl = blockIdx.x * kSpTile + lane, rb = blockIdx.y;
    const int slice = rb * kSpWarps + warp;
    __shared__ float red[kSpWarps][6][kSpTile];
    __shared__ int any_;
    const int st = T.state[sl];
    if (threadIdx.x == 0) any_ = 0;
    __syncthreads();
    if (warp == 0 && __any_sync(0xffffffffu, st != TS_IDLE) && lane == 0) any_ = 1;
    __syncthreads();
    float part[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (any_ && slice < S.n_slices) {
        const bool need = st == TS_ACTIVE || (st == TS_FINAL && s == 0);
        const int kint = need ? T.kint[sl] : 0;
        const float x = T.xs[sl], dv = T.dinv[sl], hp = T.hp[sl], dtj = T.dtf[sl];
        const int row0 = st == TS_WAIT ? T.slot[sl].s0 : -1;
        const float4 *tab = S.T4f + (size_t)kint * S.nnz_pad;
        const float2 *Cc = T.C[cur];
        const float2 *PHc = (s == 0 || s == 3) ? T.PHa : T.PHb;
        const float2 *PHn = (s == 0 || s == 1) ? T.PHb : T.PHa;
        const int off = S.sl_off[slice], width = (S.sl_off[slice + 1] - off) / kSlice;
        const int r_end = min(S.n, (slice + 1) * kSlice);
        for (int r = slice * kSlice; r < r_end; ++r) {
            const int rl = r - slice * kSlice;
            float2 w = make_float2(0.f, 0.f), u = make_float2(0.f, 0.f);
            if (need) {
                int e = 0;
                for (; e + 4 <= width; e += 4) {
                    int col[4];
                    float4 c[4];
                    float2 z[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const size_t ei = (size_t)off + (size_t)(e + i) * kSlice + rl;
                        col[i] = __ldg(S.cols + ei);
                        c[i] = __ldg(tab + ei);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) z[i] = __ldg(Cc + (size_t)col[i] * T.S + sl);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float m = fmaf(fmaf(fmaf(c[i].w, x, c[i].z), x, c[i].y), x, c[i].x);
                        const float md = fmaf(fmaf(3.0f * c[i].w, x, 2.0f * c[i].z), x, c[i].y);
                        w.x = fmaf(m, z[i].x, w.x);
                        w.y = fmaf(m, z[i].y, w.y);
                        u.x = fmaf(md, z[i].x, u.x);
                        u.y = fmaf(md, z[i].y, u.y);
                    }
                }
                for (; e < width; ++e) {
                    const size_t ei = (size_t)off + (size_t)e * kSlice + rl;
                    const float4 c = __ldg(tab + ei);
                    const float2 z = __ldg(Cc + (size_t)__ldg(S.cols + ei) * T.S + sl);
                    const float m = fmaf(fmaf(fmaf(c.w, x, c.z), x, c.y), x, c.x);
                    const float md = fmaf(fmaf(3.0f * c.w, x, 2.0f * c.z), x, c.y);
                    w.x = fmaf(m, z.x, w.x);
                    w.y = fmaf(m, z.y, w.y);
                    u.x = fmaf(md, z.x, u.x);
                    u.y = fmaf(md, z.y, u.y);
                }
            }
            if (st == TS_IDLE) continue;
            const int lev = __ldg(S.lev + r);
            const size_t e0 = (size_t)r * T.S + sl;
            const float2 c = __ldg(Cc + e0);
            const float2 cu = __ldg(Cc + (size_t)__ldg(S.up + r) * T.S + sl);
            const float2 cd = __ldg(Cc + (size_t)__ldg(S.dn + r) * T.S + sl);
            const float2 p = __ldg(PHc + (size_t)lev * T.S + sl), q = __ldg(PHn + (size_t)lev * T.S + sl);
            const float2 a0 = T.A[e0], acc = T.ACC[e0];
            const float au = __ldg(S.aupf + r), ad = __ldg(S.adnf + r), elev = S.lev_energy_f[lev];
            const float2 uu = make_float2(u.x * dv, u.y * dv);
            float2 ao, acco, co;
            const int mode = elem_core(s, st, r == row0, c, cu, cd, p, q, a0, acc, au, ad, elev, hp, dtj, w, uu, part,
                                       ao, acco, co);
            elem_store(T, S, cur, r, sl, mode, ao, acco, co);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) red[warp][k][lane] = part[k];
    __syncthreads();
    if (threadIdx.x < 6 * kSpTile) {
        const int k = threadIdx.x / kSpTile, j = threadIdx.x % kSpTile;
        float hi = 0.f, lo = 0.f;
        for (int g = 0; g < kSpWarps; ++g) {
            float e2;
            two_sum(hi, red[g][k][j], hi, e2);
            lo += e2;
        }
        T.part[((size_t)rb * 6 + k) * T.S + blockIdx.x * kSpTile + j] = make_float2(hi, lo);
    }
}

// ---------------------------------------------------------------------------------------------
// per-slot work: one warp per eight slots, lane 8 c + j carries component c of (R, P_R, Phi, P_Phi)
// of slot j, so one FP64 instruction advances four components of eight trajectories; every lane
// of the warp runs the same instructions (lanes of slots >= S compute on copies and store nothing)
struct SlotLane {
    int sc, sj, sl, slc;
    bool valid;
    unsigned m4;  // the four lanes of this slot
};

__device__ __forceinline__ SlotLane slot_lane(const TcState &T)
{
    SlotLane L;
    const int lane = threadIdx.x & 31, warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    L.sc = lane >> 3;
    L.sj = lane & 7;
    L.sl = 8 * warp + L.sj;
    L.valid = L.sl < T.S;
    L.slc = L.valid ? L.sl : T.S - 1;
    L.m4 = 0x01010101u << L.sj;
    return L;
}

// claim the next valid trajectory for slot L.sl (its four lanes together); returns the new state
// (WAIT: column initialised at the next stage 3, or IDLE) and sets the lane's component q
__device__ int tc_claim(const TcState &T, const DevSys &S, const SlotLane &L, double &q)
{
    TSlot &m = T.slot[L.sl];
    for (;;) {
        int item = 0;
        if (L.sc == 0) item = atomicAdd(T.queue, 1);
        item = __shfl_sync(L.m4, item, L.sj);
        if (item >= T.n) return TS_IDLE;
        const int t = T.order ? T.order[item] : item;
        const mqct_traj tr = T.trajs[t];
        if (!traj_valid(tr, S, T.sys_idx)) {
            if (T.diag && L.sc == 0) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                T.diag[t] = d;
            }
            __syncwarp(L.m4);
            continue;
        }
        if (T.t_start && L.sc == 0) T.t_start[t] = mqct_clock_ns();
        const int s0 = S.inv[tr.init_state];
        int k0;
        double x0;
        bool bl;
        locate_interval(S, tr.r0, k0, x0, bl);
        double mm = 0.0;  // initial mean field M_ss(r0): the four lanes split the terms
        for (int l = L.sc; l < S.L; l += 4) mm += spline_fp64(S, l, k0, x0) * S.diag_g[(size_t)l * S.n + s0];
        mm += __shfl_xor_sync(L.m4, mm, 8);
        mm += __shfl_xor_sync(L.m4, mm, 16);
        double q4[4];
        initial_state(S, tr, mm, q4);
        q = q4[L.sc];
        const bool new_dt = tr.dt != m.last_dt;
        __syncwarp(L.m4);
        if (L.sc == 0) {
            m.dt = tr.dt; m.h6 = tr.dt / 6.0; m.r_end = tr.r_end; m.max_steps = tr.max_steps;
            m.ndev = m.edev = m.jdev = 0.0;
            m.status = 0; m.steps = 0; m.traj = t; m.s0 = s0;
            m.last_dt = tr.dt;
        }
        if (new_dt)
            for (int l = L.sc; l < S.n_levels; l += 4) T.inc[(size_t)l * T.S + L.sl] = phase_increment(S.lev_energy[l], tr.dt);
        __syncwarp(L.m4);
        return TS_WAIT;
    }
}

// the quantities of the next stage at the slot's stage input qs: interval, spline values of every
// term (FP32 views), 1/R, (1/mu)/R^2, dPhi/dt; returns the TABLE_RANGE bit.  Called by every lane
// of the warp (publish: write the views of this slot).
__device__ __forceinline__ int tc_next_stage(const TcState &T, const DevSys &S, const SlotLane &L, double qs, bool publish,
                             double &ir, double &i2m, double &phid)
{
    const unsigned full = 0xffffffffu;
    const double R = __shfl_sync(full, qs, L.sj), PP = __shfl_sync(full, qs, 24 + L.sj);
    int k;
    double x;
    bool below;
    locate_interval(S, R, k, x, below);
    ir = 1.0 / R;
    i2m = T.inv_mu * ir * ir;
    phid = PP * i2m;
    if (T.plain) {
        // the element tables are evaluated by the stage kernel at (interval, x); derivatives carry
        // dx/dR (1/R on the logarithmic grid)
        if (publish && L.sc == 0) {
            T.kint[L.sl] = k;
            T.xs[L.sl] = (float)x;
            T.dinv[L.sl] = S.grid_log ? (float)ir : 1.0f;
            T.hp[L.sl] = (float)phid * 0.5f;
        }
        return below ? MQCT_TRAJ_TABLE_RANGE : 0;
    }
    const float xf = (float)x;
    float v0 = 0.f, d0 = 0.f;
    // the spline coefficients (a read-only table) of four terms per lane are loaded ahead
    for (int l0 = L.sc; l0 < S.L; l0 += 16) {
        float4 cf[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int l = l0 + 4 * i;
            cf[i] = l < S.L ? __ldg(S.vcoef_f + (size_t)l * S.n_int + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int l = l0 + 4 * i;
            if (l >= S.L) continue;
            const float4 c = cf[i];
            const float v = fmaf(xf, fmaf(xf, fmaf(xf, c.w, c.z), c.y), c.x);
            const float dv = fmaf(xf, fmaf(3.0f * xf, c.w, 2.0f * c.z), c.y);
            if (publish) {
                T.coef[(size_t)l * T.S + L.sl] = v;
                T.coef[((size_t)S.L + l) * T.S + L.sl] = dv;
            }
            if ((S.id_mask >> l) & 1ull) { v0 += v; d0 += dv; }
        }
    }
    v0 += __shfl_xor_sync(full, v0, 8);
    v0 += __shfl_xor_sync(full, v0, 16);
    d0 += __shfl_xor_sync(full, d0, 8);
    d0 += __shfl_xor_sync(full, d0, 16);
    if (publish && L.sc == 0) {
        T.vid[L.sl] = v0;
        T.vid[T.S + L.sl] = d0;
        T.hp[L.sl] = (float)phid * 0.5f;
    }
    return below ? MQCT_TRAJ_TABLE_RANGE : 0;
}

// an idle slot's published views
__device__ void tc_publish_idle(const TcState &T, const DevSys &S, const SlotLane &L)
{
    if (T.plain) {
        if (L.sc == 0) {
            T.kint[L.sl] = 0;
            T.xs[L.sl] = 0.f;
            T.dinv[L.sl] = 0.f;
            T.hp[L.sl] = 0.f;
            T.dtf[L.sl] = 1.f;
        }
        return;
    }
    for (int l = L.sc; l < S.L; l += 4) T.coef[(size_t)l * T.S + L.sl] = T.coef[((size_t)S.L + l) * T.S + L.sl] = 0.f;
    if (L.sc == 0) {
        T.vid[L.sl] = T.vid[T.S + L.sl] = 0.f;
        T.hp[L.sl] = 0.f;
        T.dtf[L.sl] = 1.f;
    }
}

// phase factors exp(-i E_l t) of the slot at stage time t = n_half dt / 2 into PH (the four lanes
// split the levels)
__device__ __forceinline__ void tc_phases(const TcState &T, const DevSys &S, const SlotLane &L, float2 *PH, unsigned n_half)
{
    // the increments are loaded four at a time ahead of the stores, so that the independent global
    // loads overlap instead of each waiting for the previous store
    constexpr int kB = 4;
    for (int l0 = L.sc; l0 < S.n_levels; l0 += 4 * kB) {
        unsigned long long v[kB];
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int l = l0 + 4 * i;
            v[i] = l < S.n_levels ? T.inc[(size_t)l * T.S + L.sl] : 0ull;
        }
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int l = l0 + 4 * i;
            if (l < S.n_levels) PH[(size_t)l * T.S + L.sl] = phase_factor(v[i], n_half);
        }
    }
}

// claim the first trajectory of every slot, initialise its column and views
__global__ void __launch_bounds__(128) k_tc_init(TcState T)
{
    const DevSys &S = *T.sys;
    const SlotLane L = slot_lane(T);
    const int lane = threadIdx.x & 31;
    double q = 0.0;
    int state = TS_IDLE;
    if (L.valid) {
        if (L.sc == 0) T.slot[L.sl].last_dt = -1.0;
        __syncwarp(L.m4);
        state = tc_claim(T, S, L, q);
    }
    double ir = 0.1, i2m = 0.0, phid = 0.0;
    const bool go = L.valid && state == TS_WAIT;
    const int tr = tc_next_stage(T, S, L, go ? q : 10.0, go, ir, i2m, phid);
    if (go) {
        TSlot &m = T.slot[L.sl];
        const int ms = m.max_steps;
        state = ms > 0 ? TS_ACTIVE : TS_FINAL;
        __syncwarp(L.m4);
        if (L.sc == 0) {
            m.status |= tr | (ms <= 0 ? MQCT_TRAJ_MAX_STEPS : 0);
            m.ir = ir; m.i2m = i2m; m.phid = phid;
            T.dtf[L.sl] = (float)m.dt;
        }
        tc_phases(T, S, L, T.PHb, 1u);
        for (int l = L.sc; l < S.n_levels; l += 4) T.PHa[(size_t)l * T.S + L.sl] = make_float2(1.f, 0.f);
    } else if (L.valid) {
        tc_publish_idle(T, S, L);
    }
    if (L.valid) {
        T.Q[(size_t)L.sc * T.S + L.sl] = q;
        T.QS[(size_t)L.sc * T.S + L.sl] = q;
        T.LACC[(size_t)L.sc * T.S + L.sl] = 0.0;
        if (L.sc == 0) {
            T.slot[L.sl].state = state;
            T.state[L.sl] = state;
        }
    }
    __syncwarp();
    // the columns of the warp's eight slots: e_s0, accumulator 0, input e_s0
    for (int j = 0; j < 8; ++j) {
        const int sl = 8 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) + j;
        if (sl >= T.S) break;
        const int st = T.slot[sl].state;
        if (st != TS_ACTIVE && st != TS_FINAL) continue;
        const int s0 = T.slot[sl].s0;
        for (int r = lane; r < S.n; r += 32) {
            const float2 v = make_float2(r == s0 ? 1.0f : 0.0f, 0.0f);
            const size_t e = (size_t)r * T.S + sl;
            T.A[e] = v; T.ACC[e] = make_float2(0.f, 0.f); T.C[0][e] = v;
        }
    }
}

// after the stage kernel of stage s: the row-tile partial sums of force, torque and diagnostics
// (compensated FP32, FP64 once per slot), bookkeeping (stage 0), the classical stage update
// (Eqs. 7-10), stop rule and refill, then the next stage's spline values, dPhi/dt and phase factors
__global__ void __launch_bounds__(128) k_tc_slots(TcState T, int s, int n_rowblocks)
{
    const DevSys &S = *T.sys;
    const unsigned full = 0xffffffffu;
    const SlotLane L = slot_lane(T);
    TSlot &m = T.slot[L.slc];
    int state = m.state;
    if (__all_sync(full, !L.valid || state == TS_IDLE)) return;  // published as idle when they became idle
    const size_t ci = (size_t)L.sc * T.S + L.slc;
    double q = T.Q[ci], qs = T.QS[ci], lacc = T.LACC[ci];
    auto comp = [&](double v, int c2) { return __shfl_sync(full, v, 8 * c2 + L.sj); };
    // row-tile sums: lane c sums quantity c (F, T, V, |a|^2), lanes c < 2 also c + 4 (E|a|^2, <J_y>)
    // (the partial sums of the previous launch are loaded four at a time ahead of the compensated
    // additions; a zero beyond the last row block leaves both parts unchanged)
    auto tsum = [&](int qq) {
        float hi = 0.f, lo = 0.f;
        for (int b0 = 0; b0 < n_rowblocks; b0 += 4) {
            float2 p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int b = b0 + i;
                p[i] = b < n_rowblocks ? __ldg(T.part + ((size_t)b * 6 + qq) * T.S + L.slc) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float e2;
                two_sum(hi, p[i].x, hi, e2);
                lo += e2 + p[i].y;
            }
        }
        return (double)hi + (double)lo;
    };
    const double v1 = tsum(L.sc), v2 = (s == 0 && L.sc < 2) ? tsum(4 + L.sc) : 0.0;
    const double F = comp(v1, 0), Tq = comp(v1, 1);
    const bool act = L.valid && state == TS_ACTIVE;
    int add_status = 0;
    if (s == 0) {
        // total energy, P_Phi + <J_y> and norm at the start of the step (or of the final state)
        const double V = comp(v1, 2), NR = comp(v1, 3), ER = comp(v2, 0), JY = comp(v2, 1);
        const double PR = comp(q, 1), PP = comp(q, 3);
        const double et = 0.5 * (T.inv_mu * PR * PR + PP * PP * m.i2m) + ER + V;
        const double jt = PP + 0.5 * JY;
        const int st0 = m.steps;
        const double e0 = st0 == 0 ? et : m.e0, j0 = st0 == 0 ? jt : m.j0;
        const double nd = fmax(m.ndev, fabs(NR - 1.0)), ed = fmax(m.edev, fabs(et - e0)),
                     jd = fmax(m.jdev, fabs(jt - j0));
        __syncwarp();
        if (L.valid && L.sc == 0 && (state == TS_ACTIVE || state == TS_FINAL)) {
            m.e0 = e0; m.j0 = j0; m.ndev = nd; m.edev = ed; m.jdev = jd;
        }
        __syncwarp();
        if (L.valid && state == TS_FINAL) {
            if (L.sc == 0) {
                if (T.diag) {
                    mqct_diag d;
                    d.steps = m.steps; d.status = m.status;
                    d.norm_dev = m.ndev; d.energy_dev = m.edev; d.angmom_dev = m.jdev;
                    d.t_final = m.steps * m.dt;
                    T.diag[m.traj] = d;
                }
                if (T.t_done) T.t_done[m.traj] = mqct_clock_ns();
            }
            __syncwarp(L.m4);
            state = tc_claim(T, S, L, q);  // WAIT (column initialised at stage 3) or IDLE
            qs = q;
            lacc = 0.0;
        }
    }
    {
        // derivative l_c: (P_R / mu, F + P_Phi^2/(mu R^3), dPhi/dt, torque)
        const double pr = comp(qs, 1), pp = comp(qs, 3);
        const double t1 = pp * m.phid * m.ir;
        const double X = L.sc == 0 ? pr : (L.sc == 1 ? F : (L.sc == 2 ? m.phid : Tq));
        const double alpha = L.sc == 0 ? T.inv_mu : 1.0, beta = L.sc == 1 ? t1 : 0.0;
        double qs2 = qs, lacc2 = lacc;
        stage_component(s, alpha, X, beta, 0.5 * m.dt, m.dt, m.h6, q, qs2, lacc2);
        if (act) { qs = qs2; lacc = lacc2; }
    }
    int steps = m.steps;
    if (s == 3) {
        const unsigned bad = __ballot_sync(full, act && !finite64(qs));
        const double R = comp(qs, 0), PR = comp(qs, 1);
        if (act) {
            q = qs;
            steps += 1;
            if ((bad >> L.sj) & 0x01010101u) {
                add_status |= MQCT_TRAJ_NONFINITE;
                state = TS_FINAL;
            } else if (ge_pos(R, m.r_end) && __double_as_longlong(PR) > 0) {
                state = TS_FINAL;
            } else if (steps >= m.max_steps) {
                add_status |= MQCT_TRAJ_MAX_STEPS;
                state = TS_FINAL;
            }
        }
    }
    const bool start = L.valid && state == TS_WAIT && s == 3;
    const bool next = (act && !(add_status & MQCT_TRAJ_NONFINITE)) || start;
    double ir = 0.1, i2m = 0.0, phid = 0.0;
    const int trng = tc_next_stage(T, S, L, next ? qs : 10.0, next, ir, i2m, phid);
    if (next) add_status |= trng;
    if (start) {
        const int ms = m.max_steps;
        state = ms > 0 ? TS_ACTIVE : TS_FINAL;
        if (ms <= 0) add_status |= MQCT_TRAJ_MAX_STEPS;
    }
    // phase factors needed ahead: after stage 1 the integer time t + dt, after stage 3 the half
    // time of the next step; a slot that starts at the next stage 0 gets t = 0 and t = dt/2
    if (start) {
        tc_phases(T, S, L, T.PHb, 1u);
        for (int l = L.sc; l < S.n_levels; l += 4) T.PHa[(size_t)l * T.S + L.sl] = make_float2(1.f, 0.f);
    } else if (act && state == TS_ACTIVE && s == 1) {
        tc_phases(T, S, L, T.PHa, 2u * steps + 2u);
    } else if (act && state == TS_ACTIVE && s == 3) {
        tc_phases(T, S, L, T.PHb, 2u * steps + 1u);
    }
    if (L.valid && state == TS_IDLE) tc_publish_idle(T, S, L);
    __syncwarp();
    if (L.valid) {
        T.Q[ci] = q;
        T.QS[ci] = qs;
        T.LACC[ci] = lacc;
        if (L.sc == 0) {
            if (next) { m.ir = ir; m.i2m = i2m; m.phid = phid; }
            m.status |= add_status;
            m.steps = steps;
            m.state = state;
            T.state[L.sl] = state;
            T.dtf[L.sl] = (float)m.dt;
        }
    }
    if (s == 3) {
        const unsigned live = __ballot_sync(full, L.valid && L.sc == 0 && state != TS_IDLE);
        if ((threadIdx.x & 31) == 0 && live) atomicAdd(T.live, __popc(live));
    }
}

// ---------------------------------------------------------------------------------------------
// PLAIN path, at the end of a chunk of steps: the slots are reordered by spline interval so that the
// 32 slots of a stage-kernel tile mostly read the same rows of the table (one transaction per element
// instead of one per slot); idle slots go last.  perm[new] = old by a stable counting sort (one
// thread: S <= 8192), then every per-slot and per-(row, slot) array is gathered into scratch and
// copied back.
struct SpSort {
    int *perm, *cnt;            // [S], [n_int + 2]
    TSlot *slot;                // scratch copies
    double *Q, *QS, *LACC;      // [4][S]
    int *state, *kint;
    float *hp, *dtf, *xs, *dinv;
    unsigned long long *inc;    // [n_levels][S]
    float2 *PHa, *PHb;          // [n_levels][S]
    float2 *A, *ACC;            // [n][S]; C[0] goes through C[1]
};

__global__ void k_sp_order(TcState T, SpSort P, int n_int)
{
    if (threadIdx.x != 0) return;
    const int S = T.S, nb = n_int + 1;  // bucket n_int: idle slots
    for (int b = 0; b <= nb; ++b) P.cnt[b] = 0;
    for (int i = 0; i < S; ++i) {
        const int k = T.state[i] == TS_IDLE ? n_int : min(max(T.kint[i], 0), n_int - 1);
        P.cnt[k + 1] += 1;
    }
    for (int b = 1; b <= nb; ++b) P.cnt[b] += P.cnt[b - 1];
    for (int i = 0; i < S; ++i) {
        const int k = T.state[i] == TS_IDLE ? n_int : min(max(T.kint[i], 0), n_int - 1);
        P.perm[P.cnt[k]++] = i;
    }
}

// gather into scratch (dir 0) or copy back (dir 1): per-slot arrays, one thread per slot
__global__ void k_sp_move_slots(TcState T, SpSort P, int n_levels, int dir)
{
    const int S = T.S;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        const int o = dir == 0 ? P.perm[i] : i;
        if (dir == 0) {
            P.slot[i] = T.slot[o];
            for (int c = 0; c < 4; ++c) {
                P.Q[(size_t)c * S + i] = T.Q[(size_t)c * S + o];
                P.QS[(size_t)c * S + i] = T.QS[(size_t)c * S + o];
                P.LACC[(size_t)c * S + i] = T.LACC[(size_t)c * S + o];
            }
            P.state[i] = T.state[o]; P.kint[i] = T.kint[o];
            P.hp[i] = T.hp[o]; P.dtf[i] = T.dtf[o]; P.xs[i] = T.xs[o]; P.dinv[i] = T.dinv[o];
            for (int l = 0; l < n_levels; ++l) {
                P.inc[(size_t)l * S + i] = T.inc[(size_t)l * S + o];
                P.PHa[(size_t)l * S + i] = T.PHa[(size_t)l * S + o];
                P.PHb[(size_t)l * S + i] = T.PHb[(size_t)l * S + o];
            }
        } else {
            T.slot[i] = P.slot[i];
            for (int c = 0; c < 4; ++c) {
                T.Q[(size_t)c * S + i] = P.Q[(size_t)c * S + i];
                T.QS[(size_t)c * S + i] = P.QS[(size_t)c * S + i];
                T.LACC[(size_t)c * S + i] = P.LACC[(size_t)c * S + i];
            }
            T.state[i] = P.state[i]; T.kint[i] = P.kint[i];
            T.hp[i] = P.hp[i]; T.dtf[i] = P.dtf[i]; T.xs[i] = P.xs[i]; T.dinv[i] = P.dinv[i];
            for (int l = 0; l < n_levels; ++l) {
                T.inc[(size_t)l * S + i] = P.inc[(size_t)l * S + i];
                T.PHa[(size_t)l * S + i] = P.PHa[(size_t)l * S + i];
                T.PHb[(size_t)l * S + i] = P.PHb[(size_t)l * S + i];
            }
        }
    }
}

// gather (dir 0: A, ACC into scratch, C[0] into C[1]) or copy back (dir 1), one thread per element
__global__ void k_sp_move_rows(TcState T, SpSort P, int n, int dir)
{
    const size_t S = T.S, total = (size_t)n * S;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        if (dir == 0) {
            const size_t r = e / S, i = e % S, o = r * S + P.perm[i];
            P.A[e] = T.A[o];
            P.ACC[e] = T.ACC[o];
            T.C[1][e] = T.C[0][o];
        } else {
            T.A[e] = P.A[e];
            T.ACC[e] = P.ACC[e];
            T.C[0][e] = T.C[1][e];
        }
    }
}

// the condition of the graph's WHILE node at the end of a chunk of steps: run another chunk while
// trajectories are live and no bounded wait has run out
__global__ void k_tc_continue(TcState T, cudaGraphConditionalHandle h)
{
    if (threadIdx.x == 0) {
        const int live = *((volatile int *)T.live), err = *((volatile int *)(T.live + 1));
        T.live[2] += 1;  // chunks run (launch accounting)
        if (h) cudaGraphSetConditional(h, live > 0 && !err ? 1u : 0u);
    }
}

__global__ void k_tc_reset_live(TcState T)
{
    if (threadIdx.x == 0) T.live[0] = 0;
}

}  // namespace

mqct_status run_tc_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st)
{
    const int n = h.n;
    // slot count: the contraction runs one CTA per SM per (row tile, 64-slot tile), and a stage
    // lasts about one CTA time per wave of CTAs, so the count of 64-slot tiles c maximises the
    // trajectories in flight per wave, min(want, c) / ceil(c * row tiles / SMs), over c up to two
    // full waves (the largest c among equals; trajectories beyond the slots wait for a refill);
    // a.tc_slots overrides (rounded up to 64)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt = std::max(1, h.n_tiles);
    const int two_waves = std::max(1, 2 * sms / nt);
    const int want = (a.n + kTcSlotsPerTile - 1) / kTcSlotsPerTile;
    int n_slot_tiles = 1;
    double best = 0.0;
    for (int c = 1; c <= std::max(1, std::min(want, two_waves)); ++c) {
        const double waves = std::ceil((double)c * nt / sms), rate = std::min(want, c) / waves;
        if (rate >= best) { best = rate; n_slot_tiles = c; }
    }
    if (a.tc_slots > 0) n_slot_tiles = (a.tc_slots + kTcSlotsPerTile - 1) / kTcSlotsPerTile;
    n_slot_tiles = std::max(1, std::min(n_slot_tiles, 8192 / kTcSlotsPerTile));
    int S = n_slot_tiles * kTcSlotsPerTile;
    int n_rowblocks = std::max(1, h.n_tiles);
    const bool plain = h.path == MQCT_PATH_PLAIN;
    if (plain) {
        // PLAIN path: every trajectory in a slot at once up to 4096 slots (tiles of 32 slots; the
        // stage kernel's CTAs are (256-row block, 32-slot tile)); a.tc_slots overrides (rounded to 32)
        S = a.tc_slots > 0 ? a.tc_slots : std::min(a.n, 4096);
        S = std::max(kSpTile, std::min(8192, (S + kSpTile - 1) / kSpTile * kSpTile));
        n_rowblocks = (h.n_slices + kSpWarps - 1) / kSpWarps;
    }
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
    T.pop = a.pop; T.amp = a.amp; T.diag = a.diag; T.nmax = a.nmax; T.sys_idx = a.sys_idx;
    T.t_start = a.t_start; T.t_done = a.t_done;
    T.inv_mu = 1.0 / h.mu;
    T.plain = plain ? 1 : 0;
    const size_t ns = (size_t)n * S;
    get((void **)&T.live, 4 * sizeof(int));
    get((void **)&T.C[0], sizeof(float2) * ns);
    get((void **)&T.C[1], sizeof(float2) * ns);
    get((void **)&T.A, sizeof(float2) * ns);
    get((void **)&T.ACC, sizeof(float2) * ns);
    get((void **)&T.coef, sizeof(float) * 2 * (size_t)h.L * S);
    get((void **)&T.vid, sizeof(float) * 2 * (size_t)S);
    get((void **)&T.hp, sizeof(float) * S);
    get((void **)&T.dtf, sizeof(float) * S);
    get((void **)&T.state, sizeof(int) * S);
    get((void **)&T.PHa, sizeof(float2) * (size_t)h.n_levels * S);
    get((void **)&T.PHb, sizeof(float2) * (size_t)h.n_levels * S);
    get((void **)&T.part, sizeof(float2) * 6 * (size_t)n_rowblocks * S);
    get((void **)&T.inc, sizeof(unsigned long long) * (size_t)h.n_levels * S);
    get((void **)&T.Q, sizeof(double) * 4 * (size_t)S);
    get((void **)&T.QS, sizeof(double) * 4 * (size_t)S);
    get((void **)&T.LACC, sizeof(double) * 4 * (size_t)S);
    get((void **)&T.slot, sizeof(TSlot) * (size_t)S);
    SpSort P;
    std::memset(&P, 0, sizeof(P));
    if (plain) {
        get((void **)&T.kint, sizeof(int) * (size_t)S);
        get((void **)&T.xs, sizeof(float) * (size_t)S);
        get((void **)&T.dinv, sizeof(float) * (size_t)S);
        get((void **)&P.perm, sizeof(int) * (size_t)S);
        get((void **)&P.cnt, sizeof(int) * (size_t)(h.n_int + 2));
        get((void **)&P.slot, sizeof(TSlot) * (size_t)S);
        get((void **)&P.Q, sizeof(double) * 4 * (size_t)S);
        get((void **)&P.QS, sizeof(double) * 4 * (size_t)S);
        get((void **)&P.LACC, sizeof(double) * 4 * (size_t)S);
        get((void **)&P.state, sizeof(int) * (size_t)S);
        get((void **)&P.kint, sizeof(int) * (size_t)S);
        get((void **)&P.hp, sizeof(float) * (size_t)S);
        get((void **)&P.dtf, sizeof(float) * (size_t)S);
        get((void **)&P.xs, sizeof(float) * (size_t)S);
        get((void **)&P.dinv, sizeof(float) * (size_t)S);
        get((void **)&P.inc, sizeof(unsigned long long) * (size_t)h.n_levels * S);
        get((void **)&P.PHa, sizeof(float2) * (size_t)h.n_levels * S);
        get((void **)&P.PHb, sizeof(float2) * (size_t)h.n_levels * S);
        get((void **)&P.A, sizeof(float2) * ns);
        get((void **)&P.ACC, sizeof(float2) * ns);
    }
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync (tensor-core path scratch)");
    }
    const size_t smem = kTcSmemFixed + sizeof(float) * 2 * kTcSlotsPerTile * (size_t)h.n_f;
    if (!plain &&
        (e = cudaFuncSetAttribute(k_tc_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    cudaMemsetAsync(T.live, 0, 4 * sizeof(int), st);
    const int slot_blocks = (S / 8 + 3) / 4;  // four warps of eight slots per block
    k_tc_init<<<slot_blocks, 128, 0, st>>>(T);
    const int n_ct = S / kTcSlotsPerTile;
    // the stage kernel: tcgen05 contraction (factorised BF16X3) or the sparse FP32 table (PLAIN)
    auto stage = [&](cudaStream_t q, int s, int cur) {
        if (plain) k_sp_stage<<<dim3(S / kSpTile, n_rowblocks), 32 * kSpWarps, 0, q>>>(T, s, cur);
        else k_tc_stage<<<h.n_tiles * n_ct, kTcThreads, smem, q>>>(T, s, cur);
    };
    // PLAIN path: the slots sorted by interval at the end of each chunk
    const int mv_blocks = (int)std::min<size_t>((ns + 255) / 256, (size_t)sms * 16);
    auto sort_slots = [&](cudaStream_t q) {
        if (!plain) return;
        k_sp_order<<<1, 32, 0, q>>>(T, P, h.n_int);
        k_sp_move_slots<<<(S + 127) / 128, 128, 0, q>>>(T, P, h.n_levels, 0);
        k_sp_move_rows<<<mv_blocks, 256, 0, q>>>(T, P, n, 0);
        k_sp_move_slots<<<(S + 127) / 128, 128, 0, q>>>(T, P, h.n_levels, 1);
        k_sp_move_rows<<<mv_blocks, 256, 0, q>>>(T, P, n, 1);
    };
    // chunks of steps inside a WHILE node: the body (one chunk) ends with k_tc_continue, which
    // sets the condition from the live-slot count; one launch of the graph runs every trajectory
    const int chunk = 4;
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphConditionalHandle cond;
    cudaGraphNode_t wnode;
    int live[4] = {0, 0, 0, 0};
    // MQCT_TC_HOST_LOOP=1: the same chunks launched directly from a host loop that reads the
    // live-slot count after each chunk (for profilers that do not follow conditional graph nodes)
    const char *hl = std::getenv("MQCT_TC_HOST_LOOP");
    const bool host_loop = hl && hl[0] == '1';
    for (long long it = 0; host_loop && e == cudaSuccess; ++it) {
        k_tc_reset_live<<<1, 32, 0, st>>>(T);
        for (int k = 0; k < chunk; ++k)
            for (int s = 0; s < 4; ++s) {
                const int cur = s & 1;
                stage(st, s, cur);
                k_tc_slots<<<slot_blocks, 128, 0, st>>>(T, s, n_rowblocks);
            }
        sort_slots(st);
        k_tc_continue<<<1, 32, 0, st>>>(T, 0);
        if ((e = cudaMemcpyAsync(live, T.live, 4 * sizeof(int), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (live[0] == 0 || live[1]) break;
    }
    if (!host_loop && e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (!host_loop && e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
    if (!host_loop && e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    if (!host_loop && e == cudaSuccess) {
        alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(npbuf);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (!host_loop && e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (!host_loop && e == cudaSuccess) {
        k_tc_reset_live<<<1, 32, 0, cap>>>(T);
        for (int k = 0; k < chunk; ++k)
            for (int s = 0; s < 4; ++s) {
                const int cur = s & 1;
                stage(cap, s, cur);
                k_tc_slots<<<slot_blocks, 128, 0, cap>>>(T, s, n_rowblocks);
            }
        sort_slots(cap);
        k_tc_continue<<<1, 32, 0, cap>>>(T, cond);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cap, &captured);
    }
    if (!host_loop && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (!host_loop && e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (!host_loop && e == cudaSuccess) e = cudaMemcpyAsync(live, T.live, 4 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!host_loop && e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core path");
    // k_tc_init, then per chunk: reset, chunk x 4 x (stage, slots), (PLAIN: the five sorting
    // kernels), continue
    count_launches(1 + (long long)live[2] * (2 + 8 * chunk + (plain ? 5 : 0)));
    if (live[1]) return fail(MQCT_ERR_TIMEOUT, "tensor-core path: a bounded MMA completion wait ran out");
    return MQCT_OK;
}

}  // namespace mqct
