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
//   k_tc_slots  one warp per slot, FP64: classical stage update (Eqs. 7-10), bookkeeping, stop
//               rule, refill, the spline values and phase factors of the next stage.
// The host runs chunks of steps as one CUDA graph and checks the number of live slots between
// chunks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace mqct {

namespace {

constexpr int kTcSlotsPerTile = 64;  // 128 real columns
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
    long long *t_start, *t_done;  // optional device clock (ns) at start / end of each trajectory
    int nmax, sys_idx;
    float2 *C[2];             // [n][S] stage amplitudes (phase rotated), double buffered
    float2 *A, *ACC;          // [n][S]
    float *coef;              // [2][L][S] v_l and v_l' at each slot's stage R
    float *vid;               // [2][S] identity-term sums of v and v'
    float *hp, *dtf;          // [S] dPhi/dt / 2 and dt (FP32 views)
    int *state;               // [S]
    float2 *PHa, *PHb;        // [n_levels][S]
    double *part;             // [n_tiles][S][6] per-row-tile partial sums
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

// the update of one element from w = M c and u = M' c (Eq. 5, RK4) and its gathered inputs;
// adds its force, torque and (stage 0) diagnostic contributions to part[6] (FP32: a thread sums
// a few rows; the sums across threads, row tiles and the classical update are FP64 -- the FP64
// pipe of this GPU is far too narrow for per-element FP64 arithmetic)
__device__ __forceinline__ void tc_elem_apply(const TcState &T, const DevSys &S, int s, int cur, int r, int sl,
                                              int st, const ElemIn &in, float2 w, float2 u, float *part)
{
    const int nxt = cur ^ 1;
    const size_t e = (size_t)r * T.S + sl;
    if (st == TS_WAIT && s == 3) {
        const float2 v = make_float2(r == T.slot[sl].s0 ? 1.0f : 0.0f, 0.0f);
        T.A[e] = v;
        T.ACC[e] = make_float2(0.f, 0.f);
        T.C[nxt][e] = v;
        return;
    }
    if (st != TS_ACTIVE && st != TS_FINAL) return;
    const float2 c = in.c, p = in.p, a0 = in.a0;
    const float2 dc = make_float2(in.ad * in.cd.x - in.au * in.cu.x, in.ad * in.cd.y - in.au * in.cu.y);
    const float2 da = make_float2(p.x * dc.x + p.y * dc.y, p.x * dc.y - p.y * dc.x);
    const float hp = T.hp[sl];
    float2 kk;
    kk.x = fmaf(hp, da.x, p.x * w.y - p.y * w.x);
    kk.y = fmaf(hp, da.y, -(p.x * w.x + p.y * w.y));
    part[0] -= c.x * u.x + c.y * u.y;
    part[1] -= dc.x * w.x + dc.y * w.y;
    if (s == 0) {
        const float pp = a0.x * a0.x + a0.y * a0.y;
        part[2] += c.x * w.x + c.y * w.y;
        part[3] += pp;
        part[4] += (float)S.lev_energy[in.lev] * pp;
        part[5] += a0.x * da.y - a0.y * da.x;
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
    float2 acc = in.acc;
    if (s == 0) {
        acc = make_float2(kk.x + acc.x, kk.y + acc.y);  // acc holds the last rounding error
    } else {
        const float wg = (s == 1 || s == 2) ? 2.0f : 1.0f;
        acc.x = fmaf(wg, kk.x, acc.x);
        acc.y = fmaf(wg, kk.y, acc.y);
    }
    const float2 q = in.q;
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
        T.C[nxt][e] = make_float2(q.x * sx - q.y * sy, q.x * sy + q.y * sx);
    } else {
        T.ACC[e] = acc;
        const float bn = s == 2 ? dtj : 0.5f * dtj;
        const float2 yn = make_float2(fmaf(bn, kk.x, a0.x), fmaf(bn, kk.y, a0.y));
        T.C[nxt][e] = make_float2(q.x * yn.x - q.y * yn.y, q.x * yn.y + q.y * yn.x);
    }
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
    double *red = reinterpret_cast<double *>(Ust + 128 * kTcWs);  // [8][64][6]
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
            for (int k = 0; k < 6; ++k) red[(g * kTcSlotsPerTile + j) * 6 + k] = (double)part[k];
        }
        __syncthreads();
        if (tid < kTcSlotsPerTile) {
            double acc6[6] = {0, 0, 0, 0, 0, 0};
            for (int g = 0; g < 8; ++g)
                for (int k = 0; k < 6; ++k) acc6[k] += red[(g * kTcSlotsPerTile + tid) * 6 + k];
            double *o = T.part + ((size_t)rt * T.S + s0 + tid) * 6;
            for (int k = 0; k < 6; ++k) o[k] = acc6[k];
        }
    } else if (tid == 0) {
        atomicOr(T.live + 1, 1);  // error flag: a bounded wait ran out
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == kTcMmaWarp) tc_tmem_dealloc(tbase, 256);
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

// spline values of the next stage, FP32 views, identity-term sums (one warp per slot; the
// slot record is final when the warp calls this)
__device__ void tc_publish(const TcState &T, const DevSys &S, int sl, int lane)
{
    const TSlot &m = T.slot[sl];
    const int state = m.state;
    if (lane == 0) T.state[sl] = state;
    if (state == TS_IDLE) {
        for (int l = lane; l < S.L; l += 32) T.coef[(size_t)l * T.S + sl] = T.coef[((size_t)S.L + l) * T.S + sl] = 0.f;
        if (lane == 0) {
            T.vid[sl] = T.vid[T.S + sl] = 0.f;
            T.hp[sl] = 0.f;
            T.dtf[sl] = 1.f;
        }
        return;
    }
    float v0 = 0.f, d0 = 0.f;
    const float x = (float)m.x;
    const int kint = m.kint;
    for (int l = lane; l < S.L; l += 32) {
        const float4 c = S.vcoef_f[(size_t)l * S.n_int + kint];
        const float v = fmaf(x, fmaf(x, fmaf(x, c.w, c.z), c.y), c.x);
        const float dv = fmaf(x, fmaf(3.0f * x, c.w, 2.0f * c.z), c.y);
        T.coef[(size_t)l * T.S + sl] = v;
        T.coef[((size_t)S.L + l) * T.S + sl] = dv;
        if ((S.id_mask >> l) & 1ull) { v0 += v; d0 += dv; }
    }
    for (int o = 16; o; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
    }
    if (lane == 0) {
        T.vid[sl] = v0;
        T.vid[T.S + sl] = d0;
        T.hp[sl] = (float)(0.5 * m.phidot);
        T.dtf[sl] = (float)m.dt;
    }
}

// phase factors exp(-i E_l t) of every level for one slot (one warp): kind 1 -> PHa at t,
// kind 2 -> PHb at t, kind 3 -> start of a trajectory: PHa = 1, PHb at t = dt/2
__device__ void tc_phases(const TcState &T, const DevSys &S, int sl, int lane, int kind, double t)
{
    for (int l = lane; l < S.n_levels; l += 32) {
        const float2 ph = tc_phase(S.lev_energy[l], t);
        if (kind == 1) T.PHa[(size_t)l * T.S + sl] = ph;
        else {
            T.PHb[(size_t)l * T.S + sl] = ph;
            if (kind == 3) T.PHa[(size_t)l * T.S + sl] = make_float2(1.f, 0.f);
        }
    }
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
        const bool ok = tr.system_idx == T.sys_idx && tr.dt > 0.0 && tr.e_coll > 0.0 && tr.b >= 0.0 && tr.r0 > 0.0 &&
                        tr.b < tr.r0 && isfinite(tr.r_end) && tr.max_steps >= 0 && tr.init_state >= 0 &&
                        tr.init_state < S.n;
        if (!ok) {
            if (T.diag) {
                mqct_diag d = {0, MQCT_TRAJ_INVALID, 0.0, 0.0, 0.0, 0.0};
                T.diag[t] = d;
            }
            continue;
        }
        if (T.t_start) T.t_start[t] = mqct_clock_ns();
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

// one warp per slot: claim the first trajectory and initialise its column
__global__ void __launch_bounds__(128) k_tc_init(TcState T)
{
    const DevSys &S = *T.sys;
    const int lane = threadIdx.x & 31, sl = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (sl >= T.S) return;
    TSlot &m = T.slot[sl];
    if (lane == 0) tc_claim(T, S, sl);
    __syncwarp();
    if (m.state == TS_WAIT) {
        for (int r = lane; r < S.n; r += 32) {
            const float2 v = make_float2(r == m.s0 ? 1.0f : 0.0f, 0.0f);
            const size_t e = (size_t)r * T.S + sl;
            T.A[e] = v; T.ACC[e] = make_float2(0.f, 0.f); T.C[0][e] = v;
        }
        __syncwarp();
        if (lane == 0) {
            m.state = m.max_steps > 0 ? TS_ACTIVE : TS_FINAL;
            if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
            tc_locate(S, m);
        }
        __syncwarp();
        tc_phases(T, S, sl, lane, 3, 0.5 * m.dt);
    }
    __syncwarp();
    tc_publish(T, S, sl, lane);
}

// one warp per slot: sum the row-block partials of force, torque and diagnostics, then (lane 0,
// FP64) the classical stage update (Eqs. 7-10), bookkeeping, stop rule and refill; the lanes
// share the phase factors and spline values of the next stage
__global__ void __launch_bounds__(128) k_tc_slots(TcState T, int s, int n_rowblocks)
{
    const DevSys &S = *T.sys;
    const int lane = threadIdx.x & 31, sl = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (sl >= T.S) return;
    TSlot &m = T.slot[sl];
    if (m.state == TS_IDLE) return;  // published as idle when it became idle
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = lane; b < n_rowblocks; b += 32) {
        const double *p = T.part + ((size_t)b * T.S + sl) * 6;
        for (int q = 0; q < 6; ++q) acc[q] += p[q];
    }
    for (int o = 16; o; o >>= 1)
        for (int q = 0; q < 6; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    int kind = 0;
    double tph = 0.0;
    if (lane == 0) {
        const double F = acc[0], Tq = acc[1], V = acc[2], NR = acc[3], ER = acc[4], JY = acc[5];
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
                    if (T.t_done) T.t_done[m.traj] = mqct_clock_ns();
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
                if (s == 1) { kind = 1; tph = m.steps * m.dt + m.dt; }
                if (s == 3 && m.state == TS_ACTIVE) { kind = 2; tph = m.steps * m.dt + 0.5 * m.dt; }
            }
        } else if (m.state == TS_WAIT && s == 3) {
            m.state = m.max_steps > 0 ? TS_ACTIVE : TS_FINAL;
            if (m.max_steps <= 0) m.status |= MQCT_TRAJ_MAX_STEPS;
            tc_locate(S, m);
            kind = 3;
            tph = 0.5 * m.dt;
        }
    }
    __syncwarp();
    kind = __shfl_sync(0xffffffffu, kind, 0);
    tph = __shfl_sync(0xffffffffu, tph, 0);
    if (kind) tc_phases(T, S, sl, lane, kind, tph);
    __syncwarp();
    tc_publish(T, S, sl, lane);
    if (lane == 0 && s == 3 && m.state != TS_IDLE) atomicAdd(T.live, 1);
}

}  // namespace

mqct_status run_tc_batched(const BatchArgs &a, const DevSys &h, cudaStream_t st)
{
    const int n = h.n;
    // slot count: the contraction runs one CTA per SM per (row tile, 64-slot tile), so the slots
    // fill whole waves -- one wave when the trajectories fit in it, else two (more slots only
    // lengthen the tail of uneven trajectories); a.tc_slots overrides (rounded up to 64)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt = std::max(1, h.n_tiles);
    const int one_wave = std::max(1, sms / nt), two_waves = std::max(1, 2 * sms / nt);
    const int want = (a.n + kTcSlotsPerTile - 1) / kTcSlotsPerTile;
    int n_slot_tiles = want <= one_wave ? want : std::min(want, two_waves);
    if (a.tc_slots > 0) n_slot_tiles = (a.tc_slots + kTcSlotsPerTile - 1) / kTcSlotsPerTile;
    n_slot_tiles = std::max(1, std::min(n_slot_tiles, 8192 / kTcSlotsPerTile));
    const int S = n_slot_tiles * kTcSlotsPerTile;
    const int n_rowblocks = std::max(1, h.n_tiles);
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
    const size_t ns = (size_t)n * S;
    get((void **)&T.live, 2 * sizeof(int));
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
    get((void **)&T.part, sizeof(double) * 6 * (size_t)n_rowblocks * S);
    get((void **)&T.slot, sizeof(TSlot) * (size_t)S);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMallocAsync (tensor-core path scratch)");
    }
    const size_t smem = kTcSmemFixed + sizeof(float) * 2 * kTcSlotsPerTile * (size_t)h.n_f;
    if ((e = cudaFuncSetAttribute(k_tc_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    cudaMemsetAsync(T.live, 0, 2 * sizeof(int), st);
    k_tc_init<<<(S + 3) / 4, 128, 0, st>>>(T);
    const int n_ct = S / kTcSlotsPerTile;
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
                k_tc_stage<<<h.n_tiles * n_ct, kTcThreads, smem, cap>>>(T, s, cur);
                k_tc_slots<<<(S + 3) / 4, 128, 0, cap>>>(T, s, n_rowblocks);
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
