#!/usr/bin/env python
"""MQCT trajectory-steps/s on one GB300 (and N GPUs as independent replicas).

Default workload: the N = 441 atom + diatom system (j <= 20), E in {100, 300, 1000, 3000}
cm^-1, j' in {0, 1, 2}, 256 midpoint impact parameters on 0-15 bohr per (E, j'): 3072
trajectories, 400-point spline grid, RK4 dt = 5 a.u.  One step = propagate every trajectory to
its end (Eqs. 4-10) plus the cross-section reduction (Sec. II), inputs resident in HBM.
Other workloads: --workload n1600 (N = 1600 diatom), asym1580 (N = 1580 asymmetric top),
mix (uneven four-basis batch in one call).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload n441|n1600|asym1580|mix] [--path plain|factorised]
                  [--precision fp64|fp32|bf16x3] [--no-autotune] [--max-traj M]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_02322_gb300 import inputs as W  # noqa: E402

METRIC = "MQCT trajectory-steps/s at N=441/1600, batched mixed vs plain FP64, same error"
WORKLOAD = "diatom j<=20 (N=441), 3072 trajectories: E in {100,300,1000,3000} cm^-1 x j' in {0,1,2} x 256 b on 0-15 bohr"
WORKLOAD_1600 = "diatom j<=39 (N=1600), 768 trajectories: E in {1000,3000} cm^-1 x j' in {0,1,2} x 128 b on 0-15 bohr"
WORKLOAD_MIX = ("uneven batch: diatom bases N = 49, 121, 441, 1600 (j <= 6, 10, 20, 39) in a seeded 1:2:4:1 mix, "
                "b ~ U(0,20), E log-uniform 10-5000 cm^-1, one propagation call")
WORKLOAD_ASYM = ("asymmetric top A,B,C = 27.88,14.51,9.28 cm^-1, J<=12 truncated to N=1580 (110 levels), 28 terms "
                 "lam<=6, 8 E log-spaced 10-2000 cm^-1, b ~ U(0,15), initial level J=0")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--path", default="factorised", choices=["plain", "factorised"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16x3"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain-FP64 comparison run (throughput and max |dP| against it)")
    ap.add_argument("--adjoint", type=int, default=1024,
                    help="time the FP64 and the mixed adjoint on this many trajectories of the gradient workload "
                         "(N = 441, E = 1000 cm^-1; 1024 = all of it; 0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-traj", type=int, default=0,
                    help="run a seeded subset of this many trajectories (profiling of a small case)")
    ap.add_argument("--max-steps", type=int, default=0,
                    help="cap every trajectory at this many RK4 steps (profiling a small case; not a bench line)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the library's automatic launch shapes instead of timing the candidates on a "
                         "probe sample first (outside the timed region) and using the fastest")
    ap.add_argument("--workload", default="n441", choices=["n441", "n1600", "asym1580", "mix"],
                    help="n441: the 3072-trajectory N = 441 workload; n1600: 768 trajectories with N = 1600; "
                         "asym1580: the N = 1580 asymmetric-top workload (a seeded subset, --max-traj, default 1024); "
                         "mix: the uneven four-basis batch (first --max-traj of its 50000 trajectories, default 4096)")
    ap.add_argument("--batch-shape", type=int, default=0,
                    help="FP32 batched kernel shape 1..7 for every system (see mqct_propagate_opts); implies "
                         "--no-autotune")
    ap.add_argument("--no-molmol", dest="molmol", action="store_false",
                    help="skip the asymmetric top + linear rotor timing")
    ap.add_argument("--sparse-jmax", type=int, default=200,
                    help="rotor jmax of the sparse paper-scale block (N = (jmax+1)^2)")
    ap.add_argument("--sparse-traj", type=int, default=1024, help="trajectories of the sparse block")
    ap.add_argument("--sparse-steps", type=int, default=2000, help="RK4 steps per trajectory of the sparse block")
    ap.add_argument("--no-sparse", dest="sparse", action="store_false",
                    help="skip the paper-scale sparse-path (log grid, truncation, N = 40401) timing")
    ap.add_argument("--no-rates", dest="rates", action="store_false",
                    help="skip the post-processing (Eq. 20 and rate coefficients) timing")
    ap.add_argument("--no-n1600", dest="n1600", action="store_false",
                    help="skip the N = 1600 block (the metric's second basis size, timed after the headline)")
    ap.add_argument("--energy", type=float, default=0.0,
                    help="keep only the trajectories at this collision energy (cm^-1)")
    return ap.parse_args()


def max_over_ranks(x: float, dist, device=None) -> float:
    """The largest value of x over all ranks (the whole job's time is its slowest rank's);
    x itself when there is one rank."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------- CPU oracle
def strat_idx(ts, n_sample, seed):
    """Seeded indices of n_sample trajectories stratified over the collision energies (the step
    count per trajectory depends mostly on E)."""
    rng = np.random.default_rng(seed)
    es = np.unique(ts.e_coll)
    per = max(1, n_sample // len(es))
    return np.sort(np.concatenate([rng.choice(np.flatnonzero(ts.e_coll == e), min(per, int(np.sum(ts.e_coll == e))),
                                              replace=False) for e in es]))


def oracle_sample(p, ts, n_sample, seed=11):
    """Bounded, seeded sample of the workload (see strat_idx)."""
    return ts.subset(strat_idx(ts, n_sample, seed))


def make_system(api, p, path, precision):
    if isinstance(p, W.AsymTopParams):
        return api.System.asym_top(p, path=path, precision=precision)
    return api.System.diatom(p, path=path, precision=precision)


def run_oracle(p, sub, threads):
    import oracle

    oracle.build()
    if isinstance(p, W.AsymTopParams):
        osys = oracle.asym_system(p)
        lab = {(int(l), int(m)): i for i, (l, m) in enumerate(zip(osys.level, osys.mq))}
        init = [lab[(int(l), int(m))] for l, m in zip(sub.init_j, sub.init_m)]
    else:
        osys = oracle.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
        init = [j * j + j + m for j, m in zip(sub.init_j, sub.init_m)]
    t0 = time.perf_counter()
    amp, res = oracle.propagate(osys, sub.e_coll, sub.b, init, r0=sub.r0, r_end=sub.r_end, dt=sub.dt,
                                max_steps=sub.max_steps, n_threads=threads)
    t1 = time.perf_counter()
    return float(res["steps"].sum()), t1 - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------- reference arm
def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    p, ts = W.workload2()
    sub = oracle_sample(p, ts, 16)
    cores = cpu_cores()
    for _ in range(args.warmup):
        run_oracle(p, oracle_sample(p, ts, 4, seed=99), cores)
    steps_tot, t_tot = 0.0, 0.0
    for _ in range(args.steps):
        s, t = run_oracle(p, sub, cores)
        steps_tot += s
        t_tot += t
    v = steps_tot / t_tot
    sample = f"{sub.n} trajectories of the workload (4 per collision energy, seeded) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "traj-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "traj-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "traj-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------- roofline
KERNEL_SRC = {"k_propagate_fp64": "propagate.cu", "k_batched_f32": "batched.cu", "k_tc_stage": "tc_batched.cu"}


def profile_traffic(kernel):
    """DRAM bytes per trajectory-stage of `kernel` from its committed ncu summary
    (profiles/<kernel>_*.md lines "dram_bytes_per_traj_stage:" and "source_sha256:"), or None
    when there is none or the kernel's source has changed since the counters were taken."""
    import glob
    import hashlib

    src = os.path.join(ROOT, "paper_2312_02322_gb300", "csrc", KERNEL_SRC[kernel])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_*.md"))):
        kv = {}
        for line in open(f):
            if ":" in line and line.split(":", 1)[0].strip() in ("dram_bytes_per_traj_stage", "source_sha256"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha256") == sha and "dram_bytes_per_traj_stage" in kv:
            return float(kv["dram_bytes_per_traj_stage"]), os.path.relpath(f, ROOT)
    return None, None


def roofline_of(api, path, precision, infos, steps, sidx, k_ms):
    """Roofline object of the dominant kernel of one propagate call (its time k_ms).

    Units: trajectory-stages (4 per RK4 step, plus the final evaluation of each trajectory).
    Useful work per trajectory-stage: the coupling contraction, 4 flops per stored non-zero of
    the coupling (factorised: sum over terms of nnz(G^l); plain: 4 spline coefficients x nnz(M));
    the per-state work (phases, Coriolis stencil, RK4 update, reductions) is reported beside it,
    not counted."""
    useful = per_state = exec_tc = stages_tot = table_bytes = 0.0
    for i, inf in enumerate(infos):
        rows = sidx == i
        stages = 4.0 * float(steps[rows].sum()) + float(rows.sum())
        n = inf["n_states"]
        if path == "plain":
            useful += 16.0 * inf["table_nnz"] * stages
            per_state += 40.0 * n * stages
            table_bytes += 32.0 * inf["table_nnz"] * (1.0 if precision == "fp64" else 0.5) * stages
        else:
            useful += 4.0 * inf["glambda_nnz"] * stages
            per_state += (8.0 * inf["n_terms"] + 40.0) * n * stages
        exec_tc += inf["tc_kchunks"] * 3 * (2.0 * 128 * 128 * 16) / 64.0 * stages
        stages_tot += stages
    kernel = {"fp64": "k_propagate_fp64", "fp32": "k_batched_f32", "bf16x3": "k_tc_stage"}[precision]
    per_stage_traffic, prof = profile_traffic(kernel)
    traffic = None if per_stage_traffic is None else per_stage_traffic * stages_tot
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    if precision == "bf16x3":
        # executed tensor work: per stage, per 64-slot tile, for every stored term and row tile its
        # non-zero 16-column K chunks x 3 split products of a 128 x 128 x 16 MMA; time = the whole
        # propagate call (stage and slot kernels): a lower bound
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        ach = exec_tc / (k_ms * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                "traffic": traffic, "kernel": "k_tc_stage (timed with the whole propagate call)",
                "peak_source": "of measured bf16 burst (MEASURED_PEAKS.json)",
                "executed_flops_per_traj_stage": exec_tc / stages_tot,
                "useful_flops_per_traj_stage": useful / stages_tot, "useful_over_executed": useful / exec_tc,
                "traj_stages_per_launch": stages_tot, "kernel_ms": k_ms, "traffic_source": prof}
    fp_peak = api.fma_rate("fp64") if precision == "fp64" else api.fma_rate("fp32")
    achieved = useful / (k_ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": fp_peak / 1e3, "unit": "TFLOP/s",
           "frac": achieved * 1e3 / fp_peak, "traffic": traffic, "kernel": kernel,
           "peak_source": f"of measured {precision.upper()} FMA rate (library probe mqct_probe_fma_rate)",
           "useful_flops_per_traj_stage": useful / stages_tot,
           "per_state_flops_per_traj_stage": per_state / stages_tot,
           "frac_with_per_state_work": (useful + per_state) / (k_ms * 1e-3) / fp_peak / 1e9,
           "traj_stages_per_launch": stages_tot, "kernel_ms": k_ms, "traffic_source": prof}
    hbm = peaks.get("hbm_gbs")
    if table_bytes and hbm:
        gbs = table_bytes / (k_ms * 1e-3) / 1e9
        out["hbm_view"] = {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                           "note": "algorithmic table bytes; the table is L2-resident, so DRAM traffic is lower"}
    return out


def compare_fp64(api, ps, tr, cidx, steps_m, pop_m, sidx, infos, dev, stream, flush, value, ws, runs=3):
    """The trajectories cidx of a measured batch through the plain FP64 path: its throughput
    (median of `runs` timed runs, L2 flushed before each) and the largest population difference of
    the measured path against it ("same error")."""
    import torch

    s64 = [make_system(api, q, "plain", "fp64") for q in ps]
    trc = torch.from_numpy(tr[cidx].view(np.uint8).copy()).to(dev)
    pop64, _, d64 = api.propagate(s64, trc, device=True, stream=stream)  # also the warm-up
    torch.cuda.synchronize()
    d64 = api.diag_to_numpy(d64)
    ms_runs = []
    for _ in range(runs):
        flush.zero_()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        api.propagate(s64, trc, want_pop=False, want_diag=False, device=True, stream=stream)
        b_.record(stream)
        torch.cuda.synchronize()
        ms_runs.append(a_.elapsed_time(b_))
    ms64 = float(np.median(ms_runs))
    same = d64["steps"] == steps_m[cidx]
    # only the first N_t entries of a row belong to its system (the rest are not written)
    width = np.array([infos[k]["n_states"] for k in sidx[cidx]])
    valid = np.arange(pop_m.shape[1])[None, :] < width[:, None]
    dp = np.where(valid, np.abs(pop_m - pop64.cpu().numpy()[:, :pop_m.shape[1]]), 0.0)
    v64 = float(d64["steps"].sum()) * ws / (ms64 * 1e-3)
    return {"path": "plain", "precision": "fp64", "value": v64, "unit": "traj-steps/s", "ms": ms64,
            "ms_runs": ms_runs, "timed_runs": runs, "trajectories": int(len(cidx)),
            "max_abs_dP_vs_fp64": float(dp.max()), "max_abs_dP_same_steps": float(dp[same].max()),
            "trajectories_same_steps": int(same.sum()), "speedup": value / v64}


def n1600_block(api, args, dev, stream, flush, ws, runs=3):
    """The N = 1600 workload (768 trajectories) through the measured precision and, beside it,
    the plain FP64 path: traj-steps/s of each (median of `runs` timed runs, L2 flushed before
    each), max |dP| between them, sigma-sets/s."""
    import torch

    p, ts = W.workload2_n1600()
    sys_ = make_system(api, p, args.path, args.precision)
    info = sys_.info
    tr = api.make_trajs(ts, sys_)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).to(dev)
    tune = {}
    if args.autotune and args.precision != "fp64":
        from paper_2312_02322_gb300 import autotune

        t_ = autotune.tune_batch([sys_], tr)
        tune = {"batch_shape": t_["batch_shape"], "tc_slots": t_["tc_slots"]}
    pop, _, diag = api.propagate(sys_, trd, device=True, stream=stream, **tune)
    torch.cuda.synchronize()
    dg = api.diag_to_numpy(diag)
    w = torch.from_numpy(api.sigma_weights(ts, dg["status"])).to(dev)
    g = torch.from_numpy(ts.group.astype(np.int32)).to(dev)
    ms_runs = []
    for _ in range(runs):
        flush.zero_()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        pp, _, _ = api.propagate(sys_, trd, want_diag=False, device=True, stream=stream, **tune)
        api.cross_sections(sys_, pp, w, g, ts.n_groups, stream=stream)
        b_.record(stream)
        torch.cuda.synchronize()
        ms_runs.append(a_.elapsed_time(b_))
    ms = float(np.median(ms_runs))
    steps = float(dg["steps"].sum())
    value = steps * ws / (ms * 1e-3)
    sidx = np.zeros(ts.n, int)
    comp = compare_fp64(api, [p], tr, np.arange(ts.n), dg["steps"], pop.cpu().numpy(), sidx, [info], dev, stream,
                        flush, value, ws, runs=runs)
    return {"workload": WORKLOAD_1600, "path": args.path, "precision": args.precision, "value": value,
            "unit": "traj-steps/s", "ms_per_step": ms, "ms_runs": ms_runs, "timed_runs": runs,
            "traj_steps_per_step": steps, "sigma_sets_per_s": ts.n_groups * ws / (ms * 1e-3),
            "launch_option": tune, "comparison": comp}


def adjoint_block(api, n_traj):
    """The gradient workload (N = 441, E = 1000 cm^-1, checkpoints every 64 steps): gradients of every
    j = 0 -> j' cross section, combined with seeded random weights, with respect to the 10 PES parameters,
    by the FP64 adjoint and the mixed (FP32-amplitude) adjoint; each timed once after a short
    warm-up call."""
    import torch

    pa, ta = W.workload5()
    if n_traj < ta.n:
        ta = ta.subset(np.linspace(0, ta.n - 1, n_traj).astype(int))
    s64 = api.System.diatom(pa, path="factorised", precision="fp64", with_params=True)
    tra = api.make_trajs(ta, s64)
    _, _, dga = api.propagate(s64, tra, device=False)
    wa = api.sigma_weights(ta, dga["status"])
    # seeded random upstream weights: unit weights would ask for the gradient of the total
    # probability, which unitarity makes zero
    dls = np.random.default_rng(W.DEFAULT_SEED).standard_normal((ta.n_groups, s64.n_levels))
    steps = float(dga["steps"].sum())
    out = {"workload": f"{ta.n} of the 1024 trajectories of the N=441, E=1000 cm^-1 gradient workload",
           "params": int(s64.n_params), "ckpt": 64, "traj_steps": steps}
    grads = {}
    for prec in ("fp64", "fp32"):
        sa = s64 if prec == "fp64" else api.System.diatom(pa, path="factorised", precision=prec, with_params=True)
        few = np.arange(min(4, ta.n))
        api.adjoint(sa, tra[few], wa[few], ta.group[few], ta.n_groups, dls, ckpt=64)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = api.adjoint(sa, tra, wa, ta.group, ta.n_groups, dls, ckpt=64)
        sec = time.perf_counter() - t0
        grads[prec] = g
        out[prec] = {"seconds": sec, "traj_steps_per_s": steps / sec, "gradients_per_s": 1.0 / sec,
                     "dL_dtheta_norm": float(np.linalg.norm(g))}
    out["mixed_vs_fp64_max_rel"] = float(np.max(np.abs(grads["fp32"] - grads["fp64"])) / np.max(np.abs(grads["fp64"])))
    return out


def rates_block(api, n_levels=1032, reps=5):
    """Post-processing at the paper's scale: Eq. 20 and the Maxwell-Boltzmann rates of both directions
    of every pair of 1032 levels (the paper's count of non-degenerate channels) on its ten collision
    energies, at five temperatures; cross sections resident on the device, timed with CUDA events."""
    import torch

    rs = W.rate_set(n_levels=n_levels)
    sig = torch.from_numpy(rs.sigma).cuda()
    api.rate_coefficients(sig, rs.u, rs.energy, rs.g, rs.mu, rs.kT)  # warm-up
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    for _ in range(reps):
        api.rate_coefficients(sig, rs.u, rs.energy, rs.g, rs.mu, rs.kT, stream=stream.cuda_stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    L, T = n_levels, len(rs.kT)
    n_rates = L * L * T
    return {"workload": f"{L} levels x {len(rs.u)} energies x {T} temperatures (synthetic cross sections)",
            "ms": ms, "rate_coefficients_per_s": n_rates / (ms * 1e-3), "transitions": L * (L - 1) // 2}


def sparse_block(api, n_traj=1024, max_steps=2000, jmax=200):
    """The paper-scale setup of Sec. III on an atom + rotor (FP32 spline table, stage-synchronous
    sparse kernel): N = (jmax+1)^2 states (jmax 200: 40 401; jmax 446: 199 809, the paper's ~2e5),
    Legendre terms lambda <= 12, the 63-point log grid on
    3-30 bohr, |M| > 1 cm^-1 at 6.03 / 7.11 bohr; n_traj seeded trajectories from 30 bohr (E log-uniform
    on 100-5000 cm^-1, b uniform on 0-10 bohr, initial j uniform on 0-10), each capped at max_steps
    RK4 steps; one warm-up call, then one timed call with the trajectories resident on the device."""
    import torch

    t0 = time.perf_counter()
    p = W.sparse_pes_params(jmax=jmax, lam_max=12)
    trunc = (float(W.cm(W.PAPER_TRUNC_CM)), *W.PAPER_TRUNC_R)
    sys_ = api.System.diatom(p, path="plain", precision="fp32", grid="log", trunc=trunc)
    build_s = time.perf_counter() - t0
    inf = sys_.info
    rng = np.random.default_rng(W.DEFAULT_SEED)
    e = W.cm(np.exp(rng.uniform(np.log(100.0), np.log(5000.0), n_traj)))
    b = rng.uniform(0.0, 10.0, n_traj)
    j = rng.integers(0, 11, n_traj).astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros(n_traj, np.int32), 1, r0=30.0, r_end=30.0, dt=5.0,
                   max_steps=max_steps, sampling="mc", b_max=10.0, n_b=0)
    tr = api.make_trajs(ts, sys_)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    few = torch.from_numpy(tr[:64].copy().view(np.uint8)).cuda()
    api.propagate(sys_, few, want_pop=False, device=True)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    pop, _, dg = api.propagate(sys_, trd, want_pop=True, device=True, stream=stream.cuda_stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    launches = api.last_launch_count()
    ms = ev[0].elapsed_time(ev[1])
    d = api.diag_to_numpy(dg)
    steps = float(d["steps"].sum())
    stages = 4.0 * steps
    # algorithmic bytes per trajectory-stage: the amplitudes streamed once (C read, A and ACC read and
    # written, the next stage's C written: 6 x 8 B per state) plus one interval's FP32 table slab
    # shared by the slots in that interval (counted once per stage launch: a lower bound)
    amp_b = 6 * 8 * inf["n_states"]
    table_b = inf["table_bytes"] / (p.n_grid - 1)
    n_launch_stage = 4.0 * float(d["steps"].max() + 1)
    algo = amp_b * stages + table_b * n_launch_stage
    gbs = algo / (ms * 1e-3) / 1e9
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return {"workload": f"{n_traj} trajectories, N = {inf['n_states']} (jmax {jmax}, lambda <= 12), log grid 3-30 bohr "
                        f"x {p.n_grid}, |M| > 1 cm^-1 at 6.03/7.11 bohr, each capped at {max_steps} steps",
            "table_nnz": int(inf["table_nnz"]), "trunc_dropped": int(inf["trunc_dropped"]),
            "table_bytes": int(inf["table_bytes"]), "build_s": build_s, "ms": ms,
            "traj_steps": steps, "traj_steps_per_s": steps / (ms * 1e-3), "gpu_launches": launches,
            "max_norm_dev": float(np.max(d["norm_dev"])),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes_per_traj_stage": amp_b, "table_slab_bytes": table_b,
                         "kernel": "k_sp_stage (timed with the whole propagate call)"}}


def molmol_block(api, n_traj=1024):
    """The molecule-molecule system of Sec. II (composite states of Eq. 3, coupling of Eqs. 13-17): a
    water-like asymmetric top (j1 <= 2) + para-H2 (j2 in {0, 2}), N = 210 states, nine PES terms;
    n_traj seeded trajectories (E log-uniform on 100-3000 cm^-1, b uniform on 0-10 bohr, from the ground
    level), FP32 batched kernel and FP64 kernel, each timed once after a warm-up call."""
    import torch

    p = W.molmol_params(j1max=2, j2=(0, 2))
    rng = np.random.default_rng(W.DEFAULT_SEED + 4)
    out = {"workload": f"{n_traj} trajectories, asymmetric top (j1 <= 2) + linear rotor (j2 in 0, 2), N = 210, "
                       f"{p.n_terms} terms"}
    pops = {}
    for prec, path in (("fp32", "factorised"), ("fp64", "factorised")):
        sys_ = api.System.molmol(p, path=path, precision=prec)
        tr = np.zeros(n_traj, api.TRAJ_DTYPE)
        tr["e_coll"] = W.cm(np.exp(rng.uniform(np.log(100.0), np.log(3000.0), n_traj))) if prec == "fp32" else tr0["e_coll"]
        tr["b"] = rng.uniform(0.0, 10.0, n_traj) if prec == "fp32" else tr0["b"]
        tr["r0"], tr["r_end"], tr["dt"], tr["max_steps"] = 30.0, 30.0, 5.0, 1_000_000
        if prec == "fp32":
            tr0 = tr.copy()
        trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
        api.propagate(sys_, trd[:64 * api.TRAJ_DTYPE.itemsize], want_pop=False, device=True)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop, _, dg = api.propagate(sys_, trd, device=True)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        d = api.diag_to_numpy(dg)
        pops[prec] = (pop.cpu().numpy(), d["steps"])
        out[prec] = {"traj_steps_per_s": float(d["steps"].sum()) / sec, "seconds": sec}
    same = pops["fp32"][1] == pops["fp64"][1]
    out["same_steps"] = f"{int(same.sum())}/{n_traj}"
    out["max_abs_dP_fp32_vs_fp64"] = (float(np.max(np.abs(pops["fp32"][0][same] - pops["fp64"][0][same])))
                                      if same.any() else None)
    out["speedup"] = out["fp32"]["traj_steps_per_s"] / out["fp64"]["traj_steps_per_s"]
    return out


# ---------------------------------------------------------------------------- GPU arm
def gpu_arm(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2312_02322_gb300 import api, build

    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # ---- workload: one system, or the uneven mix of four bases in one call
    if args.workload == "mix":
        ps, ts = W.workload4()
        workload = WORKLOAD_MIX
        if not args.max_traj:
            args.max_traj = 4096
    elif args.workload == "asym1580":
        p, ts = W.workload3()
        ps = [p]
        workload = WORKLOAD_ASYM
        if not args.max_traj:
            args.max_traj = 1024
    else:
        p, ts = W.workload2() if args.workload == "n441" else W.workload2_n1600()
        ps = [p]
        workload = WORKLOAD if args.workload == "n441" else WORKLOAD_1600
    if args.energy:
        ts = ts.subset(np.flatnonzero(np.isclose(ts.e_coll, float(W.cm(args.energy)))))
        workload = f"E = {args.energy} cm^-1 part of: {workload}"
    if args.max_traj and args.max_traj < ts.n:
        if args.workload == "mix":
            ts = ts.subset(np.arange(args.max_traj))  # the mix is already a seeded random draw
        else:
            ts = oracle_sample(ps[0], ts, args.max_traj, seed=5)
        workload = f"seeded subset of {ts.n} trajectories of: {workload}"
    if args.max_steps:
        ts.max_steps = args.max_steps
        workload = f"every trajectory capped at {args.max_steps} steps (profiling case) of: {workload}"
    systems = [make_system(api, q, args.path, args.precision) for q in ps]
    infos = [s_.info for s_ in systems]
    tr = api.make_trajs(ts, systems)
    sidx = tr["system_idx"].astype(int)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).to(dev)
    tune = {}
    if args.batch_shape:
        tune = {"batch_shape": args.batch_shape}
        tune_report = None
    elif args.autotune and args.precision != "fp64":
        from paper_2312_02322_gb300 import autotune

        t_ = autotune.tune_batch(systems, tr)
        tune = {"batch_shape": t_["batch_shape"], "tc_slots": t_["tc_slots"]}
        tune_report = [None if r is None else {"option": r["option"], "rate": r["rate"],
                                               "table": [(x["option"], round(x["rate"])) for x in r["table"]]}
                       for r in t_["reports"]]
    # per-system cross-section groups (rows of one system, its own basis width)
    groups = []
    for i, s_ in enumerate(systems):
        rows = np.flatnonzero(sidx == i)
        if len(rows) == 0:
            continue
        sub = ts.subset(rows)
        if args.workload == "mix":
            sub.group = np.zeros(len(rows), np.int32)
            sub.n_groups = 1
        groups.append((i, rows, sub))

    # the first warm-up pass also returns the step counts and statuses (every pass does the
    # same deterministic work), which fix the cross-section weights; and the completion times
    t_start = torch.zeros(ts.n, dtype=torch.int64, device=dev)
    t_done = torch.zeros(ts.n, dtype=torch.int64, device=dev)
    pop, _, diag = api.propagate(systems, trd, device=True, stream=stream, timing=(t_start, t_done), **tune)
    torch.cuda.synchronize()
    dg = api.diag_to_numpy(diag)
    traj_steps = float(dg["steps"].sum())
    n_bad = int(np.count_nonzero(dg["status"] & (api.TRAJ_MAX_STEPS | api.TRAJ_NONFINITE)))
    ts_np, td_np = t_start.cpu().numpy(), t_done.cpu().numpy()
    done_ms = (td_np - ts_np.min()) * 1e-6
    run_ms = (td_np - ts_np) * 1e-6
    latency = {"p50_ms": float(np.percentile(done_ms, 50)), "p99_ms": float(np.percentile(done_ms, 99)),
               "max_ms": float(done_ms.max()), "run_p50_ms": float(np.percentile(run_ms, 50)),
               "run_p99_ms": float(np.percentile(run_ms, 99)),
               "note": "completion time of each trajectory since the first one started (one batch submitted "
                       "at once), and each trajectory's own start-to-finish time; GPU global timer"}
    sig_args = []
    for i, rows, sub in groups:
        w = api.sigma_weights(sub, dg["status"][rows])
        sig_args.append((systems[i], torch.from_numpy(rows).to(dev), infos[i]["n_states"], torch.from_numpy(w).to(dev),
                         torch.from_numpy(sub.group.astype(np.int32)).to(dev), sub.n_groups))
    one_sys = len(systems) == 1 and len(groups) == 1 and len(groups[0][1]) == ts.n

    n_launch = [0]

    def sigma(pop_):
        for s_, rows_d, nn, w_d, g_d, ng in sig_args:
            pp = pop_ if one_sys else pop_.index_select(0, rows_d)[:, :nn].contiguous()
            api.cross_sections(s_, pp, w_d, g_d, ng, stream=stream)
            n_launch[0] += api.last_launch_count()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    for _ in range(max(0, args.warmup - 1)):
        pop, _, _ = api.propagate(systems, trd, want_diag=False, device=True, stream=stream, **tune)
        sigma(pop)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # events: step start, after the propagation call (dominant kernel), step end
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    n_launch[0] = 0  # only the timed steps
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            pop, _, _ = api.propagate(systems, trd, want_diag=False, device=True, stream=stream, **tune)
            n_launch[0] += api.last_launch_count()
            ev[k][1].record(stream)
            sigma(pop)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = sum(e[0].elapsed_time(e[2]) for e in ev)
    k_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    ms = max_over_ranks(ms, dist, dev)
    clocks = clk.summary()
    value = traj_steps * ws / (ms * 1e-3 / args.steps)
    # ---- roofline of the dominant launch: algorithmic work summed over the systems
    roofline = roofline_of(api, args.path, args.precision, infos, dg["steps"], sidx, k_ms)

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        tr_pin = torch.from_numpy(tr.view(np.uint8).copy()).pin_memory()
        tr_host = tr_pin.numpy().view(api.TRAJ_DTYPE)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop_h, _, diag_h = api.propagate(systems, tr_host, device=False, stream=stream, **tune)
        sig_bytes = 0
        for i, rows, sub in groups:
            w = api.sigma_weights(sub, diag_h["status"][rows])
            sg = api.cross_sections(systems[i], np.ascontiguousarray(pop_h[rows, :infos[i]["n_states"]]), w, sub.group,
                                    sub.n_groups, stream=stream)
            sig_bytes += sg.nbytes + w.nbytes + sub.group.astype(np.int32).nbytes
        e_ms_step = 1e3 * (time.perf_counter() - t0)
        h2d = tr.nbytes + pop_h.nbytes + sig_bytes
        d2h = pop_h.nbytes + ts.n * api.DIAG_DTYPE.itemsize + sig_bytes
        e2e = {"value": traj_steps * ws / (e_ms_step * 1e-3), "unit": "traj-steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms_step}

    # the same batch through the plain FP64 path: its throughput, and the largest population
    # difference of the measured path against it over every trajectory compared ("same error")
    compare = None
    if not args.no_compare and not (args.path == "plain" and args.precision == "fp64"):
        # one CTA per trajectory: at N = 1580 or 1600 the plain FP64 run is long, so those
        # workloads compare on a stratified 128-trajectory part of the batch
        if args.workload in ("asym1580", "mix"):
            cidx = np.sort(np.random.default_rng(9).choice(ts.n, min(128, ts.n), replace=False))
            if args.workload == "asym1580":
                cidx = strat_idx(ts, 128, seed=9)
        else:
            cidx = np.arange(ts.n)
        compare = compare_fp64(api, ps, tr, cidx, dg["steps"], pop.cpu().numpy()[cidx], sidx, infos, dev, stream,
                               flush, value, ws)

    # the N = 1600 workload, the metric's second basis size: the same measurement in short form
    n1600 = None
    if args.n1600 and args.workload == "n441" and not args.max_traj and not args.max_steps and not args.energy:
        n1600 = n1600_block(api, args, dev, stream, flush, ws)

    adj = None
    if args.adjoint:
        adj = adjoint_block(api, args.adjoint)
    rates = rates_block(api) if args.rates else None
    sparse = (sparse_block(api, n_traj=args.sparse_traj, max_steps=args.sparse_steps, jmax=args.sparse_jmax)
              if args.sparse else None)
    molmol = molmol_block(api) if args.molmol else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        p0 = ps[0] if args.workload != "mix" else ps[2]
        ts0 = ts if args.workload != "mix" else ts.subset(np.flatnonzero(sidx == 2))
        sub = oracle_sample(p0, ts0, 16) if args.workload != "mix" else ts0.subset(np.arange(min(16, ts0.n)))
        what = f"{sub.n} trajectories of the workload (stratified over the collision energies, seeded)"
        if args.workload == "asym1580":
            sub.max_steps = 400  # the oracle takes ~10 ms per step at N = 1580: the first 400 steps of each
            what += ", first 400 RK4 steps of each"
        if args.workload == "mix":
            sub.max_steps = 2000
            what = f"{sub.n} trajectories of the N = 441 part of the mix, first 2000 RK4 steps of each"
        cores = cpu_cores()
        s_, t_ = run_oracle(p0, sub, cores)
        cpu = {"value": s_ / t_, "unit": "traj-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{what}, {int(s_)} traj-steps"}
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    sigma_sets = sum(sub.n_groups for _, _, sub in groups)
    cfg = {"workload": workload, "path": args.path, "precision": args.precision,
           "n_states": [inf["n_states"] for inf in infos] if len(infos) > 1 else infos[0]["n_states"],
           "trajectories": ts.n, "traj_steps_per_step": traj_steps, "excluded_trajectories": n_bad,
           "l2": "flushed (256 MB write) before every timed step", "seed": W.DEFAULT_SEED}
    if tune:
        cfg["autotuned"] = {"option": tune, "reports": tune_report}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "traj-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "bf16x3"}[args.precision],
        "data": "synthetic", "config": cfg,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": n_launch[0], "latency": latency, "comparison": compare, "adjoint": adj,
        "sigma_sets_per_s": sigma_sets * ws / (ms * 1e-3 / args.steps),
        "sigma_set": "all cross sections out of one (collision energy, initial level) group",
        "n1600": n1600, "rates": rates, "sparse": sparse, "molmol": molmol,
    }))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
