"""Launch-shape autotuner for the mixed-precision trajectory paths.

The FP32 batched kernel exists in seven (slots per CTA, threads) instances and the BF16X3 path
runs a chosen number of trajectories in flight; which is fastest depends on the basis size, the
density of the coupling terms and the GPU.  ``tune`` times short probe runs of every candidate
on a sample of the caller's trajectories, each capped at ``probe_steps`` (E_min/E)^(1/2) RK4
steps (in proportion to its expected length, so that the probe keeps the mix of long and short
trajectories) so that a probe costs milliseconds, and returns the fastest option together with the measured table.
The options change launch shapes only, never the arithmetic of a trajectory beyond the order
of its FP32 partial sums.
"""
from __future__ import annotations

import numpy as np

from . import api


def _sample(trajs: np.ndarray, n: int) -> np.ndarray:
    if len(trajs) <= n:
        return trajs.copy()
    return trajs[np.linspace(0, len(trajs) - 1, n).astype(int)].copy()


def _time(system, tr_dev, opts, repeats, stream):
    import torch

    api.propagate(system, tr_dev, want_pop=False, want_diag=False, device=True, stream=stream, **opts)  # warm-up
    best = None
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        api.propagate(system, tr_dev, want_pop=False, want_diag=False, device=True, stream=stream, **opts)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return best


def candidates(system, n_traj: int) -> list[dict]:
    """The launch options worth timing for this system and this many trajectories."""
    info = system.info
    if info["precision"] == api.FP32:
        return [{"batch_shape": k} for k in range(1, len(api.BATCH_SHAPES) + 1)]
    if info["precision"] == api.BF16X3:
        import torch

        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        nt = max(1, info["n_row_tiles"])
        top = min(8192, 64 * ((n_traj + 63) // 64))
        # whole waves of (row tile, 64-slot tile) CTAs, and every trajectory in a slot at once
        out = sorted({min(top, 64 * max(1, (k * sms) // nt)) for k in (1, 2)} | {top})
        return [{"tc_slots": s} for s in out]
    return [{}]


def tune(system, trajs: np.ndarray, probe_steps: int = 300, max_sample: int = 8192, repeats: int = 2,
         stream=None) -> dict:
    """Time every candidate option on a sample of `trajs` (TRAJ_DTYPE, all naming this system as
    system 0) with each trajectory capped at probe_steps (E_min/E)^(1/2) steps.  Returns
    {"option": best options (keywords of api.propagate), "rate": traj-steps/s, "table": [...]}."""
    import torch

    tr = _sample(trajs, max_sample)
    # caps in proportion to each trajectory's expected length (1/velocity ~ E^-1/2), so that the
    # probe keeps the mix of long and short trajectories that decides how slots refill
    e = np.maximum(tr["e_coll"], 1e-300)
    cap = np.maximum(10, np.round(probe_steps * np.sqrt(e.min() / e))).astype(np.int32)
    tr["max_steps"] = np.minimum(tr["max_steps"], cap)
    tr["system_idx"] = 0
    tr_dev = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    _, _, dg = api.propagate(system, tr, want_pop=False, device=False)
    steps = float(dg["steps"].sum())
    table = []
    for opt in candidates(system, len(tr)):
        try:
            ms = _time(system, tr_dev, opt, repeats, stream)
        except api.MQCTError as err:
            if err.status == api.ERR_UNSUPPORTED:
                continue  # this shape does not fit the basis
            raise
        table.append({"option": opt, "ms": ms, "rate": steps / (ms * 1e-3)})
    best = max(table, key=lambda r: r["rate"])
    return {"option": best["option"], "rate": best["rate"], "table": table, "probe_steps": probe_steps,
            "sample": int(len(tr))}


def tune_joint(systems, trajs: np.ndarray, probe_steps: int = 300, max_sample: int = 8192, repeats: int = 2,
               stream=None) -> dict:
    """FP32 uneven batch: the whole call runs one persistent launch whose shape every system
    shares, so the candidates are timed on a sample of the mixed trajectories together."""
    import torch

    tr = _sample(trajs, max_sample)
    # caps in proportion to each trajectory's expected length (1/velocity ~ E^-1/2), so that the
    # probe keeps the mix of long and short trajectories that decides how slots refill
    e = np.maximum(tr["e_coll"], 1e-300)
    cap = np.maximum(10, np.round(probe_steps * np.sqrt(e.min() / e))).astype(np.int32)
    tr["max_steps"] = np.minimum(tr["max_steps"], cap)
    tr_dev = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    _, _, dg = api.propagate(systems, tr, want_pop=False, device=False)
    steps = float(dg["steps"].sum())
    table = []
    for k in range(1, len(api.BATCH_SHAPES) + 1):
        opt = {"batch_shape": [k] * len(systems)}
        try:
            ms = _time(systems, tr_dev, opt, repeats, stream)
        except api.MQCTError as err:
            if err.status == api.ERR_UNSUPPORTED:
                continue  # this shape does not fit every basis
            raise
        table.append({"option": {"batch_shape": k}, "ms": ms, "rate": steps / (ms * 1e-3)})
    best = max(table, key=lambda r: r["rate"])
    return {"option": best["option"], "rate": best["rate"], "table": table, "probe_steps": probe_steps,
            "sample": int(len(tr))}


def tune_batch(systems, trajs: np.ndarray, **kw) -> dict:
    """Launch options of a batch over one or several systems: the per-system option lists
    {"batch_shape": [...], "tc_slots": [...]} for api.propagate and the reports.  FP32: one shape for
    the single launch of the call (tune_joint); BF16X3: each system tuned on its own trajectories
    (the tensor-core path runs the systems one after another)."""
    if len(systems) > 1 and systems[0].info["precision"] == api.FP32:
        r = tune_joint(systems, trajs, **kw)
        k = int(r["option"]["batch_shape"])
        return {"batch_shape": [k] * len(systems), "tc_slots": [0] * len(systems), "reports": [r]}
    shapes, slots, reports = [], [], []
    for i, s in enumerate(systems):
        sub = trajs[trajs["system_idx"] == i]
        if len(sub) == 0:
            shapes.append(0)
            slots.append(0)
            reports.append(None)
            continue
        r = tune(s, sub, **kw)
        shapes.append(int(r["option"].get("batch_shape", 0)))
        slots.append(int(r["option"].get("tc_slots", 0)))
        reports.append(r)
    return {"batch_shape": shapes, "tc_slots": slots, "reports": reports}
