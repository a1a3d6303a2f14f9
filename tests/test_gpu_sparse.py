"""GPU parity of the paper-scale setup (Sec. III): logarithmic R grid (splines in ln R) and the
|M| truncation at two reference distances, against the oracle."""
import numpy as np
import pytest

import paper_2312_02322_gb300.inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mq():
    import torch

    assert torch.cuda.is_available()
    from paper_2312_02322_gb300 import api, build

    build.build()
    return api


@pytest.fixture(scope="module")
def ora():
    import oracle

    return oracle


TRUNC = (float(W.cm(W.PAPER_TRUNC_CM)), *W.PAPER_TRUNC_R)


def _pair(mq, ora, jmax, lam_max, path="plain", precision="fp64", trunc=TRUNC):
    p = W.sparse_pes_params(jmax=jmax, lam_max=lam_max)
    sys_ = mq.System.diatom(p, path=path, precision=precision, grid="log", trunc=trunc)
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             grid_log=True, trunc=trunc)
    return p, sys_, osys


def _trajs(mq, sys_, p, energies_cm, bs, init_js, r0=30.0, max_steps=1_000_000):
    e, b, j = np.meshgrid(W.cm(energies_cm), bs, init_js, indexing="ij")
    e, b, j = e.ravel(), b.ravel(), j.ravel().astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros_like(j), 1, r0=r0, r_end=r0, dt=5.0,
                   max_steps=max_steps, sampling="mc", b_max=float(np.max(bs)), n_b=0)
    return ts, mq.make_trajs(ts, sys_)


def _margin_ok(ora, osys, thr):
    """No element's max |M| at the two distances lies within 1e-9 (relative) of the threshold, so
    that both sides' FP64 splines take the same keep / drop decision."""
    full = ora.System(osys.energy, osys.level, osys.jq, osys.mq,
                      osys.trip if osys.G is None else osys.G, osys.v, osys.dv_ends, osys.mu, osys.r_min,
                      osys.r_max, grid_log=True, n_terms=osys.L)
    v, _, _ = ora.sys_terms(full, np.array(W.PAPER_TRUNC_R))
    G = osys.G
    m = np.maximum(np.abs(np.tensordot(v[0], G, 1)), np.abs(np.tensordot(v[1], G, 1)))
    nz = np.any(G != 0.0, axis=0)
    rel = np.abs(m[nz] - thr) / thr
    return rel.min() > 1e-9, int(nz.sum())


def test_log_grid_truncated_plain_matches_oracle(mq, ora):
    """Plain FP64 path, jmax = 6 (N = 49), lambda <= 8, 63-point log grid on 3-30 bohr, |M| > 50 cm^-1
    at 6.03 / 7.11 bohr (a threshold that drops 64 of 231 elements of this small basis): the dropped
    count equals the oracle's, and every trajectory (three energies, impact parameters through the
    wall) matches to 1e-8 with identical step counts."""
    trunc = (float(W.cm(50.0)), *W.PAPER_TRUNC_R)
    p, sys_, osys = _pair(mq, ora, 6, 8, trunc=trunc)
    ok, n_struct = _margin_ok(ora, osys, trunc[0])
    assert ok
    keep = ora.sys_kept(osys)
    G_any = np.any(osys.G != 0.0, axis=0)
    assert sys_.info["trunc_dropped"] == int((G_any & ~keep).sum()) > 0
    assert sys_.info["grid_kind"] == mq.GRID_LOG
    ts, tr = _trajs(mq, sys_, p, [100.0, 1000.0, 5000.0], [0.0, 3.0, 6.5], [0, 2])
    pop, amp, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(j), 0) for j in ts.init_j]
    oamp, ores = ora.propagate(osys, ts.e_coll, ts.b, s0, r0=30.0, r_end=30.0, dt=5.0)
    assert np.array_equal(dg["steps"], ores["steps"])
    assert np.array_equal(dg["status"], ores["status"])
    assert np.max(np.abs(pop - np.abs(oamp) ** 2)) < 1e-8


def test_log_grid_factorised_matches_oracle(mq, ora):
    """Factorised FP64 path on the log grid (no truncation): parity with the oracle to 1e-8."""
    p, sys_, osys = _pair(mq, ora, 5, 6, path="factorised", trunc=None)
    ts, tr = _trajs(mq, sys_, p, [300.0, 3000.0], [1.0, 5.0], [0, 1])
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(j), 0) for j in ts.init_j]
    oamp, ores = ora.propagate(osys, ts.e_coll, ts.b, s0, r0=30.0, r_end=30.0, dt=5.0)
    assert np.array_equal(dg["steps"], ores["steps"])
    assert np.max(np.abs(pop - np.abs(oamp) ** 2)) < 1e-8


def test_truncation_larger_basis_sampled(mq, ora):
    """jmax = 30 (N = 961), lambda <= 12: two trajectories against the oracle."""
    p, sys_, osys = _pair(mq, ora, 30, 12)
    assert sys_.info["trunc_dropped"] > 0
    ts, tr = _trajs(mq, sys_, p, [1000.0], [2.0, 7.0], [3])
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(j), 0) for j in ts.init_j]
    oamp, ores = ora.propagate(osys, ts.e_coll, ts.b, s0, r0=30.0, r_end=30.0, dt=5.0)
    assert np.array_equal(dg["steps"], ores["steps"])
    assert np.max(np.abs(pop - np.abs(oamp) ** 2)) < 1e-8


# ---------------------------------------------------------------- FP32 PLAIN path (large bases)
def _cmp_mixed(pop, dg, oamp, ores, tol=1e-4):
    assert np.max(np.abs(np.asarray(dg["steps"]) - ores["steps"])) <= 1
    assert np.array_equal(np.asarray(dg["status"]) & ~1, ores["status"] & ~1)
    err = np.max(np.abs(pop - np.abs(oamp) ** 2))
    assert err < tol, err
    return err


@pytest.mark.parametrize("grid,trunc_cm", [("uniform", None), ("log", 50.0)])
def test_fp32_plain_small_matches_oracle(mq, ora, grid, trunc_cm):
    """FP32 spline table, stage-synchronous sparse kernel: N = 49, with and without the log grid and
    truncation, against the oracle at the mixed-precision bar (1e-4, steps within one)."""
    p = W.sparse_pes_params(jmax=6, lam_max=8) if grid == "log" else W.diatom_pes_params(jmax=6, n_grid=200)
    trunc = None if trunc_cm is None else (float(W.cm(trunc_cm)), *W.PAPER_TRUNC_R)
    sys_ = mq.System.diatom(p, path="plain", precision="fp32", grid=grid, trunc=trunc)
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             grid_log=grid == "log", trunc=trunc)
    ts, tr = _trajs(mq, sys_, p, [300.0, 2000.0], [0.0, 2.5, 6.0], [0, 3])
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(j), 0) for j in ts.init_j]
    oamp, ores = ora.propagate(osys, ts.e_coll, ts.b, s0, r0=30.0, r_end=30.0, dt=5.0)
    _cmp_mixed(pop, dg, oamp, ores)


def test_fp32_plain_matches_fp64_plain_n961(mq, ora):
    """jmax = 30 (N = 961), lambda <= 12, log grid, |M| > 1 cm^-1: the FP32 sparse path against the
    FP64 plain kernel on 24 trajectories and against the oracle on two."""
    p, s64, osys = _pair(mq, ora, 30, 12)
    s32 = mq.System.diatom(p, path="plain", precision="fp32", grid="log", trunc=TRUNC)
    assert s32.info["trunc_dropped"] == s64.info["trunc_dropped"] > 0
    ts, tr = _trajs(mq, s64, p, [100.0, 1000.0, 5000.0], [0.5, 3.0, 5.0, 8.0], [0, 4])
    p64, _, d64 = mq.propagate(s64, tr, device=False)
    p32, _, d32 = mq.propagate(s32, tr, device=False)
    assert np.max(np.abs(np.asarray(d32["steps"]) - d64["steps"])) <= 1
    assert np.max(np.abs(p32 - p64)) < 1e-4
    sub = [0, len(ts.e_coll) - 1]
    s0 = [s64.state(int(ts.init_j[i]), 0) for i in sub]
    oamp, ores = ora.propagate(osys, ts.e_coll[sub], ts.b[sub], s0, r0=30.0, r_end=30.0, dt=5.0)
    _cmp_mixed(p32[sub], d32[sub], oamp, ores)


def test_fp32_plain_large_basis_sampled(mq, ora):
    """jmax = 200 (N = 40401), lambda <= 12, 63-point log grid on 3-30 bohr, |M| > 1 cm^-1 at 6.03 and
    7.11 bohr (the paper's setup on an atom + rotor): 256 trajectories started on the wall (r0 = 8)
    for 24 steps; three of them against the oracle (same cap, MAX_STEPS on both sides)."""
    p = W.sparse_pes_params(jmax=200, lam_max=12)
    sys_ = mq.System.diatom(p, path="plain", precision="fp32", grid="log", trunc=TRUNC)
    info = sys_.info
    assert info["n_states"] == 40401 and info["trunc_dropped"] > 0
    rng = np.random.default_rng(3)
    n = 256
    e = W.cm(rng.uniform(500.0, 5000.0, n))
    b = rng.uniform(0.0, 6.0, n)
    j = rng.integers(0, 30, n).astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros(n, np.int32), 1, r0=8.0, r_end=8.0, dt=5.0,
                   max_steps=24, sampling="mc", b_max=6.0, n_b=0)
    tr = mq.make_trajs(ts, sys_)
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    assert np.all(dg["steps"] == 24) and np.all(dg["status"] & 1)
    assert np.max(np.abs(pop.sum(axis=1) - 1.0)) < 1e-5
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             grid_log=True, trunc=TRUNC)
    sub = [0, 1, 2]
    s0 = [sys_.state(int(ts.init_j[i]), 0) for i in sub]
    oamp, ores = ora.propagate(osys, ts.e_coll[sub], ts.b[sub], s0, r0=8.0, r_end=8.0, dt=5.0, max_steps=24)
    assert np.all(ores["steps"] == 24)
    assert np.max(np.abs(pop[sub] - np.abs(oamp) ** 2)) < 1e-4


def test_fp32_plain_paper_size_sampled(mq, ora):
    """jmax = 446 (N = 199 809, the paper's ~2e5 states), lambda <= 12, 63-point log grid on 3-30 bohr,
    |M| > 1 cm^-1 at 6.03 and 7.11 bohr: 64 trajectories started on the wall (r0 = 8) for 4 steps keep
    their norms, and one of them matches the oracle (same cap on both sides)."""
    p = W.sparse_pes_params(jmax=446, lam_max=12)
    sys_ = mq.System.diatom(p, path="plain", precision="fp32", grid="log", trunc=TRUNC)
    info = sys_.info
    assert info["n_states"] == 199809 and info["trunc_dropped"] > 0
    rng = np.random.default_rng(5)
    n = 64
    e = W.cm(rng.uniform(500.0, 5000.0, n))
    b = rng.uniform(0.0, 6.0, n)
    j = rng.integers(0, 60, n).astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros(n, np.int32), 1, r0=8.0, r_end=8.0, dt=5.0,
                   max_steps=4, sampling="mc", b_max=6.0, n_b=0)
    tr = mq.make_trajs(ts, sys_)
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    assert np.all(dg["steps"] == 4) and np.all(dg["status"] & 1)
    assert np.max(np.abs(pop.sum(axis=1) - 1.0)) < 1e-5
    sub = [0]
    s0 = [sys_.state(int(ts.init_j[0]), 0)]
    del sys_
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             grid_log=True, trunc=TRUNC)
    oamp, ores = ora.propagate(osys, ts.e_coll[sub], ts.b[sub], s0, r0=8.0, r_end=8.0, dt=5.0, max_steps=4)
    assert np.all(ores["steps"] == 4)
    assert np.max(np.abs(pop[sub] - np.abs(oamp) ** 2)) < 1e-4
