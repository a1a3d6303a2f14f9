"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on the same
seeded inputs.  FP64 paths: 1e-8 absolute on every final population and on the cross
sections relative to pi b_max^2; identical step counts and statuses."""
import numpy as np
import pytest

from paper_2312_02322_gb300 import inputs as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8


@pytest.fixture(scope="module")
def mq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02322_gb300 import api, build

    build.build()
    return api


def oracle_system(ora, p, with_params=False):
    return ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             with_params=with_params)


def oracle_run(ora, osys, ts):
    init = [j * j + j + m for j, m in zip(ts.init_j, ts.init_m)]
    amp, res = ora.propagate(osys, ts.e_coll, ts.b, init, r0=ts.r0, r_end=ts.r_end, dt=ts.dt,
                             max_steps=ts.max_steps)
    return np.abs(amp) ** 2, res


def gpu_run(mq, sys, ts, device=False):
    tr = mq.make_trajs(ts, sys)
    if device:
        import torch

        trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
        pop, _, diag = mq.propagate(sys, trd, device=True)
        torch.cuda.synchronize()
        return pop.cpu().numpy(), mq.diag_to_numpy(diag)
    pop, _, diag = mq.propagate(sys, tr, device=False)
    return pop, diag


def compare(pop_g, diag_g, pop_o, res_o, tol=TOL_FP64):
    """Element-wise comparison.  FP64 paths take the same number of steps as the oracle; the
    mixed path may end one step earlier or later (its force carries FP32 rounding, and the
    stop test compares R with r_end), which changes the final populations only through the
    coupling beyond r_end (~1e-9 hartree)."""
    if tol <= TOL_FP64:
        assert np.array_equal(diag_g["steps"], res_o["steps"])
        assert np.allclose(diag_g["t_final"], res_o["t_final"], rtol=0, atol=0)
    else:
        assert np.max(np.abs(np.asarray(diag_g["steps"]) - res_o["steps"])) <= 1
    assert np.array_equal(diag_g["status"], res_o["status"])
    err = np.max(np.abs(pop_g - pop_o))
    assert err < tol, err
    return err


@pytest.mark.parametrize("path", ["plain", "factorised"])
def test_small_full_m_average(mq, ora, path):
    """j <= 3 (N = 16), two initial levels with every m', six b: populations, diagnostics and sigma."""
    p, ts = W.small_workload(jmax=3, n_b=6, energies=(500.0, 2000.0), init_js=(0, 1), b_max=8.0, n_grid=120)
    sys = mq.System.diatom(p, path=path)
    pop_g, diag_g = gpu_run(mq, sys, ts)
    osys = oracle_system(ora, p)
    pop_o, res_o = oracle_run(ora, osys, ts)
    compare(pop_g, diag_g, pop_o, res_o)
    # diagnostics agree with the oracle's to well within their own size
    assert np.allclose(diag_g["norm_dev"], res_o["norm_dev"], rtol=0, atol=1e-12)
    assert np.allclose(diag_g["energy_dev"], res_o["energy_dev"], rtol=0, atol=1e-12)
    assert np.allclose(diag_g["angmom_dev"], res_o["angmom_dev"], rtol=0, atol=1e-9)
    w = mq.sigma_weights(ts, diag_g["status"])
    sig_g = mq.cross_sections(sys, pop_g, w, ts.group, ts.n_groups)
    sig_o = ora.cross_sections(osys, pop_o, w, ts.group, ts.n_groups)
    assert np.max(np.abs(sig_g - sig_o)) < TOL_FP64 * np.pi * ts.b_max ** 2
    assert np.allclose(sig_g.sum(axis=1), np.pi * ts.b_max ** 2, rtol=1e-9)


def test_workload1_full(mq, ora):
    """N = 49 workload (E = 500 cm^-1, j' = 0, 32 b on 0-12 bohr): every trajectory, plain FP64."""
    p, ts = W.workload1()
    sys = mq.System.diatom(p, path="plain")
    pop_g, diag_g = gpu_run(mq, sys, ts, device=True)
    pop_o, res_o = oracle_run(ora, oracle_system(ora, p), ts)
    compare(pop_g, diag_g, pop_o, res_o)
    assert np.max(diag_g["norm_dev"]) < 1e-10


TOL_MIXED = 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_mixed_small_and_workload1(mq, ora, prec):
    """Batched mixed paths (FP32 CUDA-core contraction; BF16x3 tcgen05 contraction), FP64
    classical motion and phase arguments, against the FP64 oracle: 1e-4 absolute on every final
    population, step counts within one."""
    for p, ts in (W.small_workload(jmax=3, n_b=6, energies=(500.0, 2000.0), init_js=(0, 1), b_max=8.0, n_grid=120),
                  W.workload1()):
        sys = mq.System.diatom(p, path="factorised", precision=prec)
        pop_g, diag_g = gpu_run(mq, sys, ts)
        pop_o, res_o = oracle_run(ora, oracle_system(ora, p), ts)
        err = compare(pop_g, diag_g, pop_o, res_o, tol=TOL_MIXED)
        assert np.max(np.abs(pop_g.sum(axis=1) - 1.0)) < 1e-4
        # total-energy drift relative to the collision energy: FP32 products carry ~6e-8
        # relative error, BF16x3 products (hi.hi + hi.lo + lo.hi) ~2^-16
        ebar = {"fp32": 1e-6, "bf16x3": 1e-5}[prec]
        assert np.max(diag_g["energy_dev"]) < ebar * float(np.max(ts.e_coll))
        w = mq.sigma_weights(ts, diag_g["status"])
        sig_g = mq.cross_sections(sys, pop_g, w, ts.group, ts.n_groups)
        sig_o = ora.cross_sections(oracle_system(ora, p), pop_o, w, ts.group, ts.n_groups)
        assert np.max(np.abs(sig_g - sig_o)) < TOL_MIXED * np.pi * ts.b_max ** 2


def w2_picks(ts):
    """One seeded trajectory per (collision energy, initial j') of the N = 441 workload: every
    energy is covered, from the longest trajectories (E = 100 cm^-1, ~29k steps, the most FP32
    accumulation in the mixed paths) to the shortest (E = 3000 cm^-1, ~5.6k steps)."""
    rng = np.random.default_rng(7)
    pick = [rng.choice(np.flatnonzero((ts.e_coll == e) & (ts.init_j == j)))
            for e in np.unique(ts.e_coll) for j in (0, 1, 2)]
    return np.array(sorted(pick))


@pytest.fixture(scope="module")
def w2(ora):
    """The N = 441 workload and the oracle's populations of its stratified sample (w2_picks)."""
    p, ts = W.workload2()
    pick = w2_picks(ts)
    pop_o, res_o = oracle_run(ora, oracle_system(ora, p), ts.subset(pick))
    return p, ts, pick, pop_o, res_o


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_mixed_workload2_sampled_at_full_size(mq, w2, prec):
    """N = 441 workload, all 3072 trajectories through a batched mixed launch (the bench's launch
    configuration); one trajectory per (E, j') is compared with the oracle at 1e-4, and the whole
    batch agrees with the FP64 path to 1e-4."""
    import torch

    p, ts, pick, pop_o, res_o = w2
    sysm = mq.System.diatom(p, path="factorised", precision=prec)
    tr = mq.make_trajs(ts, sysm)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    pop, _, diag = mq.propagate(sysm, trd, device=True)
    torch.cuda.synchronize()
    pop = pop.cpu().numpy()
    diag = mq.diag_to_numpy(diag)
    assert np.all(diag["status"] == 0)
    sys64 = mq.System.diatom(p, path="factorised", precision="fp64")
    pop64, _, diag64 = mq.propagate(sys64, trd, device=True)
    torch.cuda.synchronize()
    d64 = mq.diag_to_numpy(diag64)
    same = diag["steps"] == d64["steps"]
    assert np.mean(same) > 0.99
    assert np.max(np.abs(pop[same] - pop64.cpu().numpy()[same])) < TOL_MIXED
    sub = {k: diag[k][pick] for k in diag.dtype.names}
    compare(pop[pick], sub, pop_o, res_o, tol=TOL_MIXED)


@pytest.fixture(scope="module")
def n1600(ora):
    """24 trajectories of the N = 1600 workload (12 at E = 1000 and 12 at E = 3000 cm^-1, all
    three initial j') and the oracle's populations of one per (E, j')."""
    p, ts = W.workload2_n1600()
    rng = np.random.default_rng(9)
    idx = np.sort(np.concatenate([rng.choice(np.flatnonzero(ts.e_coll == e), 12, replace=False)
                                  for e in np.unique(ts.e_coll)]))
    sub = ts.subset(idx)
    pick = np.array([np.flatnonzero((sub.e_coll == e) & (sub.init_j == j))[0]
                     for e in np.unique(sub.e_coll) for j in (0, 1, 2)])
    pop_o, res_o = oracle_run(ora, oracle_system(ora, p), sub.subset(pick))
    return p, sub, pick, pop_o, res_o


@pytest.mark.parametrize("path,prec", [("plain", "fp64"), ("factorised", "fp32"), ("factorised", "bf16x3")])
def test_n1600_sampled(mq, n1600, path, prec):
    """N = 1600 (j <= 39): 24 trajectories through the plain FP64 path and the two batched mixed
    paths; one per (E, j') recomputed by the oracle (1e-8 / 1e-4)."""
    p, sub, pick, pop_o, res_o = n1600
    sys_ = mq.System.diatom(p, path=path, precision=prec)
    pg, dg = gpu_run(mq, sys_, sub, device=True)
    assert np.all(dg["status"] == 0)
    compare(pg[pick], {k: dg[k][pick] for k in dg.dtype.names}, pop_o, res_o,
            tol=TOL_FP64 if prec == "fp64" else TOL_MIXED)


def test_paths_agree(mq):
    """PLAIN (spline of M) and FACTORISED (sum of v_l G^l) are the same function: agree to 1e-12."""
    p, ts = W.small_workload(jmax=5, n_b=5, energies=(800.0,), init_js=(1, 2), b_max=9.0, n_grid=150)
    a = mq.System.diatom(p, path="plain")
    b = mq.System.diatom(p, path="factorised")
    pa, da = gpu_run(mq, a, ts)
    pb, db = gpu_run(mq, b, ts)
    assert np.array_equal(da["steps"], db["steps"])
    assert np.max(np.abs(pa - pb)) < 1e-12


def test_host_and_device_pointers_agree(mq):
    p, ts = W.small_workload(jmax=2, n_b=4, energies=(600.0,), init_js=(1,), b_max=7.0, n_grid=80)
    sys = mq.System.diatom(p)
    ph, dh = gpu_run(mq, sys, ts, device=False)
    pd, dd = gpu_run(mq, sys, ts, device=True)
    assert np.array_equal(ph, pd)
    assert np.array_equal(dh["steps"], dd["steps"])


def test_workload2_sampled_at_full_size(mq, ora, w2):
    """N = 441 workload: the full 3072-trajectory batch in the bench launch configuration; one
    trajectory per (E, j') and the trajectory with the largest norm drift are recomputed one by
    one by the oracle (1e-8, identical step counts)."""
    import torch

    p, ts, pick, pop_o, res_o = w2
    sys = mq.System.diatom(p, path="plain")
    tr = mq.make_trajs(ts, sys)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    pop, _, diag = mq.propagate(sys, trd, device=True)
    torch.cuda.synchronize()
    pop = pop.cpu().numpy()
    diag = mq.diag_to_numpy(diag)
    assert np.all(diag["status"] == 0)
    # RK4 at dt = 5 is not exactly unitary: for this basis (couplings up to ~3000 cm^-1 at the
    # turning point, gaps up to 1480 cm^-1) the norm drifts by up to ~2e-7; the oracle shows the
    # same drift on the sampled trajectories below
    assert np.max(diag["norm_dev"]) < 1e-6
    assert np.max(np.abs(pop.sum(axis=1) - 1.0)) <= np.max(diag["norm_dev"]) * 1.0001
    sub = {k: diag[k][pick] for k in diag.dtype.names}
    compare(pop[pick], sub, pop_o, res_o)
    assert np.allclose(sub["norm_dev"], res_o["norm_dev"], rtol=1e-3, atol=1e-12)
    worst = int(np.argmax(diag["norm_dev"]))
    pw, rw = oracle_run(ora, oracle_system(ora, p), ts.subset([worst]))
    compare(pop[[worst]], {k: diag[k][[worst]] for k in diag.dtype.names}, pw, rw)


def test_edge_cases(mq, ora):
    import torch

    p, ts = W.small_workload(jmax=2, n_b=2, energies=(500.0,), init_js=(0,), b_max=6.0, n_grid=60)
    sys = mq.System.diatom(p)
    # no trajectories
    pop, _, diag = mq.propagate(sys, np.zeros(0, mq.TRAJ_DTYPE), device=False)
    assert pop.shape == (0, sys.n)
    # max_steps = 0: initial state returned, status MAX_STEPS
    tr = mq.make_trajs(ts, sys)
    tr["max_steps"] = 0
    pop, _, diag = mq.propagate(sys, tr, device=False)
    assert np.all(diag["status"] == mq.TRAJ_MAX_STEPS) and np.all(diag["steps"] == 0)
    assert np.allclose(pop[:, 0], 1.0) and np.allclose(pop[:, 1:], 0.0)
    # invalid host trajectory -> INVALID_ARG, nothing launched
    tr = mq.make_trajs(ts, sys)
    tr["init_state"][0] = sys.n
    with pytest.raises(mq.MQCTError) as ei:
        mq.propagate(sys, tr, device=False)
    assert ei.value.status == mq.ERR_INVALID_ARG
    # invalid device trajectory -> status INVALID for it, others run
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    _, _, diag = mq.propagate(sys, trd, device=True)
    d = mq.diag_to_numpy(diag)
    assert d["status"][0] == mq.TRAJ_INVALID and d["status"][1] == 0
    # head-on at high energy reaches below the grid: TABLE_RANGE reported, same as the oracle
    p2 = W.diatom_pes_params(jmax=1, n_grid=60)
    p2.r_min = 3.0
    sys2 = mq.System.diatom(p2)
    ts2 = W.regular_set([20000.0], [0], n_b=1, b_max=0.2)
    pg, dg = gpu_run(mq, sys2, ts2)
    po, ro = oracle_run(ora, oracle_system(ora, p2), ts2)
    assert dg["status"][0] & mq.TRAJ_TABLE_RANGE
    compare(pg, dg, po, ro)


def test_two_level_custom_system(mq, ora):
    """A caller-described system (dense G, Coriolis off via j = -1, single state per block of m)
    against the oracle: Rabi-type two-level problem with an R-dependent coupling."""
    import ctypes as C

    n, L, ng = 2, 2, 30
    e = np.array([0.0, 2e-3])
    lev = np.array([0, 1], np.int32)
    jj = np.array([-1, -1], np.int32)
    mm = np.array([0, 0], np.int32)
    G = np.zeros((L, n, n))
    G[0] = np.eye(2)
    G[1] = [[0.0, 1.0], [1.0, 0.0]]
    R = np.linspace(2.0, 30.0, ng)
    v = np.stack([0.5 * np.exp(-1.5 * R), 0.05 * np.exp(-1.2 * R)])
    ends = np.array([[-0.75 * np.exp(-3.0), -0.75 * np.exp(-45.0)], [-0.06 * np.exp(-2.4), -0.06 * np.exp(-36.0)]])
    d = mq.Desc()
    d.n_states, d.energy, d.level, d.j, d.m = n, e.ctypes.data, lev.ctypes.data, jj.ctypes.data, mm.ctypes.data
    d.mu, d.n_terms, d.G = 3000.0, L, G.ctypes.data
    d.n_grid, d.r_min, d.r_max, d.v, d.dv_ends = ng, 2.0, 30.0, v.ctypes.data, ends.ctypes.data
    sys = mq.System(d)
    tr = np.zeros(3, mq.TRAJ_DTYPE)
    tr["e_coll"] = [5e-3, 1e-2, 2e-2]
    tr["b"] = [0.0, 1.0, 3.0]
    tr["r0"], tr["r_end"], tr["dt"], tr["max_steps"] = 30.0, 30.0, 4.0, 100000
    pop, _, diag = mq.propagate(sys, tr, device=False)
    osys = ora.System(e, lev, jj, mm, G, v, ends, 3000.0, 2.0, 30.0)
    amp, res = ora.propagate(osys, tr["e_coll"], tr["b"], [0, 0, 0], dt=4.0, max_steps=100000)
    compare(pop, diag, np.abs(amp) ** 2, res)
    assert np.min(pop[:, 1]) > 1e-4
