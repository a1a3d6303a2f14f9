"""Uneven batches of several systems in one propagation call, per-trajectory timing, and the
launch-shape autotuner: every mixed-precision result is the same as running each system on its
own (the launch schedule does not enter a trajectory's arithmetic), and agrees with the oracle."""
import numpy as np
import pytest

from paper_2312_02322_gb300 import inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02322_gb300 import api, build

    build.build()
    return api


def mix(n_per=12, jmaxes=(3, 5, 8), seed=7):
    """Three small diatom bases, trajectories interleaved, E on 500-3000 cm^-1."""
    rng = np.random.default_rng(seed)
    ps = [W.diatom_pes_params(jmax=j, n_grid=120) for j in jmaxes]
    n = n_per * len(ps)
    sys_idx = np.repeat(np.arange(len(ps), dtype=np.int32), n_per)
    rng.shuffle(sys_idx)
    e = W.cm(rng.uniform(500.0, 3000.0, n))
    b = rng.uniform(0.0, 8.0, n)
    z = np.zeros(n, np.int32)
    ts = W.TrajSet(e, b, z, z.copy(), sys_idx.copy(), len(ps), sampling="mc", b_max=8.0, n_b=0, system=sys_idx,
                   group_e=np.zeros(len(ps)), group_j=np.zeros(len(ps), np.int32))
    return ps, ts


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp64"])
def test_uneven_batch_equals_separate_calls(mq, ora, prec):
    ps, ts = mix()
    path = "factorised"
    systems = [mq.System.diatom(p, path=path, precision=prec) for p in ps]
    tr = mq.make_trajs(ts, systems)
    pop, _, diag = mq.propagate(systems, tr, device=False)
    assert np.all(diag["status"] == 0)
    for i, p in enumerate(ps):
        rows = np.flatnonzero(ts.system == i)
        one = tr[rows].copy()
        one["system_idx"] = 0
        pop1, _, diag1 = mq.propagate(systems[i], one, device=False)
        n = systems[i].n
        assert np.array_equal(diag1["steps"], diag["steps"][rows])
        if prec == "fp64":
            assert np.max(np.abs(pop1[:, :n] - pop[rows, :n])) < 1e-13
        else:
            assert np.array_equal(pop1[:, :n], pop[rows, :n])  # same kernel shape, same arithmetic
    # a few trajectories of each system against the oracle
    tol = 1e-8 if prec == "fp64" else 1e-4
    for i, p in enumerate(ps):
        rows = np.flatnonzero(ts.system == i)[:3]
        osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
        amp, res = ora.propagate(osys, ts.e_coll[rows], ts.b[rows], np.zeros(len(rows), int), r0=ts.r0,
                                 r_end=ts.r_end, dt=ts.dt)
        n = systems[i].n
        assert np.max(np.abs(pop[rows, :n] - np.abs(amp) ** 2)) < tol


def test_timing_outputs(mq):
    import torch

    ps, ts = mix(n_per=8)
    systems = [mq.System.diatom(p, path="factorised", precision="fp32") for p in ps]
    tr = mq.make_trajs(ts, systems)
    t0 = np.zeros(ts.n, np.int64)
    t1 = np.zeros(ts.n, np.int64)
    mq.propagate(systems, tr, device=False, timing=(t0, t1))
    assert np.all(t0 > 0) and np.all(t1 > t0)
    # device arrays work the same way
    d0 = torch.zeros(ts.n, dtype=torch.int64, device="cuda")
    d1 = torch.zeros(ts.n, dtype=torch.int64, device="cuda")
    mq.propagate(systems, torch.from_numpy(tr.view(np.uint8).copy()).cuda(), device=True, timing=(d0, d1))
    torch.cuda.synchronize()
    assert bool((d1 > d0).all()) and bool((d0 > 0).all())


def test_shape_options_validated(mq):
    p, ts = W.small_workload(jmax=3)
    s = mq.System.diatom(p, path="factorised", precision="fp32")
    tr = mq.make_trajs(ts, s)
    with pytest.raises(mq.MQCTError) as e:
        mq.propagate(s, tr, device=False, batch_shape=8)
    assert e.value.status == mq.ERR_INVALID_ARG
    big = mq.System.diatom(W.diatom_pes_params(jmax=39, n_grid=60), path="factorised", precision="fp32")
    trb = mq.make_trajs(ts, big)
    with pytest.raises(mq.MQCTError) as e:
        mq.propagate(big, trb, device=False, batch_shape=1)  # 32 slots of N = 1600 do not fit
    assert e.value.status == mq.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_autotune_picks_a_valid_shape(mq, prec):
    from paper_2312_02322_gb300 import autotune

    p, ts = W.small_workload(jmax=5, n_b=32, energies=(1000.0,), init_js=(0,), m_avg="one")
    s = mq.System.diatom(p, path="factorised", precision=prec)
    tr = mq.make_trajs(ts, s)
    r = autotune.tune(s, tr, probe_steps=100, repeats=1)
    assert r["table"] and r["rate"] > 0
    assert r["option"] in [row["option"] for row in r["table"]]
    pop_a, _, _ = mq.propagate(s, tr, device=False)
    pop_t, _, _ = mq.propagate(s, tr, device=False, **r["option"])
    assert np.max(np.abs(pop_a - pop_t)) < 1e-5  # shapes change only the order of FP32 partial sums


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_launch_count(mq, prec):
    """mqct_last_launch_count: order keys + the persistent launch (FP64); order keys, the per-system
    work estimate and one persistent launch (FP32, three systems); order keys, the work estimate and
    per system the slot initialisation and 34 launches per graph chunk of four steps (BF16X3); the
    cross-section call launches two kernels."""
    ps, ts = mix(n_per=4)
    systems = [mq.System.diatom(p, path="factorised", precision=prec) for p in ps]
    tr = mq.make_trajs(ts, systems)
    pop, _, dg = mq.propagate(systems, tr, device=False)
    c = mq.last_launch_count()
    if prec == "fp64":
        assert c == 2
    elif prec == "fp32":
        assert c == 3
    else:
        assert c > 5 + 3 * 34 and (c - 5) % 34 == 0
    rows = np.flatnonzero(ts.system == 0)
    mq.cross_sections(systems[0], np.ascontiguousarray(pop[rows, :systems[0].n]), np.ones(rows.size),
                      np.zeros(rows.size, np.int32), 1)
    assert mq.last_launch_count() == 2
