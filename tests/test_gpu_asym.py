"""GPU parity on the atom + rigid asymmetric top system (Eq. 1 basis, Eq. 16 coupling): every
path and precision of the library against the CPU oracle on the same seeded inputs.  FP64:
1e-8 absolute on every final population with identical step counts; FP32 and 3xBF16
contractions: 1e-4."""
import numpy as np
import pytest

from paper_2312_02322_gb300 import inputs as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-4
COMBOS = [("plain", "fp64"), ("factorised", "fp64"), ("factorised", "fp32"), ("factorised", "bf16x3")]


@pytest.fixture(scope="module")
def mq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02322_gb300 import api, build

    build.build()
    return api


def check(pop_g, diag_g, pop_o, res_o, tol):
    if tol <= TOL_FP64:
        assert np.array_equal(diag_g["steps"], res_o["steps"])
    else:
        assert np.max(np.abs(np.asarray(diag_g["steps"]) - res_o["steps"])) <= 1
    assert np.array_equal(diag_g["status"], res_o["status"])
    err = float(np.max(np.abs(pop_g[:, : pop_o.shape[1]] - pop_o)))
    assert err < tol, err
    return err


@pytest.fixture(scope="module")
def small(ora):
    """J <= 4 truncated to N <= 60, 10 terms (lam <= 3), E in {300, 1500} cm^-1, 6 b each."""
    p, ts = W.small_asym_workload(energies=(300.0, 1500.0), n_per_e=6)
    osys = ora.asym_system(p)
    amp, res = ora.propagate(osys, ts.e_coll, ts.b, np.zeros(ts.n, int), r0=ts.r0, r_end=ts.r_end, dt=ts.dt)
    return p, ts, np.abs(amp) ** 2, res


@pytest.mark.parametrize("path,prec", COMBOS)
def test_small_asym_every_path(mq, small, path, prec):
    p, ts, pop_o, res_o = small
    sys = mq.System.asym_top(p, path=path, precision=prec)
    assert sys.info["n_states"] == pop_o.shape[1]
    tr = mq.make_trajs(ts, sys)
    pop, _, diag = mq.propagate(sys, tr, device=False)
    check(pop, diag, pop_o, res_o, TOL_FP64 if prec == "fp64" else TOL_MIXED)
    if prec == "fp64":
        assert np.allclose(diag["norm_dev"], res_o["norm_dev"], rtol=0, atol=1e-12)
    # cross sections per final level against the oracle's reduction
    w = mq.sigma_weights(ts, diag["status"])
    sig = mq.cross_sections(sys, pop, w, ts.group, ts.n_groups)
    assert sig.shape == (ts.n_groups, sys.n_levels)


@pytest.fixture(scope="module")
def full(ora):
    """The N = 1580 workload (110 levels, 28 terms).  The GPU runs 48 of its trajectories (the
    three highest energies) in one launch together with three sampled ones at the highest energy
    (b = 0.5, 2.5, 5 bohr) that start, like every trajectory of the workload, at R0 = 30 bohr; the
    oracle runs the sampled ones one by one."""
    p, ts = W.workload3(n_per_e=64)
    keep = np.flatnonzero(ts.e_coll >= ts.e_coll.max() * 0.2)
    rng = np.random.default_rng(3)
    bulk = ts.subset(np.sort(rng.choice(keep, 48, replace=False)))
    samp = ts.subset(np.flatnonzero(ts.e_coll == ts.e_coll.max())[:3])
    samp.b = np.array([0.5, 2.5, 5.0])
    assert samp.r0 == 30.0 and samp.r_end == 30.0
    osys = ora.asym_system(p)
    amp, res = ora.propagate(osys, samp.e_coll, samp.b, np.zeros(samp.n, int), r0=samp.r0, r_end=samp.r_end,
                             dt=samp.dt)
    return p, bulk, samp, np.abs(amp) ** 2, res


@pytest.mark.parametrize("path,prec", COMBOS)
def test_full_size_sampled(mq, full, path, prec):
    p, bulk, samp, pop_o, res_o = full
    sys = mq.System.asym_top(p, path=path, precision=prec)
    assert sys.info["n_states"] == 1580 and sys.info["max_block"] == 110
    tr = np.concatenate([mq.make_trajs(bulk, sys), mq.make_trajs(samp, sys)])
    pop, _, diag = mq.propagate(sys, tr, device=False)
    k = bulk.n
    check(pop[k:], {key: diag[key][k:] for key in diag.dtype.names}, pop_o, res_o,
          TOL_FP64 if prec == "fp64" else TOL_MIXED)
    # every trajectory of the launch ends normally and keeps its norm
    assert np.all(diag["status"] == 0)
    assert np.all(diag["norm_dev"] < (1e-6 if prec == "fp64" else 1e-3))
