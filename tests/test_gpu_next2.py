"""GPU parity of the decoupled classical motion (MQCT_DECOUPLED_TRAJ: the AT-MQCT decoupling of
Sec. III in the library's reading) against the oracle."""
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


@pytest.mark.parametrize("path", ["plain", "factorised"])
def test_decoupled_matches_oracle(mq, ora, path):
    """N = 49 diatom, three energies and impact parameters through the wall: populations to 1e-8,
    identical steps and status, the classical-energy and P_Phi diagnostics of the decoupled mode."""
    p = W.diatom_pes_params(jmax=6, n_grid=200)
    sys_ = mq.System.diatom(p, path=path, decoupled=True)
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
    e, b, j = np.meshgrid(W.cm([200.0, 1000.0, 4000.0]), [0.0, 2.5, 6.0], [0, 3], indexing="ij")
    e, b, j = e.ravel(), b.ravel(), j.ravel().astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros_like(j), 1, sampling="mc", b_max=6.0, n_b=0)
    tr = mq.make_trajs(ts, sys_)
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(jj), 0) for jj in j]
    oamp, ores = ora.propagate(osys, e, b, s0, flags=ora.F_DECOUPLED)
    assert np.array_equal(dg["steps"], ores["steps"])
    assert np.array_equal(dg["status"], ores["status"])
    assert np.max(np.abs(pop - np.abs(oamp) ** 2)) < 1e-8
    assert np.allclose(dg["energy_dev"], ores["energy_dev"], rtol=0, atol=1e-12)
    assert np.all(dg["angmom_dev"] == 0.0)
    # the path is the same for every initial state of one (E, b)
    st = dg["steps"].reshape(3, 3, 2)
    assert np.all(st[..., 0] == st[..., 1])


@pytest.mark.parametrize("path,decoupled", [("plain", False), ("factorised", False), ("factorised", True)])
def test_adaptive_steps_match_oracle(mq, ora, path, decoupled):
    """Step-doubling adaptive steps (tolerance 1e-6, steps between dt = 5 and 80 a.u.): the same accepted
    step count, final time, status and populations (1e-8) as the oracle's identical step control."""
    p = W.diatom_pes_params(jmax=5, n_grid=200)
    tol, hmax = 1e-6, 16
    sys_ = mq.System.diatom(p, path=path, decoupled=decoupled, adapt=(tol, hmax))
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             adapt=(tol, hmax))
    e, b, j = np.meshgrid(W.cm([150.0, 900.0, 3500.0]), [0.0, 3.0, 7.0], [0, 2], indexing="ij")
    e, b, j = e.ravel(), b.ravel(), j.ravel().astype(np.int32)
    ts = W.TrajSet(e, b, j, np.zeros_like(j), np.zeros_like(j), 1, sampling="mc", b_max=7.0, n_b=0)
    tr = mq.make_trajs(ts, sys_)
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    s0 = [sys_.state(int(jj), 0) for jj in j]
    oamp, ores = ora.propagate(osys, e, b, s0, flags=ora.F_DECOUPLED if decoupled else 0)
    assert np.array_equal(dg["steps"], ores["steps"])
    assert np.array_equal(dg["t_final"], ores["t_final"])
    assert np.array_equal(dg["status"], ores["status"])
    assert np.max(np.abs(pop - np.abs(oamp) ** 2)) < 1e-8
    # far fewer steps than the fixed dt would take
    assert np.all(dg["t_final"] / dg["steps"] > 2.0 * 5.0)


def test_adaptive_rejections(mq):
    """adapt_hmax not a power of 2, mixed precision or prescribed motion with adaptive steps."""
    p = W.diatom_pes_params(jmax=2, n_grid=100)
    with pytest.raises(mq.MQCTError):
        mq.System.diatom(p, adapt=(1e-6, 12))
    with pytest.raises(mq.MQCTError):
        mq.System.diatom(p, path="factorised", precision="fp32", adapt=(1e-6, 16))
    with pytest.raises(mq.MQCTError):
        mq.System.diatom(p, prescribed=True, adapt=(1e-6, 16))
