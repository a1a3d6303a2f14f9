"""Prescribed-trajectory mode (MQCT_PRESCRIBED_TRAJ) on the GPU: the quantum equations (Eqs. 4-6)
along a time-symmetric straight line instead of the Ehrenfest motion.  Its populations agree with
the oracle's prescribed-line mode to 1e-8, and the discrete propagator obeys microscopic
reversibility (Eq. 19) exactly: g' P(l' -> l'') = g'' P(l'' -> l') to rounding."""
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


def line_trajs(mq, sys_, e, b, dt, steps, init):
    tr = np.zeros(len(init), mq.TRAJ_DTYPE)
    tr["e_coll"], tr["b"], tr["r0"], tr["r_end"] = e, b, 30.0, 30.0
    tr["dt"], tr["max_steps"], tr["init_state"] = dt, steps, init
    return tr


@pytest.mark.parametrize("path", ["plain", "factorised"])
def test_prescribed_line_matches_oracle(mq, ora, path):
    p = W.diatom_pes_params(jmax=3, n_grid=120)
    sys_ = mq.System.diatom(p, path=path, prescribed=True)
    v, dt = 1.2e-3, 4.0
    e = 0.5 * p.mu * v * v
    steps = int(round(2 * 28.0 / v / dt))
    init = [0, 2, 5, 9]
    bs = [2.5, 3.0, 4.0, 5.0]  # the line stays on the spline grid (R >= r_min)
    tr = line_trajs(mq, sys_, e, bs, dt, steps, init)
    pop, _, diag = mq.propagate(sys_, tr, device=False)
    assert np.all(diag["status"] == 0) and np.all(diag["steps"] == steps)
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
    vline = np.sqrt(2.0 * np.full(len(init), e) / p.mu)  # the speed the library derives from e_coll
    amp, res = ora.propagate(osys, [e] * len(init), bs, init, dt=dt, max_steps=steps, flags=ora.F_PRESCRIBED,
                             line_speed=vline)
    assert np.array_equal(res["steps"], diag["steps"])
    err = np.max(np.abs(pop - np.abs(amp) ** 2))
    assert err < 1e-8, err
    assert np.max(pop[:, 1:]) > 1e-3  # the line passes close enough to couple the states


def test_detailed_balance_exact_on_gpu(mq):
    """Every initial state of a j <= 2 basis along one line: the level-summed transition
    probabilities S[l'][l''] = sum_{i in l', f in l''} |U_fi|^2 form a symmetric matrix."""
    p = W.diatom_pes_params(jmax=2, n_grid=120)
    sys_ = mq.System.diatom(p, path="factorised", prescribed=True)
    v, b = 1.2e-3, 3.0
    e = 0.5 * p.mu * v * v
    for dt in (4.0, 2.0):
        steps = int(round(2 * 28.0 / v / dt))
        n = sys_.n
        tr = line_trajs(mq, sys_, e, [b] * n, dt, steps, list(range(n)))
        pop, _, diag = mq.propagate(sys_, tr, device=False)
        assert np.all(diag["status"] == 0)
        S = np.zeros((3, 3))
        for i in range(n):
            for f in range(n):
                S[sys_.level[i], sys_.level[f]] += pop[i, f]
        assert np.max(S - np.diag(np.diag(S))) > 1e-3
        assert np.max(np.abs(S - S.T)) < 1e-12, np.max(np.abs(S - S.T))


def test_prescribed_needs_fp64(mq):
    p = W.diatom_pes_params(jmax=1, n_grid=40)
    with pytest.raises(mq.MQCTError) as ei:
        mq.System.diatom(p, path="factorised", precision="fp32", prescribed=True)
    assert ei.value.status == mq.ERR_UNSUPPORTED
