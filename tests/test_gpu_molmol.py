"""GPU parity of an asymmetric top + linear rotor system (composite states of Eq. 3, coupling of
Eqs. 13-17, the paper's kind of system) against the oracle."""
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


def oracle_system(ora, p):
    lev_J, lev_E, lev_b = [], [], []
    for J in range(p.j1max + 1):
        E, b = ora.asym_levels(J, p.A, p.B, p.C)
        for e_, bb in zip(E, b):
            row = np.zeros(2 * p.j1max + 1)
            row[p.j1max - J:p.j1max + J + 1] = bb
            lev_J.append(J); lev_E.append(e_); lev_b.append(row)
    lev_J = np.array(lev_J, np.int32)
    e, lev, jt, mt, l1, j2 = ora.molmol_states(lev_J, p.j2, lev_E, p.bconst2)
    G = np.stack([ora.molmol_G(lev_J, np.array(lev_b), p.j1max, l1, j2, jt, mt, *t) for t in p.terms])
    v, ends, _, _ = ora.diatom_pes(p.coef, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
    return ora.System(e, lev, jt, mt, G, v, ends, p.mu, p.r_min, p.r_max), e


def _trajs(mq, sys_, e_cm, bs, init_states, dt=5.0):
    e, b, s = np.meshgrid(W.cm(e_cm), bs, init_states, indexing="ij")
    tr = np.zeros(e.size, mq.TRAJ_DTYPE)
    tr["e_coll"], tr["b"], tr["init_state"] = e.ravel(), b.ravel(), s.ravel()
    tr["r0"], tr["r_end"], tr["dt"], tr["max_steps"] = 30.0, 30.0, dt, 1_000_000
    return tr


@pytest.mark.parametrize("path,precision,tol", [("plain", "fp64", 1e-8), ("factorised", "fp64", 1e-8),
                                                ("factorised", "fp32", 1e-4)])
def test_molmol_matches_oracle(mq, ora, path, precision, tol):
    """Water-like top (j1 <= 2) + para-H2 (j2 in {0, 2}), nine PES terms: N = 210 composite states;
    trajectories from three initial states (ground level, (1_11)0, (0_00)2) at two energies and three
    impact parameters against the oracle."""
    p = W.molmol_params(j1max=2, j2=(0, 2))
    sys_ = mq.System.molmol(p, path=path, precision=precision)
    osys, e = oracle_system(ora, p)
    assert sys_.n == len(e)
    init = [0, int(np.flatnonzero(osys.level == 2)[0]), int(np.flatnonzero(osys.level == 1)[0])]
    tr = _trajs(mq, sys_, [300.0, 2000.0], [0.0, 3.0, 6.5], init)
    pop, _, dg = mq.propagate(sys_, tr, device=False)
    oamp, ores = ora.propagate(osys, tr["e_coll"], tr["b"], tr["init_state"])
    if tol <= 1e-8:
        assert np.array_equal(dg["steps"], ores["steps"])
    else:
        assert np.max(np.abs(np.asarray(dg["steps"]) - ores["steps"])) <= 1
    assert np.array_equal(dg["status"], ores["status"])
    err = np.max(np.abs(pop - np.abs(oamp) ** 2))
    assert err < tol, err
    # something happened: population left the initial states
    assert np.min(pop[np.arange(len(tr)), tr["init_state"]]) < 0.99
