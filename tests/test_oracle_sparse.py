"""Pins of the oracle's paper-scale setup (Sec. III): the logarithmic R grid (spline in ln R), the
|M| truncation and the sparse (triplet) input of large bases.  CPU only."""
import numpy as np
import pytest

import paper_2312_02322_gb300.inputs as W


@pytest.fixture(scope="module")
def ora():
    import oracle

    return oracle


def _log_system(ora, v, ends, n_grid, r_min, r_max, trunc=None):
    G = np.zeros((1, 1, 1))
    G[0] = 1.0
    return ora.System([0.0], [0], [-1], [0], G, v, ends, mu=3000.0, r_min=r_min, r_max=r_max, grid_log=True,
                      trunc=trunc)


def test_log_grid_spline_reproduces_cubic_in_lnR(ora):
    """A clamped spline in x = ln R reproduces any cubic in ln R; its R-derivatives follow the chain
    rule f' = f_x / R and f'' = (f_xx - f_x) / R^2 (a spline in R, or a missing 1/R, fails)."""
    a, b, c, d = 0.3, -0.7, 0.25, -0.04
    f = lambda x: a + b * x + c * x ** 2 + d * x ** 3
    fx = lambda x: b + 2 * c * x + 3 * d * x ** 2
    fxx = lambda x: 2 * c + 6 * d * x
    r_min, r_max, n = 3.0, 30.0, 63
    R = r_min * (r_max / r_min) ** (np.arange(n) / (n - 1))
    v = f(np.log(R))[None, :]
    ends = np.array([[fx(np.log(r_min)) / r_min, fx(np.log(r_max)) / r_max]])
    sys = _log_system(ora, v, ends, n, r_min, r_max)
    Rq = np.array([3.0, 3.37, 5.5, 6.03, 7.11, 12.9, 29.99, 30.0])
    val, d1, d2 = ora.sys_terms(sys, Rq)
    x = np.log(Rq)
    assert np.allclose(val[:, 0], f(x), rtol=0, atol=1e-13)
    assert np.allclose(d1[:, 0], fx(x) / Rq, rtol=1e-11, atol=1e-14)
    assert np.allclose(d2[:, 0], (fxx(x) - fx(x)) / Rq ** 2, rtol=1e-10, atol=1e-14)


def test_log_grid_pes_fourth_order(ora):
    """The diatom PES on 63 and 125 log-spaced points over 3-30 bohr (Sec. III): the interpolation
    error of v_lambda(R) and of dv/dR shrinks as h^4 and h^3 in the ln R spacing."""
    p = W.diatom_pes_params(jmax=2)
    Rq = np.linspace(3.05, 29.9, 997)
    exact = []
    for l in range(len(p.A)):
        e = p.A[l] * np.exp(-p.beta[l] * Rq)
        de = -p.beta[l] * e
        if l == 0:
            u = (Rq / p.rd) ** 6
            e = e - p.c6 * Rq ** -6 * (1 - np.exp(-u))
            de = de + 6 * p.c6 * Rq ** -7 * (1 - np.exp(-u)) - p.c6 * Rq ** -6 * np.exp(-u) * 6 * u / Rq
        exact.append((e, de))
    errs = []
    for n in (63, 125):
        sys = ora.diatom_system(2, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, n, 3.0, 30.0, grid_log=True)
        val, d1, _ = ora.sys_terms(sys, Rq)
        ev = max(np.max(np.abs(val[:, l] - exact[l][0]) / np.max(np.abs(exact[l][0]))) for l in range(len(p.A)))
        ed = max(np.max(np.abs(d1[:, l] - exact[l][1]) / np.max(np.abs(exact[l][1]))) for l in range(len(p.A)))
        errs.append((ev, ed))
    assert 11 < errs[0][0] / errs[1][0] < 22
    assert 6 < errs[0][1] / errs[1][1] < 11
    assert errs[0][0] < 1e-4


def _two_level(ora, delta, vc, trunc=None, n_grid=8):
    G = np.zeros((2, 2, 2))
    G[0] = [[1, 0], [0, 1]]
    G[1] = [[0, 1], [1, 0]]
    v = np.zeros((2, n_grid))
    v[0] = 1e-3
    v[1] = vc
    return ora.System([0.0, delta], [0, 1], [-1, -1], [0, 0], G, v, np.zeros((2, 2)), mu=7000.0, r_min=2.0,
                      r_max=30.0, trunc=trunc)


@pytest.mark.parametrize("thr_frac, coupled", [(0.5, True), (2.0, False)])
def test_truncation_two_level_rabi(ora, thr_frac, coupled):
    """Two levels with a constant coupling vc: a threshold below vc keeps the Rabi closed form
    4 vc^2 / Om^2 sin^2(Om t / 2); one above drops the coupling and the population stays put
    (the diagonal 1e-3 hartree is above both thresholds and is kept)."""
    delta, vc = 1e-3, 2e-4
    sys = _two_level(ora, delta, vc, trunc=(thr_frac * vc, 6.03, 7.11))
    keep = ora.sys_kept(sys)
    assert keep[0, 0] and keep[1, 1] and keep[0, 1] == coupled and keep[1, 0] == coupled
    amp, res = ora.propagate(sys, [0.1], [0.0], [0], dt=5.0, max_steps=2000, flags=ora.F_NO_STOP)
    T = res["t_final"][0]
    om = np.sqrt(delta ** 2 + 4 * vc ** 2)
    want = 4 * vc ** 2 / om ** 2 * np.sin(om * T / 2) ** 2 if coupled else 0.0
    assert abs(abs(amp[0, 1]) ** 2 - want) < 1e-10


def test_truncation_mask_properties(ora):
    """On the diatom of the paper-scale setup: the mask is symmetric, nested in the threshold, only
    couples equal m, keeps every element at threshold 0 (identical propagation to no truncation)
    and, at a threshold above every off-diagonal |M| at 6.03 and 7.11 bohr but below the diagonal,
    only the diagonal -- a b = 0 trajectory then stays in its initial state (no Coriolis coupling
    without rotation)."""
    p = W.sparse_pes_params(jmax=4, lam_max=4)
    args = (4, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, 63, 3.0, 30.0)
    full = ora.diatom_system(*args, grid_log=True)
    masks = []
    for thr in (10.0, 100.0, 150.0, 400.0):
        s = ora.diatom_system(*args, grid_log=True, trunc=(W.cm(thr), 6.03, 7.11))
        k = ora.sys_kept(s)
        assert np.array_equal(k, k.T)
        assert not np.any(k & (full.mq[:, None] != full.mq[None, :]))
        masks.append(k)
    for a, b in zip(masks, masks[1:]):
        assert np.all(b <= a) and b.sum() < a.sum()
    # at 400 cm^-1 (off-diagonal |M| < 280, diagonal > 1470 cm^-1 at the two distances)
    assert np.array_equal(masks[-1], np.eye(full.n, dtype=bool))
    s0 = ora.diatom_system(*args, grid_log=True, trunc=(0.0, 6.03, 7.11))
    a0, r0 = ora.propagate(s0, [W.cm(1000.0)], [2.0], [3])
    a1, r1 = ora.propagate(full, [W.cm(1000.0)], [2.0], [3])
    assert np.array_equal(a0, a1) and np.array_equal(r0["steps"], r1["steps"])
    sd = ora.diatom_system(*args, grid_log=True, trunc=(W.cm(400.0), 6.03, 7.11))
    ad, rd = ora.propagate(sd, [W.cm(1000.0)], [0.0], [3])
    pop = np.abs(ad[0]) ** 2
    assert np.all(np.delete(pop, 3) == 0.0)          # nothing leaves the initial state
    assert abs(pop[3] - 1.0) < 1e-8                  # RK4's norm drift of a pure phase rotation


def test_triplet_input_equals_dense(ora):
    """The sparse (triplet) form of G gives the same propagation as the dense one."""
    p = W.sparse_pes_params(jmax=5, lam_max=6)
    args = (5, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, 63, 3.0, 30.0)
    for kw in ({}, {"grid_log": True, "trunc": (W.cm(1.0), 6.03, 7.11)}):
        sd = ora.diatom_system(*args, sparse=False, **kw)
        ss = ora.diatom_system(*args, sparse=True, **kw)
        e, b, s0 = W.cm([800.0, 2500.0]), [1.5, 6.0], [0, 7]
        ad, rd = ora.propagate(sd, e, b, s0)
        as_, rs = ora.propagate(ss, e, b, s0)
        assert np.max(np.abs(ad - as_)) < 1e-13
        assert np.array_equal(rd["steps"], rs["steps"])
