"""Pins of the oracle's decoupled classical motion (the AT-MQCT decoupling of Sec. III, read as:
R and Phi move in the isotropic potential v_0 alone, with no torque, and the amplitudes follow
Eq. 5 along that path) and of its adaptive step control.  CPU only."""
import numpy as np
import pytest

import paper_2312_02322_gb300.inputs as W


@pytest.fixture(scope="module")
def ora():
    import oracle

    return oracle


def _diatom(ora, jmax=3, iso=True, aniso=1.0, n_grid=200):
    p = W.diatom_pes_params(jmax=jmax, n_grid=n_grid)
    A = np.array(p.A, dtype=np.float64)
    c6 = p.c6
    if not iso:
        A[0] = 0.0
        c6 = 0.0
    A[1:] *= aniso
    return ora.diatom_system(jmax, p.bconst, p.mu, A, p.beta, c6, p.rd, n_grid, p.r_min, p.r_max), p


def test_decoupled_free_motion_is_a_straight_line(ora):
    """No isotropic potential, strong anisotropy: the decoupled classical motion is the free straight
    line R(t)^2 = b^2 + (v t - sqrt(r0^2 - b^2))^2 with Phi the angle swept, whatever the amplitudes
    do; P_Phi is exactly constant.  The coupled (Ehrenfest) motion is not a straight line here."""
    sys, p = _diatom(ora, iso=False, aniso=3.0)
    e, b, r0 = W.cm(800.0), 4.0, 30.0
    amp, res = ora.propagate(sys, [e], [b], [0], r0=r0, r_end=r0, dt=5.0, flags=ora.F_DECOUPLED)
    v = np.sqrt(2 * e / p.mu)
    t = res["t_final"][0]
    x0 = -np.sqrt(r0 ** 2 - b ** 2)
    x = x0 + v * t
    assert res["R"][0] == pytest.approx(np.hypot(b, x), rel=1e-9)
    assert res["Phi"][0] == pytest.approx(np.arctan2(x, b) - np.arctan2(x0, b), rel=1e-8)
    assert res["PPhi"][0] == b * np.sqrt(2 * p.mu * e)
    assert res["angmom_dev"][0] == 0.0
    # the amplitudes did change (the coupling acts on them, not on the path)
    assert abs(amp[0, 0]) ** 2 < 0.999
    _, rc = ora.propagate(sys, [e], [b], [0], r0=r0, r_end=r0, dt=5.0)
    assert abs(rc["R"][0] - res["R"][0]) > 1e-3 or rc["steps"][0] != res["steps"][0]


def test_decoupled_path_does_not_depend_on_the_initial_state(ora):
    """The classical path is the same for every initial state (bit for bit)."""
    sys, _ = _diatom(ora)
    e, b = W.cm(1500.0), 3.0
    _, res = ora.propagate(sys, [e] * 4, [b] * 4, [0, 3, 5, 13], flags=ora.F_DECOUPLED)
    for k in ("steps", "R", "PR", "Phi", "PPhi"):
        assert np.all(res[k] == res[k][0])
    _, rc = ora.propagate(sys, [e] * 2, [b] * 2, [0, 13])
    assert rc["R"][0] != rc["R"][1] or rc["steps"][0] != rc["steps"][1]


def test_decoupled_classical_energy_converges(ora):
    """The classical energy P_R^2/2mu + P_Phi^2/(2 mu R^2) + v_0(R) is conserved to the integrator's
    order (third: the force is the derivative of a C^2 spline)."""
    sys, _ = _diatom(ora)
    e, b = W.cm(1000.0), 2.0
    devs = []
    for dt in (4.0, 2.0):
        _, res = ora.propagate(sys, [e], [b], [2], dt=dt, flags=ora.F_DECOUPLED)
        devs.append(res["energy_dev"][0])
    assert devs[0] < 1e-7 * e
    assert devs[0] / devs[1] > 6.0


def test_decoupled_reversibility(ora):
    """Along a decoupled path the classical motion is time-symmetric about its turning point, so the
    state-to-state probabilities obey microscopic reversibility P(i->f) = P(f->i) up to the
    asymmetry of the stop rule's last step (below 3e-5 here); the coupled Ehrenfest path depends on
    the initial state and misses it by 400 times more."""
    sys, _ = _diatom(ora, jmax=2)
    e, b = W.cm(600.0), 1.0
    states = [0, 4]            # (j, m) = (0, 0) and (2, -2)
    rel = {}
    for fl in (ora.F_DECOUPLED, 0):
        a_f, _ = ora.propagate(sys, [e, e], [b, b], states, dt=2.0, flags=fl)
        p_if = abs(a_f[0, states[1]]) ** 2
        p_fi = abs(a_f[1, states[0]]) ** 2
        assert p_if > 1e-4
        rel[fl] = abs(p_if - p_fi) / p_if
    assert rel[ora.F_DECOUPLED] < 3e-5
    assert rel[0] > 100 * rel[ora.F_DECOUPLED]


def test_decoupled_needs_isotropic_identity_term(ora):
    G = np.zeros((1, 2, 2))
    G[0] = [[0, 1], [1, 0]]
    s = ora.System([0.0, 1e-3], [0, 1], [-1, -1], [0, 0], G, np.full((1, 8), 1e-4), np.zeros((1, 2)), mu=7000.0,
                   r_min=2.0, r_max=30.0)
    with pytest.raises(RuntimeError):
        ora.propagate(s, [0.01], [0.0], [0], flags=ora.F_DECOUPLED)


# ------------------------------------------------------------------ adaptive step control
def _adapt_sys(ora, adapt, jmax=3):
    p = W.diatom_pes_params(jmax=jmax, n_grid=200)
    return ora.diatom_system(jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, 200, p.r_min, p.r_max, adapt=adapt), p


def test_adaptive_limits_are_fixed_half_steps(ora):
    """Step doubling keeps the two-half-step result: with a tolerance no step can meet, every step is
    the smallest (dt) and the run equals fixed steps of dt/2; with a tolerance every step meets, every
    step is the largest (16 dt) and the run equals fixed steps of 8 dt -- bit for bit."""
    e, b = W.cm([900.0]), [2.0]
    s_tiny, _ = _adapt_sys(ora, (1e-300, 16))
    s_huge, _ = _adapt_sys(ora, (1e300, 16))
    s_fix, _ = _adapt_sys(ora, None)
    a1, r1 = ora.propagate(s_tiny, e, b, [1], dt=4.0, max_steps=300, flags=ora.F_NO_STOP)
    a2, r2 = ora.propagate(s_fix, e, b, [1], dt=2.0, max_steps=600, flags=ora.F_NO_STOP)
    assert np.array_equal(a1, a2) and r1["R"][0] == r2["R"][0] and r1["t_final"][0] == r2["t_final"][0]
    a3, r3 = ora.propagate(s_huge, e, b, [1], dt=4.0, max_steps=40, flags=ora.F_NO_STOP)
    a4, r4 = ora.propagate(s_fix, e, b, [1], dt=32.0, max_steps=80, flags=ora.F_NO_STOP)
    assert np.array_equal(a3, a4) and r3["R"][0] == r4["R"][0] and r3["t_final"][0] == 40 * 64.0


def test_adaptive_error_follows_tolerance(ora):
    """Against a fixed-step run at dt = 0.5 (converged): the level populations (summed over m, which
    the frame rotation beyond r_end does not change) of adaptive runs stay within 1e-6 and get no
    worse with a tighter tolerance, while the adaptive runs take over ten times fewer steps than fixed
    dt = 5 -- large steps where the coupling is weak -- and more with a tighter tolerance."""
    e, b, s0 = W.cm([300.0, 1500.0]), [1.0, 4.0], [0, 4]
    ref_sys, _ = _adapt_sys(ora, None)
    lev = lambda a: np.stack([np.bincount(ref_sys.level, weights=np.abs(x) ** 2) for x in a])
    aref, _ = ora.propagate(ref_sys, e, b, s0, dt=0.5)
    _, rfix = ora.propagate(ref_sys, e, b, s0, dt=5.0)
    errs, steps = [], []
    for tol in (1e-4, 1e-8):
        s, _ = _adapt_sys(ora, (tol, 16))
        a, r = ora.propagate(s, e, b, s0, dt=5.0)
        assert np.all(r["status"] == 0)
        errs.append(np.max(np.abs(lev(a) - lev(aref))))
        steps.append(r["steps"].sum())
    assert errs[0] < 1e-6 and errs[1] <= errs[0]
    assert steps[0] < 0.1 * rfix["steps"].sum() and steps[1] >= steps[0]
