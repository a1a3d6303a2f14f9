"""Pins of the oracle's decoupled classical motion (the AT-MQCT decoupling of Sec. III, in the
reading of the design notes: R and Phi move in the isotropic potential v_0 alone, with no torque,
and the amplitudes follow Eq. 5 along that path).  CPU only."""
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
