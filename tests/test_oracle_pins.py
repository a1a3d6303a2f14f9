"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a different part of the oracle so that a plausible mistake
(a dropped term, a wrong sign, a transposed operand, a wrong factor) fails one:
  CG coefficients        textbook closed forms, orthogonality              (Eq. 3, 15)
  G^lambda               Gauss-Legendre quadrature of Y* P_lambda Y        (Eq. 11 vs Eq. 12-15 check, Sec. II)
  spline                 cubic reproduction, O(h^4), knot interpolation    (Sec. III)
  Coriolis term          free rotor seen from the rotating frame: d^1(Phi) (Eq. 5)
  potential coupling     two-level Rabi formula; sudden limit exp(-i theta G) (Eq. 5, 12)
  first order            perturbative limit along the isotropic trajectory (Eq. 5)
  classical motion       free straight line                                 (Eqs. 7-9)
  conservation           norm, total energy, P_Phi + <J_y>                  (Sec. II; Eq. 10 reading)
  symmetries             J_y sign convention, m -> -m reflection, detailed balance (Eq. 19)
  tangent                central finite differences of the oracle itself
"""
import numpy as np
import pytest

from paper_2312_02322_gb300 import inputs as W
from tests import _refs


def idx(j, m):
    return j * j + j + m


# --------------------------------------------------------------------------- CG / G
def test_cg_textbook_j2_one(ora):
    for j1 in range(1, 11):
        for J in (j1 - 1, j1, j1 + 1):
            for m1 in range(-j1, j1 + 1):
                for m2 in (-1, 0, 1):
                    M = m1 + m2
                    if abs(M) > J:
                        continue
                    assert ora.cg(j1, m1, 1, m2, J, M) == pytest.approx(_refs.cg_j2_one(j1, m1, m2, J), abs=1e-14)


def test_cg_golden_exact_values(ora):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "cg_exact.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.lstrip().startswith("#")]
    assert len(rows) >= 10
    for r in rows:
        j1, m1, j2, m2, J, M, sg, num, den = map(int, r)
        assert ora.cg(j1, m1, j2, m2, J, M) == pytest.approx(sg * np.sqrt(num / den), abs=1e-15), r


def test_cg_special_values_and_orthogonality(ora):
    assert ora.cg(1, 0, 1, 0, 0, 0) == pytest.approx(-1 / np.sqrt(3), abs=1e-15)
    assert ora.cg(1, 1, 1, -1, 0, 0) == pytest.approx(1 / np.sqrt(3), abs=1e-15)
    assert ora.cg(1, 0, 1, 0, 2, 0) == pytest.approx(np.sqrt(2 / 3), abs=1e-15)
    assert ora.cg(2, 0, 2, 0, 4, 0) == pytest.approx(np.sqrt(18 / 35), abs=1e-15)
    # selection rules (Eq. 3): m = m1 + m2, triangle rule
    assert ora.cg(2, 1, 1, 0, 2, 0) == 0.0
    assert ora.cg(1, 0, 1, 0, 3, 0) == 0.0
    # sum_{m1, m2} C^{JM}_{j1 m1 j2 m2} C^{J'M'}_{j1 m1 j2 m2} = delta_JJ' delta_MM'
    j1, j2 = 7, 4
    for J in range(abs(j1 - j2), j1 + j2 + 1):
        for Jp in range(abs(j1 - j2), j1 + j2 + 1):
            M = min(J, Jp) - 1 if min(J, Jp) > 0 else 0
            s = sum(ora.cg(j1, m1, j2, M - m1, J, M) * ora.cg(j1, m1, j2, M - m1, Jp, M)
                    for m1 in range(-j1, j1 + 1) if abs(M - m1) <= j2)
            assert s == pytest.approx(1.0 if J == Jp else 0.0, abs=1e-13)


@pytest.mark.parametrize("lam", [0, 1, 2, 3, 4, 6])
def test_glambda_matches_quadrature(ora, lam):
    jmax = 12
    G = ora.diatom_G(jmax, lam)
    Gq = _refs.g_quadrature(jmax, lam)
    assert np.max(np.abs(G - Gq)) < 1e-13
    assert np.max(np.abs(G - G.T)) < 1e-14
    if lam == 0:
        assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-14


def test_glambda_selection_rules(ora):
    jmax = 8
    for lam in range(5):
        G = ora.diatom_G(jmax, lam)
        for j2 in range(jmax + 1):
            for j1 in range(jmax + 1):
                for m2 in range(-j2, j2 + 1):
                    for m1 in range(-j1, j1 + 1):
                        allowed = m1 == m2 and abs(j1 - j2) <= lam <= j1 + j2 and (j1 + j2 + lam) % 2 == 0
                        if not allowed:
                            assert G[idx(j2, m2), idx(j1, m1)] == 0.0


def test_glambda_large_j_quadrature(ora):
    # the largest basis of the workloads (j <= 39)
    G = ora.diatom_G(39, 4)
    Gq = _refs.g_quadrature(39, 4, nq=128)
    assert np.max(np.abs(G - Gq)) < 1e-12


# --------------------------------------------------------------------------- spline
def test_spline_reproduces_cubic(ora):
    n, r0, r1 = 40, 2.0, 30.0
    h = (r1 - r0) / (n - 1)
    R = r0 + h * np.arange(n)
    p = lambda x: 0.3 - 1.2 * x + 0.07 * x ** 2 - 0.002 * x ** 3
    dp = lambda x: -1.2 + 0.14 * x - 0.006 * x ** 2
    coef = ora.spline(p(R), h, dp(r0), dp(r1))
    Rt = np.linspace(1.5, 30.5, 997)  # includes both extrapolated ends
    f, df, d2f = ora.spline_eval(coef, n, r0, r1, Rt)
    assert np.max(np.abs(f - p(Rt))) < 1e-12
    assert np.max(np.abs(df - dp(Rt))) < 1e-12
    assert np.max(np.abs(d2f - (0.14 - 0.012 * Rt))) < 1e-11


def test_spline_fourth_order(ora):
    errs = []
    for n in (50, 100, 200):
        h = 28.0 / (n - 1)
        R = 2.0 + h * np.arange(n)
        y = np.exp(-1.8 * R)
        coef = ora.spline(y, h, -1.8 * np.exp(-3.6), -1.8 * np.exp(-54.0))
        Rt = np.linspace(2.0, 30.0, 5001)
        f, _, _ = ora.spline_eval(coef, n, 2.0, 30.0, Rt)
        errs.append(np.max(np.abs(f - np.exp(-1.8 * Rt))))
        # interpolates the knots
        fk, _, _ = ora.spline_eval(coef, n, 2.0, 30.0, R[:-1])
        assert np.max(np.abs(fk - y[:-1])) < 1e-15
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20


# --------------------------------------------------------------------------- systems
def diatom(ora, jmax=2, scale_aniso=1.0, zero=False, n_grid=200, with_params=False, A=None):
    p = W.diatom_pes_params(jmax=jmax, n_grid=n_grid)
    A = np.array(p.A if A is None else A, dtype=np.float64)
    A[1:] *= scale_aniso
    c6 = p.c6
    if zero:
        A[:] = 0.0
        c6 = 0.0
    return ora.diatom_system(jmax, p.bconst, p.mu, A, p.beta, c6, p.rd, n_grid, p.r_min, p.r_max,
                             with_params=with_params), p


def level_pop(sys, amp):
    pop = np.abs(amp) ** 2
    out = np.zeros((pop.shape[0], sys.n_levels))
    for s in range(sys.n):
        out[:, sys.level[s]] += pop[:, s]
    return out


# --------------------------------------------------------------------------- Coriolis, classical
def test_free_motion_and_coriolis_rotation(ora):
    """Zero coupling: straight-line motion; body-frame amplitudes of a free rotor rotate by the swept
    angle, |a_{m'}|^2 = |d^1_{m' m}(Phi)|^2 (Eq. 5 Coriolis term, its factor 1/2 and ladder factors)."""
    sys, p = diatom(ora, jmax=2, zero=True)
    E = float(W.cm(500.0))
    b = 5.0
    amp, res = ora.propagate(sys, [E, E], [b, b], [idx(1, 0), idx(1, 1)], r0=30.0, r_end=30.0, dt=5.0)
    v = np.sqrt(2 * E / p.mu)
    x0 = -np.sqrt(30.0 ** 2 - b ** 2)
    for i in range(2):
        T = res["t_final"][i]
        x = x0 + v * T
        assert res["R"][i] == pytest.approx(np.hypot(b, x), abs=1e-9)
        sweep = np.arctan2(x, b) - np.arctan2(x0, b)
        assert res["Phi"][i] == pytest.approx(sweep, abs=1e-9)
        assert res["PPhi"][i] == pytest.approx(b * np.sqrt(2 * p.mu * E), rel=1e-14)
        d = _refs.wigner_d1(res["Phi"][i])
        m0 = [0, 1][i]
        want = d[:, m0 + 1] ** 2
        got = np.abs(amp[i, [idx(1, -1), idx(1, 0), idx(1, 1)]]) ** 2
        assert np.max(np.abs(got - want)) < 1e-9
        assert np.abs(amp[i, idx(0, 0)]) == 0.0 and np.all(amp[i, 4:] == 0.0)
    assert np.all(res["status"] == 0)


def test_zero_coupling_j0_is_unchanged(ora):
    sys, _ = diatom(ora, jmax=3, zero=True)
    E = float(W.cm(300.0))
    amp, res = ora.propagate(sys, [E] * 3, [0.5, 4.0, 11.0], [0, 0, 0])
    e0 = np.zeros(sys.n)
    e0[0] = 1.0
    assert np.max(np.abs(amp - e0)) == 0.0
    assert np.all(res["norm_dev"] == 0.0)


# --------------------------------------------------------------------------- potential coupling
def two_level(ora, delta, vc, n_grid=8):
    G = np.zeros((2, 2, 2))
    G[1] = [[0, 1], [1, 0]]
    v = np.zeros((2, n_grid))
    v[1] = vc
    return ora.System([0.0, delta], [0, 1], [-1, -1], [0, 0], G, v, np.zeros((2, 2)), mu=7000.0, r_min=2.0,
                      r_max=30.0)


def rabi_error(ora, delta, vc, dt, steps):
    sys = two_level(ora, delta, vc)
    amp, res = ora.propagate(sys, [0.1], [0.0], [0], dt=dt, max_steps=steps, flags=ora.F_NO_STOP)
    T = res["t_final"][0]
    om = np.sqrt(delta ** 2 + 4 * vc ** 2)
    want = 4 * vc ** 2 / om ** 2 * np.sin(om * T / 2) ** 2
    return abs(abs(amp[0, 1]) ** 2 - want), res


def test_rabi_closed_form(ora):
    err, res = rabi_error(ora, 1e-3, 2e-4, 5.0, 2000)
    assert err < 1e-10
    assert res["status"][0] & ora.ST_MAX_STEPS
    assert res["status"][0] & ora.ST_TABLE_RANGE  # R ran below the grid (constant coupling, exact extrapolation)


def test_rabi_fourth_order(ora):
    e1, _ = rabi_error(ora, 0.02, 0.005, 5.0, 200)
    e2, _ = rabi_error(ora, 0.02, 0.005, 2.5, 400)
    assert 13 < e1 / e2 < 19


def test_sudden_limit_matrix_exponential(ora):
    """B = 0, b = 0, one anisotropic term: U = exp(-i int v0) exp(-i theta G^2), theta = int v2(R(t)) dt,
    R(t) the 1-D motion in v0 + <G^2> v2 (Eq. 5 potential term + Eq. 9 mean-field force)."""
    jmax, lam = 3, 2
    p = W.diatom_pes_params(jmax=jmax, n_grid=400)
    A = np.zeros(5)
    A[0], A[lam] = p.A[0], p.A[lam]
    sys = ora.diatom_system(jmax, 0.0, p.mu, A, p.beta, p.c6, p.rd, 400, p.r_min, p.r_max)
    E = float(W.cm(800.0))
    s0 = idx(1, 0)
    amp, res = ora.propagate(sys, [E], [0.0], [s0], dt=2.0)
    Gq = _refs.g_quadrature(jmax, lam)
    g = Gq[s0, s0]
    v, dv = _refs.pes_terms(A, p.beta, p.c6, p.rd)
    T = res["t_final"][0]
    sol = _refs.radial_motion(lambda R: v(0, R) + g * v(lam, R), lambda R: dv(0, R) + g * dv(lam, R), p.mu, 30.0, E,
                              T)
    theta = np.real(_refs.integrate_on(sol, lambda R, t: v(lam, R), T))
    ev, U = np.linalg.eigh(Gq)
    Ug = U @ np.diag(np.exp(-1j * theta * ev)) @ U.T
    want = np.abs(Ug[:, s0]) ** 2
    got = np.abs(amp[0]) ** 2
    assert np.max(np.abs(got - want)) < 2e-7
    # classical end point: agrees up to the O(h^4) spline error of the tabulated potential
    assert res["R"][0] == pytest.approx(sol.sol(T)[0], abs=2e-5)


def test_first_order_perturbative_limit(ora):
    """Weak anisotropy eps: P_{0->2}/eps^2 -> |int v_2(R0(t)) G^2_{20,00} exp(i w t) dt|^2 along the
    isotropic trajectory (first-order solution of Eq. 5).  The leading correction is linear in eps
    (interference with the second-order amplitude through the diagonal coupling of j = 2), so the
    limit is taken by linear extrapolation from eps = 1e-3 and 1e-4."""
    p = W.diatom_pes_params(jmax=2, n_grid=400)
    E = float(W.cm(500.0))
    v, dv = _refs.pes_terms(p.A, p.beta, p.c6, p.rd)
    g = _refs.g_quadrature(2, 2)[idx(2, 0), idx(0, 0)]
    om = p.bconst * 6.0
    rels = []
    for eps in (1e-3, 1e-4):
        sys, _ = diatom(ora, jmax=2, scale_aniso=eps, n_grid=400)
        amp, res = ora.propagate(sys, [E], [0.0], [0], dt=5.0)
        T = res["t_final"][0]
        sol = _refs.radial_motion(lambda R: v(0, R), lambda R: dv(0, R), p.mu, 30.0, E, T)
        I = _refs.integrate_on(sol, lambda R, t: v(2, R) * g * np.exp(1j * om * t), T, pieces=100)
        want = abs(I) ** 2
        got = abs(amp[0, idx(2, 0)]) ** 2 / eps ** 2
        rels.append((got - want) / want)
    assert 8 < rels[0] / rels[1] < 12
    limit = (10 * rels[1] - rels[0]) / 9
    assert abs(limit) < 1e-5


# --------------------------------------------------------------------------- conservation
def run_w1(ora, dt, bs=(1.0, 5.0, 9.0), j0=1, m0=0, flags=0):
    sys, p = diatom(ora, jmax=6)
    E = float(W.cm(500.0))
    amp, res = ora.propagate(sys, [E] * len(bs), list(bs), [idx(j0, m0)] * len(bs), dt=dt, flags=flags)
    return sys, amp, res


def test_unitarity_energy_angular_momentum(ora):
    """Sum |a|^2 = 1 to 1e-10 at dt = 5 (N = 49 workload); total energy and P_Phi + <J_y> are conserved
    up to the integrator error, which falls with dt: O(dt^4) for the norm and P_Phi + <J_y>, and at
    least O(dt^3) for the energy (the force is the derivative of a C^2 cubic spline, so RK4 loses one
    order at each knot crossing)."""
    sys, amp, r5 = run_w1(ora, 5.0, bs=(0.5, 2.0, 6.0, 10.0))
    assert np.all(r5["status"] == 0)
    assert np.max(r5["norm_dev"]) < 1e-10
    E = float(W.cm(500.0))
    assert np.max(r5["energy_dev"]) < 1e-8 * E
    _, _, r10 = run_w1(ora, 10.0, bs=(0.5, 2.0))
    re = r10["energy_dev"] / r5["energy_dev"][:2]
    rj = r10["angmom_dev"] / r5["angmom_dev"][:2]
    rn = r10["norm_dev"] / r5["norm_dev"][:2]
    assert np.all(re > 6), re
    assert np.all((rj > 12) & (rj < 20)), rj
    assert np.all((rn > 12) & (rn < 20)), rn
    # transitions actually happen in this case
    lp = level_pop(sys, amp)
    assert np.max(1 - lp[:, 1]) > 1e-3


def test_conservation_pins_catch_planted_mistakes(ora):
    """A torque with the wrong sign breaks the conservation of P_Phi + <J_y> and of the total energy;
    a Coriolis term without its factor 1/2 breaks the conservation of the total energy (it still
    commutes with J_y).  The readings of Eq. 5 and Eq. 10 are therefore fixed by the conservation
    laws (mistakes planted in the oracle, on the CPU)."""
    _, _, r = run_w1(ora, 5.0, bs=(5.0,))
    _, _, rf = run_w1(ora, 5.0, bs=(5.0,), flags=ora.F_FLIP_JY)
    _, _, rt = run_w1(ora, 5.0, bs=(5.0,), flags=ora.F_PLANT_TORQUE)
    _, _, rc = run_w1(ora, 5.0, bs=(5.0,), flags=ora.F_PLANT_CORIOLIS)
    assert rf["angmom_dev"][0] == pytest.approx(r["angmom_dev"][0], rel=1e-3)
    assert rt["angmom_dev"][0] > 1e4 * r["angmom_dev"][0]
    assert rt["energy_dev"][0] > 1e4 * r["energy_dev"][0]
    assert rc["energy_dev"][0] > 1e4 * r["energy_dev"][0]


def test_jy_sign_convention_invariance(ora):
    _, a1, _ = run_w1(ora, 5.0, bs=(3.0, 7.0), j0=2, m0=1)
    _, a2, _ = run_w1(ora, 5.0, bs=(3.0, 7.0), j0=2, m0=1, flags=ora.F_FLIP_JY)
    assert np.max(np.abs(np.abs(a1) ** 2 - np.abs(a2) ** 2)) < 1e-13


def test_m_reflection(ora):
    sys, a1, _ = run_w1(ora, 5.0, bs=(2.0, 6.0), j0=2, m0=1)
    _, a2, _ = run_w1(ora, 5.0, bs=(2.0, 6.0), j0=2, m0=-1)
    assert np.max(np.abs(level_pop(sys, a1) - level_pop(sys, a2))) < 1e-12


def test_large_impact_parameter_no_transition(ora):
    sys, p = diatom(ora, jmax=3)
    E = float(W.cm(500.0))
    amp, res = ora.propagate(sys, [E], [27.0], [0])
    assert 1.0 - abs(amp[0, 0]) ** 2 < 1e-12


def test_detailed_balance_prescribed_line(ora):
    """Eq. 19 holds exactly for a time-symmetric prescribed trajectory: g' P(l'->l'') = g'' P(l''->l').
    With stage times symmetric about the midpoint the discrete RK4 propagator keeps the symmetry, so
    the equality holds to rounding at any dt."""
    sys, p = diatom(ora, jmax=2)
    v = 1.2e-3
    b = 3.0
    viol = []
    for dt in (4.0, 2.0):
        steps = int(round(2 * 28.0 / v / dt))
        n = sys.n
        amp, res = ora.propagate(sys, [1e-3] * n, [b] * n, list(range(n)), dt=dt, max_steps=steps,
                                 flags=ora.F_PRESCRIBED, line_speed=[v] * n)
        U2 = np.abs(amp) ** 2  # U2[i, f] = |U_{f i}|^2
        S = np.zeros((3, 3))
        for i in range(n):
            for f in range(n):
                S[sys.level[i], sys.level[f]] += U2[i, f]
        assert np.max(S) > 0.05 and np.max(S - np.diag(np.diag(S))) > 1e-3
        viol.append(np.max(np.abs(S - S.T)))
    assert max(viol) < 1e-12


# --------------------------------------------------------------------------- cross sections
def test_cross_section_sum_rule(ora):
    """Regular midpoint b grid with the full m' average: sum_l'' sigma(l'->l'') = pi b_max^2 (norm 1)."""
    sys, p = diatom(ora, jmax=3, n_grid=150)
    ts = W.regular_set([600.0], [1], n_b=5, b_max=9.0, m_avg="all")
    init = [idx(j, m) for j, m in zip(ts.init_j, ts.init_m)]
    amp, res = ora.propagate(sys, ts.e_coll, ts.b, init)
    db = ts.b_max / ts.n_b
    w = 2 * np.pi * ts.b * db / (2 * ts.init_j + 1)
    sig = ora.cross_sections(sys, np.abs(amp) ** 2, w, ts.group, ts.n_groups)
    assert sig.sum() == pytest.approx(np.pi * ts.b_max ** 2, rel=1e-9)
    assert np.all(sig >= 0)


# --------------------------------------------------------------------------- tangent
def test_tangent_matches_central_differences(ora):
    jmax = 3
    p = W.diatom_pes_params(jmax=jmax, n_grid=150)
    E = float(W.cm(700.0))
    bs, init = [1.5, 4.0], [idx(0, 0), idx(1, 1)]

    def build(A, beta, with_params=False):
        return ora.diatom_system(jmax, p.bconst, p.mu, A, beta, p.c6, p.rd, 150, p.r_min, p.r_max, with_params)

    sys = build(p.A, p.beta, True)
    amp, dpop, res = ora.tangent(sys, [E, E], bs, init)
    amp2, res2 = ora.propagate(build(p.A, p.beta), [E, E], bs, init)
    assert np.max(np.abs(amp - amp2)) < 1e-13
    for k in range(10):
        th = np.concatenate([p.A, p.beta])
        h = 1e-5 * abs(th[k])
        pops = []
        steps = []
        for sgn in (1, -1):
            t2 = th.copy()
            t2[k] += sgn * h
            a, r = ora.propagate(build(t2[:5], t2[5:]), [E, E], bs, init)
            pops.append(np.abs(a) ** 2)
            steps.append(r["steps"])
        assert np.array_equal(steps[0], steps[1]) and np.array_equal(steps[0], res["steps"])
        fd = (pops[0] - pops[1]) / (2 * h)
        scale = np.max(np.abs(dpop[:, k, :]))
        assert np.max(np.abs(fd - dpop[:, k, :])) <= 1e-5 * scale + 1e-12, k
