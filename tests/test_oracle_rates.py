"""Pins of the post-processing oracle (Sec. III, Eqs. 19-20; readings R1-R5 of oracle/rates.py)
against closed forms, limits and exact identities.  CPU only."""
import math

import numpy as np
import pytest

from oracle import rates as R


def _lower_inc(n, a, b, th):
    """int_a^b U^n exp(-U/th) dU for n = 1, 2 from the antiderivatives
    -th e^{-U/th} (U + th) and -th e^{-U/th} (U^2 + 2 th U + 2 th^2)."""
    if n == 1:
        F = lambda U: -th * math.exp(-U / th) * (U + th)
    else:
        F = lambda U: -th * math.exp(-U / th) * (U * U + 2 * th * U + 2 * th * th)
    return F(b) - F(a)


def _upper1(a, th):
    return th * math.exp(-a / th) * (a + th)


def _pref(mu, th, dE, g):
    return math.sqrt(8.0 / (math.pi * mu)) * th ** -1.5 * math.exp(-dE / (2 * th)) / g


def test_eq20_symmetric_and_reduces_when_eq19_holds():
    rng = np.random.default_rng(5)
    K, L = 4, 6
    g = rng.integers(1, 9, L).astype(float)
    sig = rng.uniform(0.1, 3.0, (K, L, L))
    st = R.sigma_sym(sig, g)
    assert np.array_equal(st, np.transpose(st, (0, 2, 1)))
    # when Eq. 19 holds exactly, sigma~ is g' sigma_{n'->n''} itself
    gs = g[None, :, None] * sig
    sym = 0.5 * (gs + np.transpose(gs, (0, 2, 1)))
    exact = sym / g[None, :, None]          # sigma obeying g' s' = g'' s''
    assert np.allclose(R.sigma_sym(exact, g), g[None, :, None] * exact, rtol=1e-15, atol=0)
    # one element by hand
    a, b = 1, 4
    assert st[2, a, b] == pytest.approx(0.5 * (g[a] * sig[2, a, b] + g[b] * sig[2, b, a]), rel=1e-15)


def test_natural_spline_three_knots_by_hand():
    # equal spacing h, M0 = M2 = 0: 4h M1 = 6 (y0 - 2 y1 + y2) / h  ->  M1 = 3 (y0 - 2y1 + y2) / (2 h^2);
    # value at the middle of a piece: (y_i + y_{i+1})/2 - h^2 (M_i + M_{i+1}) / 16
    u = np.array([1.0, 3.0, 5.0])
    y = np.array([2.0, 7.0, 1.0])
    h = 2.0
    M1 = 3 * (y[0] - 2 * y[1] + y[2]) / (2 * h * h)
    sp = R.natural_spline(u, y)
    assert float(sp(2.0)) == pytest.approx(0.5 * (y[0] + y[1]) - h * h * M1 / 16, rel=1e-14)
    assert float(sp(4.0)) == pytest.approx(0.5 * (y[1] + y[2]) - h * h * M1 / 16, rel=1e-14)
    assert float(sp(1.0, 2)) == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("th", [2e-5, 3e-4, 4e-3])
def test_constant_sigma_elastic_closed_form(th):
    # dE = 0: u0 = 0, ramp 0 -> c on [0, U_1], constant c above (tail p = 0)
    u = np.array([1e-4, 4e-4, 1e-3, 5e-3, 2e-2])
    c, mu, g = 3.7, 1800.0, 5.0
    y = np.full(len(u), c)
    I = c / u[0] * _lower_inc(2, 0.0, u[0], th) + c * _upper1(u[0], th)
    assert R.flux_integral(u, y, 0.0, th) == pytest.approx(I, rel=1e-12)
    k = R.rate_pair(u, y, 0.01, 0.01, g, mu, th)
    assert k == pytest.approx(_pref(mu, th, 0.0, g) * I, rel=1e-12)


def test_constant_sigma_high_temperature_is_mean_speed_times_sigma():
    # ramp negligible when U_1 << kT: k -> sqrt(8 kT / (pi mu)) sigma / g
    u = np.array([1e-9, 1e-8, 1e-7])
    c, mu, g, th = 2.0, 1000.0, 3.0, 1e-3
    k = R.rate_pair(u, np.full(3, c), 0.0, 0.0, g, mu, th)
    assert k == pytest.approx(math.sqrt(8 * th / (math.pi * mu)) * c / g, rel=1e-5)


def test_linear_sigma_inelastic_closed_form():
    # the natural spline reproduces linear data; the tail slope of increasing data clips to p = 0
    u = np.array([2e-4, 6e-4, 1.5e-3, 4e-3])
    al, be = 0.5, 900.0
    y = al + be * u
    dE, th, mu, ga, gb = 1.2e-4, 8e-4, 2500.0, 3.0, 7.0
    u0 = dE / 2
    I = (y[0] / (u[0] - u0)) * (_lower_inc(2, u0, u[0], th) - u0 * _lower_inc(1, u0, u[0], th))
    I += al * _lower_inc(1, u[0], u[-1], th) + be * _lower_inc(2, u[0], u[-1], th)
    I += y[-1] * _upper1(u[-1], th)
    assert R.flux_integral(u, y, u0, th) == pytest.approx(I, rel=1e-11)
    assert R.rate_pair(u, y, 0.0, dE, ga, mu, th) == pytest.approx(_pref(mu, th, dE, ga) * I, rel=1e-11)
    assert R.rate_pair(u, y, dE, 0.0, gb, mu, th) == pytest.approx(_pref(mu, th, -dE, gb) * I, rel=1e-11)


def test_threshold_above_first_energy_cuts_the_spline():
    u = np.array([1e-4, 3e-4, 9e-4])
    c, th = 1.5, 2e-4
    for u0 in (2e-4, 5e-4, 2e-3):   # inside the first piece, the second, and above U_K
        assert R.flux_integral(u, np.full(3, c), u0, th) == pytest.approx(c * _upper1(u0, th), rel=1e-12)


@pytest.mark.parametrize("p", [-1.0, -0.5])
def test_power_law_tail_closed_form(p):
    # two points: the natural spline is the straight line between them; the tail follows
    # (U/U_2)^p with Gamma(1, x) = e^-x and Gamma(3/2, x) = sqrt(pi) erfc(sqrt x)/2 + sqrt(x) e^-x
    u = np.array([3e-4, 1.2e-3])
    y = np.array([4.0, 4.0 * (u[1] / u[0]) ** p])
    th, u0 = 5e-4, 1e-4
    I = (y[0] / (u[0] - u0)) * (_lower_inc(2, u0, u[0], th) - u0 * _lower_inc(1, u0, u[0], th))
    sl = (y[1] - y[0]) / (u[1] - u[0])
    I += (y[0] - sl * u[0]) * _lower_inc(1, u[0], u[1], th) + sl * _lower_inc(2, u[0], u[1], th)
    x = u[1] / th
    s = 2 + p
    G = math.exp(-x) if p == -1.0 else 0.5 * math.sqrt(math.pi) * math.erfc(math.sqrt(x)) + math.sqrt(x) * math.exp(-x)
    I += y[1] * u[1] ** (-p) * th ** s * G
    assert R.tail_exponent(u, y) == pytest.approx(p, abs=1e-14)
    assert R.flux_integral(u, y, u0, th) == pytest.approx(I, rel=1e-11)


def test_tail_exponent_clipping():
    u = np.array([1.0, 2.0])
    assert R.tail_exponent(u, np.array([1.0, 3.0])) == 0.0        # growing -> 0
    assert R.tail_exponent(u, np.array([1.0, 0.01])) == -1.0      # steeper than 1/U -> -1
    assert R.tail_exponent(u, np.array([0.0, 1.0])) == 0.0        # non-positive point -> 0


def test_detailed_balance_of_rates_is_exact():
    rng = np.random.default_rng(11)
    K, L = 5, 4
    u = np.sort(rng.uniform(1e-4, 3e-2, K))
    g = np.array([1.0, 3.0, 5.0, 7.0])
    E = np.array([0.0, 2e-4, 7e-4, 1.5e-3])
    sig = rng.uniform(0.2, 5.0, (K, L, L))
    kT = np.array([3e-4, 1.5e-3])
    k = R.rates(sig, u, E, g, 1500.0, kT)
    for t, th in enumerate(kT):
        for a in range(L):
            for b in range(L):
                lhs = g[a] * k[t, a, b]
                rhs = g[b] * k[t, b, a] * math.exp(-(E[b] - E[a]) / th)
                assert lhs == pytest.approx(rhs, rel=1e-13)


def test_planted_mistakes_fail_a_pin():
    # dividing by the final degeneracy, or dropping the flux factor U, breaks the closed form
    u = np.array([1e-4, 4e-4, 1e-3])
    c, mu, th, ga, gb = 3.0, 1800.0, 3e-4, 3.0, 5.0
    y = np.full(3, c)
    I = c / u[0] * _lower_inc(2, 0.0, u[0], th) + c * _upper1(u[0], th)
    good = _pref(mu, th, 0.0, ga) * I
    assert R.rate_pair(u, y, 0.0, 0.0, ga, mu, th) == pytest.approx(good, rel=1e-12)
    wrong_g = _pref(mu, th, 0.0, gb) * I
    assert abs(wrong_g - good) > 1e-3 * good
    I_noflux = c / u[0] * _lower_inc(1, 0.0, u[0], th) + c * th * math.exp(-u[0] / th)
    assert abs(_pref(mu, th, 0.0, ga) * I_noflux - good) > 1e-3 * good
