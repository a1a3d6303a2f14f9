"""Independent references used to pin the oracle (test-side only).

Nothing here calls the oracle or the CUDA library: coupling matrices come from
Gauss-Legendre quadrature of scipy's spherical harmonics, classical motion from
scipy's adaptive ODE solver, closed forms from textbook formulas.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad, solve_ivp
from scipy.special import eval_legendre, sph_harm_y


def g_quadrature(jmax: int, lam: int, nq: int = 96) -> np.ndarray:
    """<j'' m | P_lambda(cos theta) | j' m> = 2 pi int Y*_{j''m} P_lambda Y_{j'm} sin(theta) dtheta,
    by Gauss-Legendre quadrature in x = cos(theta); j-major state order s = j^2 + j + m."""
    x, w = np.polynomial.legendre.leggauss(nq)
    theta = np.arccos(x)
    n = (jmax + 1) ** 2
    Y = np.zeros((n, nq))
    for j in range(jmax + 1):
        for m in range(-j, j + 1):
            Y[j * j + j + m] = np.real(sph_harm_y(j, m, theta, 0.0) * 1.0)
    P = eval_legendre(lam, x)
    G = np.zeros((n, n))
    for j2 in range(jmax + 1):
        for j1 in range(jmax + 1):
            for m in range(-min(j1, j2), min(j1, j2) + 1):
                r, c = j2 * j2 + j2 + m, j1 * j1 + j1 + m
                G[r, c] = 2.0 * np.pi * np.sum(w * Y[r] * P * Y[c])
    return G


def cg_j2_one(j1: int, m1: int, m2: int, J: int) -> float:
    """Textbook closed forms of <j1 m1, 1 m2 | J M> (Condon-Shortley phase), M = m1 + m2."""
    M = m1 + m2
    if J == j1 + 1:
        if m2 == 1:
            return np.sqrt((j1 + M) * (j1 + M + 1) / ((2 * j1 + 1) * (2 * j1 + 2)))
        if m2 == 0:
            return np.sqrt((j1 - M + 1) * (j1 + M + 1) / ((2 * j1 + 1) * (j1 + 1)))
        return np.sqrt((j1 - M) * (j1 - M + 1) / ((2 * j1 + 1) * (2 * j1 + 2)))
    if J == j1:
        if m2 == 1:
            return -np.sqrt((j1 + M) * (j1 - M + 1) / (2 * j1 * (j1 + 1)))
        if m2 == 0:
            return M / np.sqrt(j1 * (j1 + 1))
        return np.sqrt((j1 - M) * (j1 + M + 1) / (2 * j1 * (j1 + 1)))
    if J == j1 - 1:
        if m2 == 1:
            return np.sqrt((j1 - M) * (j1 - M + 1) / (2 * j1 * (2 * j1 + 1)))
        if m2 == 0:
            return -np.sqrt((j1 - M) * (j1 + M) / (j1 * (2 * j1 + 1)))
        return np.sqrt((j1 + M + 1) * (j1 + M) / (2 * j1 * (2 * j1 + 1)))
    return 0.0


def pes_terms(A, beta, c6, rd):
    """Analytic v_lambda(R) and dv_lambda/dR of the synthetic PES (lambda = 0 carries the C6 tail)."""

    def v(l, R):
        val = A[l] * np.exp(-beta[l] * R)
        if l == 0:
            val = val - c6 * R ** -6 * (1.0 - np.exp(-(R / rd) ** 6))
        return val

    def dv(l, R):
        d = -beta[l] * A[l] * np.exp(-beta[l] * R)
        if l == 0:
            u = (R / rd) ** 6
            d = d + 6 * c6 * R ** -7 * (1 - np.exp(-u)) - c6 * R ** -6 * np.exp(-u) * 6 * u / R
        return d

    return v, dv


def radial_motion(vfun, dvfun, mu, r0, e_coll, t_end, t_eval=None):
    """Head-on (b = 0) classical motion in the potential vfun, started inbound at r0 with the
    kinetic energy e_coll - vfun(r0); adaptive RK (DOP853) to tight tolerance."""
    p0 = -np.sqrt(2.0 * mu * (e_coll - vfun(r0)))

    def f(t, y):
        return [y[1] / mu, -dvfun(y[0])]

    sol = solve_ivp(f, (0.0, t_end), [r0, p0], method="DOP853", rtol=1e-12, atol=1e-12, dense_output=True,
                    t_eval=t_eval)
    return sol


def integrate_on(sol, g, t_end, pieces=400):
    """int_0^t_end g(R(t), t) dt with adaptive quadrature over short pieces (complex g allowed)."""
    edges = np.linspace(0.0, t_end, pieces + 1)
    tot = 0.0 + 0.0j
    for a, b in zip(edges[:-1], edges[1:]):
        re = quad(lambda t: np.real(g(sol.sol(t)[0], t)), a, b, epsabs=1e-15, epsrel=1e-12, limit=200)[0]
        im = quad(lambda t: np.imag(g(sol.sol(t)[0], t)), a, b, epsabs=1e-15, epsrel=1e-12, limit=200)[0]
        tot += re + 1j * im
    return tot


def wigner_d1(beta: float) -> np.ndarray:
    """Textbook d^1_{m' m}(beta), rows/cols ordered m = -1, 0, 1."""
    c, s = np.cos(beta), np.sin(beta)
    r2 = np.sqrt(2.0)
    # d^1_{1,1}=(1+c)/2, d^1_{1,0}=-s/r2, d^1_{1,-1}=(1-c)/2, d^1_{0,0}=c
    d = np.array([
        [(1 + c) / 2, s / r2, (1 - c) / 2],    # m' = -1
        [-s / r2, c, s / r2],                  # m' = 0
        [(1 - c) / 2, -s / r2, (1 + c) / 2],   # m' = 1
    ])
    return d
