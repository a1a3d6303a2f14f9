"""Oracle of the post-processing step: symmetrised cross sections and Maxwell-Boltzmann
rate coefficients (arXiv 2312.02322, Sec. III, Eq. 19 and Eq. 20).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the CPU-baseline leg of ``bench.py``.
The CUDA library never imports it.  Plain numpy / scipy in FP64, one pair of levels and one
temperature at a time, with adaptive quadrature for the integrals.

What the paper fixes (Sec. III):
  * Eq. 20: sigma~_{n'n''}(U) = [g' sigma_{n'->n''}(U) + g'' sigma_{n''->n'}(U)] / 2 with the
    rotational degeneracies g = (2j_1+1)(2j_2+1) of Eq. 19 (2j+1 for an atom + rotor);
  * the rate coefficients of both directions come from integrating sigma~ over the
    Maxwell-Boltzmann distribution of collision energies, after a cubic spline of sigma~
    through the computed energies, extrapolated to zero at the excitation threshold and
    continued towards high energies.

Readings where the paper defers to its ref. [44]:
  R1 (energy variable)  U, the energy at which both directions are compared in Eq. 19, is the
     mean of the incoming and outgoing translational energies, so the incoming energy of
     n'->n'' is U + dE/2 with dE = E'' - E'.
  R2 (rates)  k_{n'->n''}(T) = (8/(pi mu))^(1/2) (kT)^(-3/2) exp(-dE/(2kT)) / g'
                                * int_{u0}^inf sigma~(U) U exp(-U/kT) dU,
     i.e. the textbook <v sigma> over the incoming energy with the flux factor E sigma(E) of
     one direction replaced by U sigma~(U)/g'.  Both directions then obey
     g' k_{n'->n''} = g'' k_{n''->n'} exp(-dE/kT) exactly.
  R3 (spline)  natural cubic spline of sigma~ in U through the computed energies U_1 < ... < U_K;
     negative spline values are taken as zero (a cross section is not negative).
  R4 (threshold)  u0 = |dE| / 2 (outgoing energy zero under R1).  Below U_1, sigma~ falls
     linearly to zero at u0 when u0 < U_1; when u0 >= U_1 the spline is cut at u0.  Elastic
     pairs (dE = 0) have u0 = 0.
  R5 (high energies)  above U_K, sigma~(U) = sigma~_K (U/U_K)^p with p the log-log slope of the
     last two points, clipped to [-1, 0] (0 when either point is not positive).

All quantities in atomic units: energies and kT in hartree, mu in electron masses, sigma in
bohr^2, rates in bohr^3 per atomic unit of time.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, interpolate, special


def sigma_sym(sigma: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Eq. 20 for every pair of levels: sigma[k][a][b] = sigma_{a->b}(U_k); g[a] degeneracy."""
    sigma = np.asarray(sigma, np.float64)
    g = np.asarray(g, np.float64)
    gs = g[None, :, None] * sigma
    return 0.5 * (gs + np.transpose(gs, (0, 2, 1)))


def natural_spline(u: np.ndarray, y: np.ndarray):
    """R3: the natural cubic spline (zero second derivative at both ends) through (u_k, y_k)."""
    return interpolate.CubicSpline(np.asarray(u, np.float64), np.asarray(y, np.float64), bc_type="natural")


def tail_exponent(u: np.ndarray, y: np.ndarray) -> float:
    """R5: log-log slope of the last two points, clipped to [-1, 0]."""
    if y[-1] <= 0.0 or y[-2] <= 0.0:
        return 0.0
    p = np.log(y[-1] / y[-2]) / np.log(u[-1] / u[-2])
    return float(min(0.0, max(-1.0, p)))


def flux_integral(u, y, u0: float, kT: float) -> float:
    """int_{u0}^inf sigma~(U) U exp(-U/kT) dU for the piecewise sigma~ of R3-R5."""
    u = np.asarray(u, np.float64)
    y = np.asarray(y, np.float64)
    K = len(u)
    sp = natural_spline(u, y)
    total = 0.0
    opts = dict(epsabs=0.0, epsrel=1e-13, limit=400)
    # R4: linear ramp from zero at u0 up to the first computed energy
    if u0 < u[0]:
        f = lambda U: y[0] * (U - u0) / (u[0] - u0) * U * np.exp(-U / kT)
        total += integrate.quad(f, u0, u[0], **opts)[0]
    # R3: spline pieces above max(u0, U_k)
    for k in range(K - 1):
        a, b = max(u[k], u0), u[k + 1]
        if b <= a:
            continue
        f = lambda U: max(0.0, float(sp(U))) * U * np.exp(-U / kT)
        total += integrate.quad(f, a, b, **opts)[0]
    # R5: power-law tail, integrated in closed form with the upper incomplete gamma function:
    #   int_a^inf (U/U_K)^p U exp(-U/kT) dU = U_K^-p kT^(2+p) Gamma(2+p, a/kT)
    p = tail_exponent(u, y)
    a = max(u[-1], u0)
    s = 2.0 + p
    upper = special.gammaincc(s, a / kT) * special.gamma(s)
    total += y[-1] * u[-1] ** (-p) * kT ** s * upper
    return total


def rate_pair(u, y, e_from: float, e_to: float, g_from: float, mu: float, kT: float) -> float:
    """R2: k_{from->to}(T) from the symmetrised sigma~ values y on the grid u."""
    dE = e_to - e_from
    u0 = 0.5 * abs(dE)
    I = flux_integral(u, y, u0, kT)
    return np.sqrt(8.0 / (np.pi * mu)) * kT ** -1.5 * np.exp(-dE / (2.0 * kT)) / g_from * I


def rates(sigma, u, energy, g, mu: float, kT, pairs=None):
    """k[t][a][b] = k_{a->b}(T_t) for every ordered pair (or only the listed (a, b) pairs,
    the other entries left NaN); sigma[k][a][b] = sigma_{a->b}(U_k)."""
    st = sigma_sym(sigma, g)
    L = st.shape[1]
    kT = np.atleast_1d(np.asarray(kT, np.float64))
    out = np.full((len(kT), L, L), np.nan)
    todo = [(a, b) for a in range(L) for b in range(L)] if pairs is None else list(pairs)
    for (a, b) in todo:
        for t, th in enumerate(kT):
            out[t, a, b] = rate_pair(u, st[:, a, b], energy[a], energy[b], g[a], mu, th)
    return out
