"""Pins of the oracle's asymmetric top + linear rotor coupling (Eqs. 3, 13-17) against the direct
angular quadrature of Eq. 11 -- the paper's own check of its CG algebra (Sec. II: the two agree to
~1e-10 cm^-1).  The quadrature here builds the states of Eq. 3 and the angular functions of Eq. 13
from Wigner's explicit d-matrix formula and sympy's exact Clebsch-Gordan coefficients, so it shares
no step with the oracle's Racah-formula algebra.  CPU only."""
import math

import numpy as np
import pytest

sympy_wigner = pytest.importorskip("sympy.physics.wigner")


@pytest.fixture(scope="module")
def ora():
    import oracle

    return oracle


def wigner_d(j, mp, m, beta):
    """d^j_{m' m}(beta) by Wigner's explicit sum."""
    beta = np.asarray(beta, np.float64)
    c, s = np.cos(beta / 2), np.sin(beta / 2)
    f = math.factorial
    pre = math.sqrt(f(j + mp) * f(j - mp) * f(j + m) * f(j - m))
    out = np.zeros_like(beta)
    for k in range(max(0, m - mp), min(j + m, j - mp) + 1):
        num = (-1) ** (mp - m + k)
        den = f(j + m - k) * f(k) * f(mp - m + k) * f(j - mp - k)
        out += num / den * c ** (2 * j + m - mp - 2 * k) * s ** (mp - m + 2 * k)
    return pre * out


def cg(j1, m1, j2, m2, J, M):
    if m1 + m2 != M or abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    return float(sympy_wigner.clebsch_gordan(j1, j2, J, m1, m2, M))


def Dstar(j, m, k, al, be, ga):
    """D^{j*}_{m k}(alpha, beta, gamma) = e^{i m alpha} d^j_{m k}(beta) e^{i k gamma}."""
    return np.exp(1j * m * al) * wigner_d(j, m, k, be) * np.exp(1j * k * ga)


def Y(l, m, be, al):
    """Y^l_m(beta, alpha) = sqrt((2l+1)/4pi) D^{l*}_{m 0}(alpha, beta, 0)."""
    return math.sqrt((2 * l + 1) / (4 * math.pi)) * np.exp(1j * m * al) * wigner_d(l, m, 0, be)


def test_molmol_coupling_matches_angular_quadrature(ora):
    # water-like top, levels J <= 1; rotor j2 in {0, 1}
    A, B, Cc = 27.88, 14.51, 9.28
    lev_J, lev_E, lev_b = [], [], []
    for J in (0, 1):
        E, b = ora.asym_levels(J, A, B, Cc)
        for e_, bb in zip(E, b):
            lev_J.append(J)
            lev_E.append(e_)
            row = np.zeros(3)
            row[1 - J:1 + J + 1] = bb
            lev_b.append(row)
    lev_J = np.array(lev_J, np.int32)
    lev_b = np.array(lev_b)
    jmax1 = 1
    e, lev, jt, mt, l1, j2 = ora.molmol_states(lev_J, [0, 1], lev_E, 60.0)
    n = len(e)
    assert n == 40
    # quadrature grids: trapezoid in the three azimuths (exact for the frequencies present), Gauss-Legendre in cos beta
    na, nb = 12, 8
    az = 2 * np.pi * np.arange(na) / na
    xb, wb = np.polynomial.legendre.leggauss(nb)
    be = np.arccos(xb)
    a1, b1, g1, b2, a2 = np.meshgrid(az, be, az, be, az, indexing="ij")
    w = (np.ones(na)[:, None, None, None, None] * wb[None, :, None, None, None] * np.ones(na)[None, None, :, None, None]
         * wb[None, None, None, :, None] * np.ones(na)[None, None, None, None, :]) * (2 * np.pi / na) ** 3
    shape = a1.shape
    # the states of Eq. 3
    psi = np.zeros((n,) + shape, complex)
    for s in range(n):
        J = int(lev_J[l1[s]])
        for m1 in range(-J, J + 1):
            m2 = int(mt[s]) - m1
            c = cg(J, m1, int(j2[s]), m2, int(jt[s]), int(mt[s]))
            if c == 0.0:
                continue
            top = sum(lev_b[l1[s]][k + jmax1] * Dstar(J, m1, k, a1, b1, g1) for k in range(-J, J + 1))
            psi[s] += c * math.sqrt((2 * J + 1) / (8 * math.pi ** 2)) * top * Y(int(j2[s]), m2, b2, a2)
    flat = psi.reshape(n, -1)
    wf = w.reshape(-1)
    # orthonormality of the composite states (checks the quadrature itself)
    ov = (flat.conj() * wf) @ flat.T
    assert np.max(np.abs(ov - np.eye(n))) < 1e-12
    for (lam1, mu1, lam2, lam) in [(1, 0, 0, 1), (1, 1, 1, 0), (1, 1, 1, 2), (2, 2, 1, 1), (2, 0, 2, 0), (2, 1, 1, 2)]:
        sgn = (-1) ** (lam1 + mu1 + lam2 + lam)
        tau = np.zeros(shape, complex)
        for eta in range(-min(lam1, lam2), min(lam1, lam2) + 1):
            c = cg(lam1, eta, lam2, -eta, lam, 0)
            if c == 0.0:
                continue
            tau += c * (Dstar(lam1, eta, mu1, a1, b1, g1) + sgn * Dstar(lam1, eta, -mu1, a1, b1, g1)) * Y(lam2, -eta, b2, a2)
        tau *= math.sqrt((2 * lam1 + 1) / (4 * math.pi))
        tf = tau.reshape(-1)
        Gq = (flat.conj() * (wf * tf)) @ flat.T
        Go = ora.molmol_G(lev_J, lev_b, jmax1, l1, j2, jt, mt, lam1, mu1, lam2, lam)
        assert np.max(np.abs(Gq.imag)) < 1e-12, (lam1, mu1, lam2, lam)
        assert np.max(np.abs(Gq.real - Go)) < 1e-12, (lam1, mu1, lam2, lam)
        assert np.max(np.abs(Go)) > 1e-3
        assert np.allclose(Go, Go.T, atol=1e-14)
        assert not np.any((Go != 0) & (mt[:, None] != mt[None, :]))


def test_molmol_coupling_quadrature_at_bench_size(ora):
    """The same check at the size the benchmark runs: water-like top with J <= 2 and para-H2
    j2 in {0, 2} (N = 210 composite states), four PES terms including lambda2 = 2.  Azimuthal
    frequencies reach 6 and the polar integrands are polynomials of degree <= 6 in cos(beta), so an
    8-point trapezoid rule per azimuth and 8 Gauss-Legendre nodes per polar angle are exact."""
    import paper_2312_02322_gb300.inputs as W

    p = W.molmol_params(j1max=2, j2=(0, 2))
    jmax1 = p.j1max
    lev_J, lev_E, lev_b = [], [], []
    for J in range(jmax1 + 1):
        E, b = ora.asym_levels(J, p.A, p.B, p.C)
        for e_, bb in zip(E, b):
            row = np.zeros(2 * jmax1 + 1)
            row[jmax1 - J:jmax1 + J + 1] = bb
            lev_J.append(J); lev_E.append(e_); lev_b.append(row)
    lev_J = np.array(lev_J, np.int32)
    lev_b = np.array(lev_b)
    e, lev, jt, mt, l1, j2 = ora.molmol_states(lev_J, list(p.j2), lev_E, p.bconst2)
    n = len(e)
    assert n == 210
    na, nb = 8, 8
    az = 2 * np.pi * np.arange(na) / na
    xb, wb = np.polynomial.legendre.leggauss(nb)
    be = np.arccos(xb)
    a1, b1, g1, b2, a2 = np.meshgrid(az, be, az, be, az, indexing="ij")
    w = (wb[None, :, None, None, None] * wb[None, None, None, :, None] * np.ones(a1.shape)) * (2 * np.pi / na) ** 3
    shape = a1.shape
    dcache, ycache = {}, {}

    def D(j, m, k):
        if (j, m, k) not in dcache:
            dcache[(j, m, k)] = Dstar(j, m, k, a1, b1, g1)
        return dcache[(j, m, k)]

    def Yc(l, m):
        if (l, m) not in ycache:
            ycache[(l, m)] = Y(l, m, b2, a2)
        return ycache[(l, m)]

    psi = np.zeros((n,) + shape, complex)
    for s in range(n):
        J = int(lev_J[l1[s]])
        for m1 in range(-J, J + 1):
            m2 = int(mt[s]) - m1
            c = cg(J, m1, int(j2[s]), m2, int(jt[s]), int(mt[s]))
            if c == 0.0:
                continue
            top = sum(lev_b[l1[s]][k + jmax1] * D(J, m1, k) for k in range(-J, J + 1))
            psi[s] += c * math.sqrt((2 * J + 1) / (8 * math.pi ** 2)) * top * Yc(int(j2[s]), m2)
    flat = psi.reshape(n, -1)
    wf = w.reshape(-1)
    ov = (flat.conj() * wf) @ flat.T
    assert np.max(np.abs(ov - np.eye(n))) < 1e-12
    terms = [t for t in p.terms if t[2] == 2][:3] + [t for t in p.terms if t[2] == 0 and t[0] > 0][:1]
    assert len(terms) == 4
    for (lam1, mu1, lam2, lam) in terms:
        sgn = (-1) ** (lam1 + mu1 + lam2 + lam)
        tau = np.zeros(shape, complex)
        for eta in range(-min(lam1, lam2), min(lam1, lam2) + 1):
            c = cg(lam1, eta, lam2, -eta, lam, 0)
            if c == 0.0:
                continue
            tau += c * (D(lam1, eta, mu1) + sgn * D(lam1, eta, -mu1)) * Yc(lam2, -eta)
        tau *= math.sqrt((2 * lam1 + 1) / (4 * math.pi))
        Gq = (flat.conj() * (wf * tau.reshape(-1))) @ flat.T
        Go = ora.molmol_G(lev_J, lev_b, jmax1, l1, j2, jt, mt, lam1, mu1, lam2, lam)
        assert np.max(np.abs(Gq.imag)) < 1e-12, (lam1, mu1, lam2, lam)
        assert np.max(np.abs(Gq.real - Go)) < 1e-12, (lam1, mu1, lam2, lam)
        assert np.max(np.abs(Go)) > 1e-3
