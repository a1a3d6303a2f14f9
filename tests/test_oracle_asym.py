"""Pins of the oracle's asymmetric-top system (Eq. 1 basis, Eq. 16 coupling) against facts
fixed outside the oracle: textbook closed-form rotor energies, the symmetric-top limits,
the symmetry classes of Wang's functions, a direct numerical integral of the Wigner-D
wavefunctions (no Clebsch-Gordan algebra), and the linear-rotor limit of Eq. 15."""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2312_02322_gb300 import inputs

H2O = (27.88, 14.51, 9.28)   # cm^-1; the pins are unit-free
OTHER = (5.3, 2.9, 1.7)


@pytest.mark.parametrize("abc", [H2O, OTHER])
def test_energies_j1_j2_closed_forms(abc):
    # textbook rigid-rotor levels: J = 1: B+C, A+C, A+B; J = 2: A+B+4C, A+4B+C, 4A+B+C and
    # 2(A+B+C) -+ 2 sqrt((B-C)^2 + (A-C)(A-B))
    A, B, C = abc
    E1, _ = oracle.asym_levels(1, A, B, C)
    assert np.allclose(E1, sorted([B + C, A + C, A + B]), rtol=0, atol=1e-12)
    E2, _ = oracle.asym_levels(2, A, B, C)
    r = np.sqrt((B - C) ** 2 + (A - C) * (A - B))
    ref = sorted([A + B + 4 * C, A + 4 * B + C, 4 * A + B + C, 2 * (A + B + C) - 2 * r, 2 * (A + B + C) + 2 * r])
    assert np.allclose(E2, ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("J", [3, 6, 12])
def test_symmetric_top_limits(J):
    # prolate (B = C): E = B J(J+1) + (A-B) K^2;  oblate (A = B): E = A J(J+1) + (C-A) K^2
    Ks = np.arange(-J, J + 1)
    E, _ = oracle.asym_levels(J, 7.0, 3.0, 3.0)
    assert np.allclose(E, np.sort(3.0 * J * (J + 1) + 4.0 * Ks ** 2), rtol=1e-13, atol=1e-11)
    E, _ = oracle.asym_levels(J, 7.0, 7.0, 3.0)
    assert np.allclose(E, np.sort(7.0 * J * (J + 1) - 4.0 * Ks ** 2), rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("J", [1, 4, 9, 12])
def test_eigenvectors_orthonormal_and_in_one_wang_class(J):
    E, b = oracle.asym_levels(J, *H2O)
    n = 2 * J + 1
    assert np.abs(b @ b.T - np.eye(n)).max() < 1e-13
    K = np.arange(-J, J + 1)
    classes = []
    for e in range(n):
        v = b[e]
        par = {int(k) % 2 for k in K[np.abs(v) > 1e-12]}
        assert len(par) == 1                                    # one K parity
        big = np.abs(v[K > 0]) > 1e-12
        if big.any():
            sign = np.sign(v[::-1][K > 0][big] * v[K > 0][big])
            assert np.all(sign == sign[0])                       # b_{-K} = +- b_K for every K
            classes.append((par.pop(), int(sign[0])))
        else:
            classes.append((0, 1))
    # the even-K, b_{-K} = +b_K class has one function per K = 0, 2, 4, ... <= J
    even_p = sum(1 for c in classes if c == (0, 1))
    assert even_p == J // 2 + 1


def _wigner_d(J, beta):
    """d^J(beta) = expm(-i beta J_y) from the angular-momentum matrices (index M + J); then
    D^J_{M'M}(alpha, beta, gamma) = exp(-i M' alpha) d^J_{M'M}(beta) exp(-i M gamma)."""
    m = np.arange(-J, J + 1)
    jp = np.zeros((2 * J + 1, 2 * J + 1))
    for k in range(2 * J):
        jp[k + 1, k] = np.sqrt(J * (J + 1) - m[k] * (m[k] + 1))
    jy = (jp - jp.T) / 2j
    return expm(-1j * beta * jy)


def _numerical_G(lev_J, lev_b, jmax, terms, nb=24, ng=24, na=8):
    """<psi'' | f_{lam mu} | psi'> by quadrature over all three Euler angles: Gauss-Legendre in
    cos(beta), uniform grids in alpha and gamma (exact for the trigonometric degrees involved)."""
    xq, wq = np.polynomial.legendre.leggauss(nb)
    gam = 2 * np.pi * np.arange(ng) / ng
    alp = 2 * np.pi * np.arange(na) / na
    states = [(l, J, M) for l, J in enumerate(lev_J) for M in range(-J, J + 1)]
    n = len(states)
    Js = sorted(set(int(j) for j in lev_J) | {l for l, _ in terms})
    d = {J: np.stack([_wigner_d(J, np.arccos(x)) for x in xq]) for J in Js}  # [q][M'][M]

    def Dconj(J, Mp, M):
        # conj(D^J_{Mp M}) on the (alpha, beta, gamma) grid
        return (np.exp(1j * Mp * alp)[:, None, None] * np.conj(d[J][:, Mp + J, M + J])[None, :, None]
                * np.exp(1j * M * gam)[None, None, :])

    psi = np.zeros((n, na, nb, ng), complex)
    for s, (l, J, M) in enumerate(states):
        for K in range(-J, J + 1):
            bk = lev_b[l][jmax + K]
            if bk != 0.0:
                psi[s] += np.sqrt((2 * J + 1) / (8 * np.pi ** 2)) * bk * Dconj(J, M, K)
    w = (2 * np.pi / na) * wq[None, :, None] * (2 * np.pi / ng)
    out = []
    for lam, mu in terms:
        f = (Dconj(lam, 0, mu) + ((-1) ** mu) * Dconj(lam, 0, -mu)) / (2.0 if mu == 0 else 1.0)
        assert np.abs(f.imag).max() < 1e-13                     # the angular function is real
        out.append(np.einsum("aijk,ijk,bijk->ab", np.conj(psi), w * f, psi, optimize=True))
    return out


def test_G_against_direct_euler_angle_quadrature():
    A, B, C = H2O
    jmax = 3
    lj, lt, le, lb = oracle.asym_basis(jmax, A, B, C, 1000)
    assert len(lj) == 16
    terms = [(l, m) for l in range(4) for m in range(l + 1)]
    Gnum = _numerical_G(lj, lb, jmax, terms)
    for (lam, mu), Gn in zip(terms, Gnum):
        Go = oracle.asym_G(lj, lb, jmax, lam, mu)
        assert np.abs(Gn.imag).max() < 1e-12
        assert np.abs(Go - Gn.real).max() < 1e-12, (lam, mu)


def test_G_identity_symmetry_and_m_blocks():
    p = inputs.asym_pes_params(jmax=6, max_states=200, lam_max=4)
    lj, lt, le, lb = oracle.asym_basis(p.jmax, p.A, p.B, p.C, p.max_states)
    e, lev, jq, mq = oracle.asym_states(lj, le)
    G0 = oracle.asym_G(lj, lb, p.jmax, 0, 0)
    assert np.abs(G0 - np.eye(len(e))).max() < 1e-13
    for lam, mu in [(1, 0), (2, 1), (3, 3), (4, 2)]:
        G = oracle.asym_G(lj, lb, p.jmax, lam, mu)
        assert np.abs(G - G.T).max() < 1e-14
        assert np.all(G[mq[:, None] != mq[None, :]] == 0.0)
        dJ = np.abs(jq[:, None] - jq[None, :])
        assert np.all(G[dJ > lam] == 0.0)


def test_prolate_limit_reduces_to_linear_rotor_coupling():
    # with B = C the K = 0 functions are eigenstates, and f_{lam 0} = P_lam(cos beta): the
    # coupling between K = 0 levels is the Gaunt integral of Eq. 15 of a linear rotor
    jmax = 5
    lj, lt, le, lb = oracle.asym_basis(jmax, 7.0, 3.0, 3.0, 10_000)
    e, lev, jq, mq = oracle.asym_states(lj, le)
    k0 = [l for l in range(len(lj)) if abs(lb[l][jmax]) > 0.5]
    assert sorted(lj[k0].tolist()) == list(range(jmax + 1))
    for lam in range(4):
        Ga = oracle.asym_G(lj, lb, jmax, lam, 0)
        Gd = oracle.diatom_G(jmax, lam)
        for l2 in k0:
            for l1 in k0:
                J2, J1 = lj[l2], lj[l1]
                for M in range(-min(J1, J2), min(J1, J2) + 1):
                    r = oracle.asym_states(lj, le)[1].tolist().index(l2) + M + J2
                    c = oracle.asym_states(lj, le)[1].tolist().index(l1) + M + J1
                    ref = Gd[J2 * J2 + J2 + M, J1 * J1 + J1 + M] * lb[l2][jmax] * lb[l1][jmax]
                    assert abs(Ga[r, c] - ref) < 1e-13


def test_truncation_keeps_whole_levels_in_energy_order():
    p = inputs.asym_pes_params()
    lj, lt, le, lb = oracle.asym_basis(p.jmax, p.A, p.B, p.C, p.max_states)
    n = int(np.sum(2 * lj + 1))
    assert n <= 1600 and np.all(np.diff(le) >= 0)
    # the first level left out would overflow the limit
    allj, allt, alle, _ = oracle.asym_basis(p.jmax, p.A, p.B, p.C, 10 ** 6)
    nxt = len(lj)
    assert n + 2 * allj[nxt] + 1 > 1600
    assert np.array_equal(allj[:nxt], lj) and np.array_equal(allt[:nxt], lt)
    assert (n, len(lj)) == (1580, 110)


def test_small_asym_propagation_conserves_norm_and_energy():
    p, ts = inputs.small_asym_workload()
    sysA = oracle.asym_system(p)
    amp, res = oracle.propagate(sysA, ts.e_coll[:3], ts.b[:3], np.zeros(3, int), r0=ts.r0, r_end=ts.r_end,
                                dt=ts.dt)
    assert np.all(res["status"] == 0)
    assert np.all(res["norm_dev"] < 1e-7)
    assert np.all(res["energy_dev"] < 1e-6 * ts.e_coll[0])
    pop = np.abs(amp) ** 2
    assert pop[:, 1:].sum(axis=1).max() > 1e-2                 # the anisotropy does transfer population
