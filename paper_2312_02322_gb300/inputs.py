"""Seeded synthetic workloads for the MQCT trajectory path.

This module only produces input numbers -- physical constants, PES parameters,
basis sizes, collision energies, impact parameters, initial states and seeds --
in atomic units.  It holds none of the method's arithmetic (no coupling matrices,
no splines, no equations of motion, no cross-section weights), so that the CUDA
library and the CPU oracle can both be fed from it without sharing any step of
the computation.

The workloads stand in for the paper's H2O + H2 production run (its PES and
comparison data are not available here): an atom + rigid linear rotor with an
exponentially anisotropic PES expanded in Legendre polynomials (the form of the
expansion in Eq. 12), tabulated on an R grid for cubic-spline interpolation
(Sec. III), with regular or Monte-Carlo impact-parameter sampling (Sec. III).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# CODATA-derived unit conversions
HARTREE_CM = 219474.6313632  # cm^-1 per hartree
AMU_ME = 1822.888486         # electron masses per unified atomic mass unit
BOHR2_A2 = 0.2800285         # square angstrom per square bohr

DEFAULT_SEED = 20231204


def cm(x):
    """cm^-1 -> hartree."""
    return np.asarray(x, dtype=np.float64) / HARTREE_CM


@dataclass
class DiatomParams:
    """Atom + rigid diatom; energies E_j = B j (j + 1); PES
    V(R, theta) = sum_l A_l exp(-beta_l R) P_l(cos theta) - C6 R^-6 (1 - exp(-(R/Rd)^6))."""
    jmax: int
    bconst: float            # hartree
    mu: float                # electron masses
    A: np.ndarray            # hartree, one per Legendre order 0..L-1
    beta: np.ndarray         # 1/bohr
    c6: float                # hartree bohr^6
    rd: float = 3.0          # bohr
    n_grid: int = 200
    r_min: float = 2.0
    r_max: float = 30.0

    @property
    def n_states(self) -> int:
        return (self.jmax + 1) ** 2

    @property
    def n_terms(self) -> int:
        return len(self.A)


@dataclass
class TrajSet:
    """A list of trajectories; energies in hartree, lengths in bohr, time in a.u."""
    e_coll: np.ndarray
    b: np.ndarray
    init_j: np.ndarray
    init_m: np.ndarray
    group: np.ndarray         # cross-section group of each trajectory
    n_groups: int
    r0: float = 30.0
    r_end: float = 30.0
    dt: float = 5.0
    max_steps: int = 1_000_000
    sampling: str = "regular"  # "regular": midpoint b grid; "mc": b ~ U(0, b_max)
    b_max: float = 12.0
    n_b: int = 32              # b-grid points per group (regular sampling)
    m_avg: str = "one"         # "one": one m' per b; "all": every m' of the initial level per b
    system: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))  # system index per trajectory
    group_e: np.ndarray = field(default_factory=lambda: np.zeros(0))           # energy of each group
    group_j: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32)) # initial level of each group
    init_by: str = "j"         # "j": init_j is the rotor j label; "level": init_j is a level index

    @property
    def n(self) -> int:
        return len(self.e_coll)

    def subset(self, idx) -> "TrajSet":
        idx = np.asarray(idx)
        return TrajSet(self.e_coll[idx], self.b[idx], self.init_j[idx], self.init_m[idx], self.group[idx],
                       self.n_groups, self.r0, self.r_end, self.dt, self.max_steps, self.sampling, self.b_max,
                       self.n_b, self.m_avg,
                       self.system[idx] if len(self.system) else self.system, self.group_e, self.group_j,
                       self.init_by)


def diatom_pes_params(jmax=6, n_grid=200, mu_amu=4.0):
    """The exponential-anisotropic PES used by every diatom workload."""
    return DiatomParams(
        jmax=jmax,
        bconst=float(cm(10.0)),
        mu=mu_amu * AMU_ME,
        A=cm([2e5, 5e4, 2e4, 8e3, 3e3]),
        beta=np.array([1.8, 1.9, 2.0, 2.1, 2.2]),
        c6=float(cm(3e5)),
        rd=3.0,
        n_grid=n_grid,
        r_min=2.0,
        r_max=30.0,
    )


def regular_set(energies_cm, init_js, n_b, b_max, m_avg="one", dt=5.0, r0=30.0) -> TrajSet:
    """Midpoint impact-parameter grid b_i = (i + 1/2) b_max / n_b for every (E, j') group.

    m_avg="one": one trajectory per b with m'_i = (i mod (2j'+1)) - j';
    m_avg="all": 2j'+1 trajectories per b, one per m'."""
    e, b, jj, mm, g = [], [], [], [], []
    ge, gj = [], []
    gid = 0
    for E in energies_cm:
        for j in init_js:
            ge.append(float(cm(E)))
            gj.append(j)
            for i in range(n_b):
                bi = (i + 0.5) * b_max / n_b
                ms = [(i % (2 * j + 1)) - j] if m_avg == "one" else list(range(-j, j + 1))
                for m in ms:
                    e.append(float(cm(E))); b.append(bi); jj.append(j); mm.append(m); g.append(gid)
            gid += 1
    return TrajSet(np.array(e), np.array(b), np.array(jj, np.int32), np.array(mm, np.int32),
                   np.array(g, np.int32), gid, r0=r0, r_end=r0, dt=dt, sampling="regular", b_max=b_max, n_b=n_b,
                   m_avg=m_avg, group_e=np.array(ge), group_j=np.array(gj, np.int32))


@dataclass
class AsymTopParams:
    """Atom + rigid asymmetric top: rotor A Ja^2 + B Jb^2 + C Jc^2 (J <= jmax, whole levels kept in
    ascending energy while N <= max_states); PES sum_t coef_t exp(-beta_t R) f_{lam_t mu_t} with the
    real angular functions f_{lam mu} (P_lam(cos beta) for mu = 0, 2 d^lam_{0 mu}(beta) cos(mu gamma)
    otherwise) and the damped -C6 R^-6 dispersion on term 0 = (0, 0)."""
    jmax: int
    A: float                 # hartree
    B: float
    C: float
    max_states: int
    mu: float                # electron masses
    lam: np.ndarray
    mproj: np.ndarray
    coef: np.ndarray         # hartree
    beta: np.ndarray         # 1/bohr
    c6: float
    rd: float = 3.0
    n_grid: int = 400
    r_min: float = 2.0
    r_max: float = 30.0

    @property
    def n_terms(self) -> int:
        return len(self.coef)


def asym_pes_params(jmax=12, max_states=1600, lam_max=6, n_grid=400, mu_amu=3.3, seed=DEFAULT_SEED):
    """Rigid asymmetric top with water-like constants A, B, C = 27.88, 14.51, 9.28 cm^-1 and all
    cos-type terms 0 <= mu <= lam <= lam_max.  The isotropic term is the diatom workloads' repulsive
    wall 2e5 exp(-1.8 R) cm^-1 with the damped C6 = 3e5 cm^-1 bohr^6 dispersion; the anisotropic
    coefficients are drawn as coef ~ N(0, (2e4 / (1 + lam))^2) cm^-1 with beta = 1.8 + 0.1 lam."""
    rng = np.random.default_rng(seed)
    lam, mproj, coef, beta = [], [], [], []
    for l in range(lam_max + 1):
        for m in range(l + 1):
            lam.append(l)
            mproj.append(m)
            coef.append(2e5 if l == 0 else rng.normal(0.0, 2e4 / (1.0 + l)))
            beta.append(1.8 + 0.1 * l)
    return AsymTopParams(jmax=jmax, A=float(cm(27.88)), B=float(cm(14.51)), C=float(cm(9.28)),
                         max_states=max_states, mu=mu_amu * AMU_ME, lam=np.array(lam, np.int32),
                         mproj=np.array(mproj, np.int32), coef=cm(coef), beta=np.array(beta), c6=float(cm(3e5)),
                         rd=3.0, n_grid=n_grid, r_min=2.0, r_max=30.0)


def mc_set(energies_cm, n_per_e, b_max, seed=DEFAULT_SEED, init_level=0, init_m=0, dt=5.0, r0=30.0) -> TrajSet:
    """Monte-Carlo impact parameters b ~ U(0, b_max), n_per_e per energy, one group per energy,
    initial state (level, m) addressed by level index."""
    rng = np.random.default_rng(seed + 1)
    ne = len(energies_cm)
    e = np.repeat(cm(np.asarray(energies_cm, np.float64)), n_per_e)
    b = rng.uniform(0.0, b_max, ne * n_per_e)
    g = np.repeat(np.arange(ne, dtype=np.int32), n_per_e)
    n = ne * n_per_e
    return TrajSet(e, b, np.full(n, init_level, np.int32), np.full(n, init_m, np.int32), g, ne, r0=r0, r_end=r0,
                   dt=dt, sampling="mc", b_max=b_max, n_b=n_per_e, m_avg="one",
                   group_e=cm(np.asarray(energies_cm, np.float64)), group_j=np.full(ne, init_level, np.int32),
                   init_by="level")


# ----------------------------------------------------------------------------
# The workloads
# ----------------------------------------------------------------------------
def workload1():
    """N = 49 (j <= 6), E = 500 cm^-1, j' = 0, 32 midpoint b on 0-12 bohr, 200-point grid."""
    return diatom_pes_params(jmax=6, n_grid=200), regular_set([500.0], [0], n_b=32, b_max=12.0)


def workload2():
    """N = 441 (j <= 20), E in {100, 300, 1000, 3000} cm^-1, j' in {0, 1, 2}, 256 midpoint b on
    0-15 bohr per (E, j'): 3072 trajectories; 400-point grid."""
    return (diatom_pes_params(jmax=20, n_grid=400),
            regular_set([100.0, 300.0, 1000.0, 3000.0], [0, 1, 2], n_b=256, b_max=15.0))


def workload2_n1600():
    """N = 1600 (j <= 39): E in {1000, 3000} cm^-1, j' in {0, 1, 2}, 128 midpoint b on 0-15 bohr
    per (E, j'): 768 trajectories; 400-point grid."""
    return (diatom_pes_params(jmax=39, n_grid=400),
            regular_set([1000.0, 3000.0], [0, 1, 2], n_b=128, b_max=15.0))


def workload3(n_per_e=2500, seed=DEFAULT_SEED):
    """Asymmetric top, J <= 12 truncated to whole levels with N <= 1600 (N = 1580, 110 levels),
    28 cos-type terms lam <= 6, mu = 3.3 amu; 8 energies log-spaced on 10-2000 cm^-1, n_per_e
    trajectories per energy with b ~ U(0, 15), initial state the ground level (J = 0)."""
    energies = np.geomspace(10.0, 2000.0, 8)
    return asym_pes_params(seed=seed), mc_set(energies, n_per_e, 15.0, seed=seed)


def small_asym_workload(jmax=4, max_states=60, lam_max=3, energies=(300.0,), n_per_e=6, b_max=8.0, n_grid=120):
    """A reduced asymmetric-top case that the oracle finishes in seconds (parity tests)."""
    return (asym_pes_params(jmax=jmax, max_states=max_states, lam_max=lam_max, n_grid=n_grid),
            mc_set(list(energies), n_per_e, b_max))


def workload5():
    """N = 441, E = 1000 cm^-1, j' = 0, 1024 midpoint b on 0-15 bohr (gradient workload)."""
    return diatom_pes_params(jmax=20, n_grid=400), regular_set([1000.0], [0], n_b=1024, b_max=15.0)


def workload4(seed=DEFAULT_SEED, n_traj=50_000):
    """Uneven batch: bases j <= 6, 10, 20, 39 (N = 49, 121, 441, 1600) in a 1:2:4:1 mix,
    b ~ U(0, 20), E log-uniform on 10-5000 cm^-1, j' = 0; 400-point grids."""
    rng = np.random.default_rng(seed)
    jmaxes = [6, 10, 20, 39]
    systems = [diatom_pes_params(jmax=j, n_grid=400) for j in jmaxes]
    mix = np.array([1, 2, 4, 1], np.float64)
    counts = np.floor(mix / mix.sum() * n_traj).astype(int)
    counts[2] += n_traj - counts.sum()
    sys_idx = np.concatenate([np.full(c, i, np.int32) for i, c in enumerate(counts)])
    rng.shuffle(sys_idx)
    e = cm(np.exp(rng.uniform(np.log(10.0), np.log(5000.0), n_traj)))
    b = rng.uniform(0.0, 20.0, n_traj)
    z = np.zeros(n_traj, np.int32)
    ts = TrajSet(e, b, z, z.copy(), sys_idx.copy(), len(jmaxes), sampling="mc", b_max=20.0, n_b=0, system=sys_idx,
                 group_e=np.zeros(len(jmaxes)), group_j=np.zeros(len(jmaxes), np.int32))
    return systems, ts


def small_workload(jmax=3, n_b=6, energies=(500.0,), init_js=(0, 1), b_max=8.0, n_grid=120, m_avg="all"):
    """A reduced diatom case that the oracle finishes in seconds (used by parity tests)."""
    return (diatom_pes_params(jmax=jmax, n_grid=n_grid),
            regular_set(list(energies), list(init_js), n_b=n_b, b_max=b_max, m_avg=m_avg))


# the ten collision energies U of the paper's production run (Sec. III), cm^-1
PAPER_ENERGIES_CM = (20.00, 41.28, 84.00, 170.47, 346.41, 703.89, 1430.0, 2906.3, 5906.0, 12000.0)


@dataclass
class RateSet:
    u: np.ndarray           # [K] collision energies (hartree)
    energy: np.ndarray      # [L] level energies (hartree)
    g: np.ndarray           # [L] degeneracies
    sigma: np.ndarray       # [K][L][L] sigma_{a->b}(U_k) (bohr^2)
    kT: np.ndarray          # [T] k_B T (hartree)
    mu: float               # reduced mass (electron masses)


def rate_set(n_levels=30, temps_k=(10.0, 50.0, 100.0, 300.0, 1000.0), emax_cm=8000.0, mu_amu=1.8,
             mismatch=0.3, seed=DEFAULT_SEED) -> RateSet:
    """Synthetic state-to-state cross sections on the paper's ten energies: levels with energies
    uniform on [0, emax] cm^-1 (sorted; the first at 0) and degeneracies 2j+1, j uniform on 0..28;
    sigma_{a->b}(U) = s0 exp(-|dE| / 300 cm^-1) U / (U + |dE|) / g_a, s0 log-uniform on 0.1-30 bohr^2
    per pair (so that Eq. 19 holds before the perturbation), times an independent factor
    1 + mismatch * r, r uniform on [-1, 1], per direction and energy (the scatter of Fig. 1);
    elastic sigma_{a->a} = 50 bohr^2 / (1 + U / 1000 cm^-1).  kB = 3.1668115634556e-6 hartree/K."""
    rng = np.random.default_rng(seed)
    L = n_levels
    E = np.sort(rng.uniform(0.0, emax_cm, L))
    E[0] = 0.0
    j = rng.integers(0, 29, L)
    g = (2 * j + 1).astype(np.float64)
    U = np.asarray(PAPER_ENERGIES_CM, np.float64)
    dE = np.abs(E[None, :] - E[:, None])
    s0 = np.exp(rng.uniform(np.log(0.1), np.log(30.0), (L, L)))
    s0 = np.sqrt(s0 * s0.T)
    base = s0[None] * np.exp(-dE / 300.0)[None] * (U[:, None, None] / (U[:, None, None] + dE[None])) / g[None, :, None]
    sig = base * (1.0 + mismatch * rng.uniform(-1.0, 1.0, base.shape))
    for a in range(L):
        sig[:, a, a] = 50.0 / (1.0 + U / 1000.0)
    kT = np.asarray(temps_k, np.float64) * 3.1668115634556e-6
    return RateSet(u=cm(U), energy=cm(E), g=g, sigma=sig, kT=kT, mu=float(mu_amu * AMU_ME))


def sparse_pes_params(jmax=200, lam_max=12, n_grid=63, mu_amu=1.8, bconst_cm=None):
    """The paper-scale setup of Sec. III on an atom + rigid rotor: a 63-point logarithmic R grid on
    3-30 bohr, Legendre terms lam <= lam_max, wall and anisotropy placed where the paper's
    truncation distances (6.03, 7.11 bohr) sit on the repulsive wall:
    v_0 = 1e4 cm^-1 exp(-1.8 (R - 5)) - damped C6 (3e5 cm^-1 bohr^6, Rd = 3), and for lam >= 1
    v_lam = 3000 cm^-1 0.6^(lam-1) exp(-(1.8 + 0.05 lam)(R - 5)).  The rotational constant puts the
    top of the basis near the paper's 8000 cm^-1 (B = 8000 / (jmax (jmax + 1)) cm^-1, at most
    10 cm^-1); mu = 1.8 amu (H2O + H2)."""
    L = lam_max + 1
    beta = np.array([1.8] + [1.8 + 0.05 * l for l in range(1, L)])
    a5 = np.array([1e4] + [3000.0 * 0.6 ** (l - 1) for l in range(1, L)])
    A = cm(a5 * np.exp(beta * 5.0))
    B = bconst_cm if bconst_cm is not None else min(10.0, 8000.0 / max(1, jmax * (jmax + 1)))
    return DiatomParams(jmax=jmax, bconst=float(cm(B)), mu=mu_amu * AMU_ME, A=A, beta=beta, c6=float(cm(3e5)),
                        rd=3.0, n_grid=n_grid, r_min=3.0, r_max=30.0)


# the paper's truncation (Sec. III): |M| > 1 cm^-1 at R = 6.03 or 7.11 bohr
PAPER_TRUNC_CM = 1.0
PAPER_TRUNC_R = (6.03, 7.11)


@dataclass
class MolMolParams:
    """Asymmetric top + linear rotor (Sec. II, Eqs. 3 and 13): molecule-1 levels j1 <= j1max, rotor
    j2 values, PES terms (lam1, mu1, lam2, lam) with v_t = coef_t exp(-beta_t R) (+ damped C6 on term 0)."""
    A: float
    B: float
    C: float
    j1max: int
    bconst2: float
    j2: list
    mu: float
    terms: list               # (lam1, mu1, lam2, lam)
    coef: np.ndarray          # hartree
    beta: np.ndarray          # 1/bohr
    c6: float
    rd: float = 3.0
    n_grid: int = 200
    r_min: float = 2.0
    r_max: float = 30.0

    @property
    def n_terms(self) -> int:
        return len(self.terms)


def molmol_params(j1max=2, j2=(0, 2), n_grid=200):
    """Water-like top (A, B, C = 27.88, 14.51, 9.28 cm^-1) + para-H2 (B = 60.85 cm^-1, j2 in {0, 2}),
    mu = 1.8 amu; terms: the isotropic (0,0,0,0) -- whose tau is 1/(2 pi), so its coefficient is
    2 pi x (2e5 cm^-1) exp(-1.8 R) with the damped C6 = 3e5 cm^-1 bohr^6 -- and eight anisotropic
    (lam1, mu1, lam2, lam) terms with lam1, lam2 <= 2 and coefficients 2e4 / (1 + lam1 + lam2) cm^-1,
    beta = 1.9 + 0.1 (lam1 + lam2) bohr^-1 (a stand-in for the H2O + H2 PES, which is not available)."""
    terms = [(0, 0, 0, 0), (1, 0, 0, 1), (1, 1, 0, 1), (2, 0, 0, 2), (2, 2, 0, 2), (0, 0, 2, 2), (1, 0, 2, 1),
             (2, 0, 2, 0), (2, 2, 2, 2)]
    coef = [2 * np.pi * 2e5] + [2e4 / (1 + a + b) for (a, _, b, _) in terms[1:]]
    beta = [1.8] + [1.9 + 0.1 * (a + b) for (a, _, b, _) in terms[1:]]
    return MolMolParams(A=float(cm(27.88)), B=float(cm(14.51)), C=float(cm(9.28)), j1max=j1max,
                        bconst2=float(cm(60.85)), j2=list(j2), mu=1.8 * AMU_ME, terms=terms, coef=cm(coef),
                        beta=np.array(beta), c6=float(cm(3e5) * 2 * np.pi), n_grid=n_grid)

