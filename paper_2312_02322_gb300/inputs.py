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

    @property
    def n(self) -> int:
        return len(self.e_coll)

    def subset(self, idx) -> "TrajSet":
        idx = np.asarray(idx)
        return TrajSet(self.e_coll[idx], self.b[idx], self.init_j[idx], self.init_m[idx], self.group[idx],
                       self.n_groups, self.r0, self.r_end, self.dt, self.max_steps, self.sampling, self.b_max,
                       self.n_b, self.m_avg,
                       self.system[idx] if len(self.system) else self.system, self.group_e, self.group_j)


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


# ----------------------------------------------------------------------------
# The five workloads
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
