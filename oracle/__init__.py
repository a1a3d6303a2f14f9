"""Python side of the MQCT oracle (plain FP64 CPU reference of the trajectory method).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``.  The CUDA library never imports it.

The arithmetic lives in ``mqct_oracle.c`` (built with gcc into ``oracle/_build``);
this module only marshals numpy arrays through ctypes.  Every quantity is in
atomic units (hartree, bohr, electron masses, atomic units of time).

Paper passages followed (arXiv 2312.02322): Eq. 4-10 (equations of motion), Eq. 12
(factorised PES), Eq. 15 (Gaunt integral), Eq. 1 and Eq. 16 (asymmetric-top states and
their coupling), Sec. III (cubic spline of the coupling),
Sec. II (cross sections from final populations).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mqct_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_MAX_STEPS = 1
ST_TABLE_RANGE = 2
ST_NONFINITE = 4

F_NO_STOP = 1
F_PRESCRIBED = 2
F_FLIP_JY = 4
F_PLANT_TORQUE = 8      # planted mistake: torque sign reversed alone
F_PLANT_CORIOLIS = 16   # planted mistake: Coriolis factor 1/2 dropped
F_DECOUPLED = 32        # classical motion in the isotropic potential alone (AT-MQCT decoupling)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP over trajectories)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("n_terms", C.c_int), ("n_grid", C.c_int),
        ("mu", C.c_double), ("r_min", C.c_double), ("r_max", C.c_double),
        ("energy", C.c_void_p), ("level", C.c_void_p), ("jq", C.c_void_p), ("mq", C.c_void_p),
        ("G", C.c_void_p), ("v", C.c_void_p), ("dv_ends", C.c_void_p),
        ("n_params", C.c_int), ("dvp", C.c_void_p), ("dvp_ends", C.c_void_p),
        ("grid_log", C.c_int), ("trunc_thr", C.c_double), ("trunc_r", C.c_double * 2),
        ("g_nnz", C.c_longlong), ("g_term", C.c_void_p), ("g_row", C.c_void_p), ("g_col", C.c_void_p),
        ("g_val", C.c_void_p), ("adapt_tol", C.c_double), ("adapt_hmax_factor", C.c_int),
    ]


class _Traj(C.Structure):
    _fields_ = [("e_coll", C.c_double), ("b", C.c_double), ("r0", C.c_double), ("r_end", C.c_double),
                ("dt", C.c_double), ("init_state", C.c_int), ("max_steps", C.c_int)]


class _Res(C.Structure):
    _fields_ = [("steps", C.c_int), ("status", C.c_int), ("norm_dev", C.c_double), ("energy_dev", C.c_double),
                ("angmom_dev", C.c_double), ("t_final", C.c_double), ("R", C.c_double), ("PR", C.c_double),
                ("Phi", C.c_double), ("PPhi", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.ora_cg.restype = C.c_double
            L.ora_cg.argtypes = [C.c_int] * 6
            L.ora_diatom_n.restype = C.c_int
            L.ora_spline.restype = C.c_int
            L.ora_propagate.restype = C.c_int
            L.ora_tangent.restype = C.c_int
            L.ora_num_threads.restype = C.c_int
            L.ora_asym_levels.restype = C.c_int
            L.ora_asym_basis.restype = C.c_int
            L.ora_sys_terms.restype = C.c_int
            L.ora_sys_kept.restype = C.c_int
            L.ora_diatom_G_triplets.restype = C.c_longlong
            L.ora_diatom_G_triplets.argtypes = [C.c_int, C.c_int, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def cg(j1, m1, j2, m2, J, M) -> float:
    """Clebsch-Gordan coefficient <j1 m1 j2 m2 | J M> (Racah formula)."""
    return lib().ora_cg(j1, m1, j2, m2, J, M)


def num_threads() -> int:
    return lib().ora_num_threads()


class System:
    """Atom + rigid-rotor system in the oracle's own representation (atomic units).

    energy[n], level[n], jq[n], mq[n] label the states (jq < 0 disables the Coriolis
    term for that state); G[L][n][n] are the angular coupling matrices of Eq. 12, or, for
    large bases, a tuple of triplet arrays (term, row, col, value) with n_terms L;
    v[L][n_grid] and dv_ends[L][2] (dv/dR) define the clamped splines of v_lambda(R) --
    in ln R on a logarithmic grid when grid_log (Sec. III).  trunc = (threshold, R_a, R_b)
    drops every M_rc with |M_rc| <= threshold at both R_a and R_b (Sec. III).  adapt = (tol,
    hmax_factor) switches on the step-doubling step control (steps between dt and hmax_factor dt).
    """

    def __init__(self, energy, level, jq, mq, G, v, dv_ends, mu, r_min, r_max, dvp=None, dvp_ends=None,
                 grid_log=False, trunc=None, n_terms=None, adapt=None):
        self.energy = np.ascontiguousarray(energy, np.float64)
        self.level = np.ascontiguousarray(level, np.int32)
        self.jq = np.ascontiguousarray(jq, np.int32)
        self.mq = np.ascontiguousarray(mq, np.int32)
        if isinstance(G, tuple):
            self.G = None
            self.trip = tuple(np.ascontiguousarray(a, t) for a, t in zip(G, (np.int32, np.int32, np.int32, np.float64)))
        else:
            self.G = np.ascontiguousarray(G, np.float64)
            self.trip = None
        self.v = np.ascontiguousarray(v, np.float64)
        self.dv_ends = np.ascontiguousarray(dv_ends, np.float64)
        self.mu, self.r_min, self.r_max = float(mu), float(r_min), float(r_max)
        self.n = self.energy.shape[0]
        self.L = self.G.shape[0] if self.G is not None else int(n_terms if n_terms is not None else self.v.shape[0])
        self.grid_log = bool(grid_log)
        self.adapt = None if adapt is None else (float(adapt[0]), int(adapt[1]))
        self.trunc = None if trunc is None else tuple(float(x) for x in trunc)
        self.n_grid = self.v.shape[1]
        self.n_levels = int(self.level.max()) + 1
        self.dvp = None if dvp is None else np.ascontiguousarray(dvp, np.float64)
        self.dvp_ends = None if dvp_ends is None else np.ascontiguousarray(dvp_ends, np.float64)
        assert self.G is None or self.G.shape == (self.L, self.n, self.n)
        assert self.v.shape == (self.L, self.n_grid) and self.dv_ends.shape == (self.L, 2)

    def _desc(self):
        d = _Desc()
        d.n, d.n_terms, d.n_grid = self.n, self.L, self.n_grid
        d.mu, d.r_min, d.r_max = self.mu, self.r_min, self.r_max
        d.energy, d.level, d.jq, d.mq = _p(self.energy), _p(self.level), _p(self.jq), _p(self.mq)
        d.G = _p(self.G) if self.G is not None else None
        d.v, d.dv_ends = _p(self.v), _p(self.dv_ends)
        if self.trip is not None:
            d.g_nnz = self.trip[0].shape[0]
            d.g_term, d.g_row, d.g_col, d.g_val = (_p(a) for a in self.trip)
        d.grid_log = 1 if self.grid_log else 0
        if self.adapt is not None:
            d.adapt_tol, d.adapt_hmax_factor = self.adapt
        if self.trunc is not None:
            d.trunc_thr = self.trunc[0]
            d.trunc_r[0], d.trunc_r[1] = self.trunc[1], self.trunc[2]
        if self.dvp is not None:
            d.n_params = self.dvp.shape[0]
            d.dvp, d.dvp_ends = _p(self.dvp), _p(self.dvp_ends)
        return d


def diatom_basis(jmax: int, bconst: float):
    n = lib().ora_diatom_n(jmax)
    e = np.zeros(n)
    lev, jq, mq = (np.zeros(n, np.int32) for _ in range(3))
    lib().ora_diatom_basis(C.c_int(jmax), C.c_double(bconst), _p(e), _p(lev), _p(jq), _p(mq))
    return e, lev, jq, mq


def diatom_G(jmax: int, lam: int) -> np.ndarray:
    """<j'' m | P_lambda | j' m> in j-major state order (Eq. 15)."""
    n = lib().ora_diatom_n(jmax)
    G = np.zeros((n, n))
    lib().ora_diatom_G(C.c_int(jmax), C.c_int(lam), _p(G))
    return G


def sys_terms(sys: System, R):
    """v_lambda(R), dv/dR, d2v/dR2 from the system's splines: arrays [len(R)][L]."""
    R = np.ascontiguousarray(np.atleast_1d(R), np.float64)
    out = [np.zeros((R.size, sys.L)) for _ in range(3)]
    d = sys._desc()
    st = lib().ora_sys_terms(C.byref(d), C.c_int(R.size), _p(R), *(_p(o) for o in out))
    assert st == 0, st
    return tuple(out)


def sys_kept(sys: System) -> np.ndarray:
    """The truncation's keep mask [n][n] (1: M_rc retained; 0 also between different m)."""
    keep = np.zeros((sys.n, sys.n), np.uint8)
    d = sys._desc()
    st = lib().ora_sys_kept(C.byref(d), _p(keep))
    assert st == 0, st
    return keep.astype(bool)


def diatom_G_triplets(jmax: int, lam: int):
    """The non-zero <j'' m | P_lambda | j' m> (Eq. 15) as (row, col, value) arrays."""
    n = lib().ora_diatom_n(jmax)
    cap = n * (2 * lam + 1) + 16
    row, col = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    val = np.zeros(cap)
    k = lib().ora_diatom_G_triplets(jmax, lam, cap, _p(row), _p(col), _p(val))
    assert k >= 0
    return row[:k], col[:k], val[:k]


def diatom_pes(A, beta, c6, rd, n_grid, r_min, r_max, with_params=False, grid_log=False):
    """Grid tables of v_l(R) = A_l exp(-beta_l R) (+ damped -C6 R^-6 on term 0), end slopes dv/dR
    and, with with_params, their derivatives with respect to (A_0.., beta_0..); grid uniform in R,
    or in ln R with grid_log."""
    A = np.ascontiguousarray(A, np.float64)
    beta = np.ascontiguousarray(beta, np.float64)
    L = A.shape[0]
    v = np.zeros((L, n_grid))
    ends = np.zeros((L, 2))
    dvp = np.zeros((2 * L, L, n_grid)) if with_params else None
    dvpe = np.zeros((2 * L, L, 2)) if with_params else None
    lib().ora_diatom_pes_grid(C.c_int(L), _p(A), _p(beta), C.c_double(c6), C.c_double(rd), C.c_int(n_grid),
                              C.c_double(r_min), C.c_double(r_max), C.c_int(1 if grid_log else 0), _p(v), _p(ends),
                              _p(dvp) if with_params else None, _p(dvpe) if with_params else None)
    return v, ends, dvp, dvpe


def diatom_system(jmax, bconst, mu, A, beta, c6, rd, n_grid, r_min, r_max, with_params=False, grid_log=False,
                  trunc=None, sparse=None, adapt=None) -> System:
    """Atom + linear rotor (Eq. 2 basis, Eq. 15 coupling, PES of the form used in the tests);
    sparse (default: N > 2000) passes G as triplets."""
    e, lev, jq, mq = diatom_basis(jmax, bconst)
    L = len(A)
    if sparse is None:
        sparse = e.shape[0] > 2000
    if sparse:
        parts = [diatom_G_triplets(jmax, l) for l in range(L)]
        G = (np.concatenate([np.full(p[0].shape[0], l, np.int32) for l, p in enumerate(parts)]),
             np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
             np.concatenate([p[2] for p in parts]))
    else:
        G = np.stack([diatom_G(jmax, l) for l in range(L)])
    v, ends, dvp, dvpe = diatom_pes(A, beta, c6, rd, n_grid, r_min, r_max, with_params, grid_log)
    return System(e, lev, jq, mq, G, v, ends, mu, r_min, r_max, dvp, dvpe, grid_log=grid_log, trunc=trunc,
                  n_terms=L, adapt=adapt)


def asym_levels(J: int, A: float, B: float, Cc: float):
    """Eigenstates of the rigid asymmetric top for one J (Eq. 1): energies ascending (tau = -J..J)
    and b[e][K + J]."""
    n = 2 * J + 1
    E = np.zeros(n)
    b = np.zeros((n, n))
    if lib().ora_asym_levels(C.c_int(J), C.c_double(A), C.c_double(B), C.c_double(Cc), _p(E), _p(b)):
        raise MemoryError("ora_asym_levels")
    return E, b


def asym_basis(jmax: int, A: float, B: float, Cc: float, max_states: int):
    """Levels kept for the asymmetric-top basis: (J, tau, E, b[l][K + jmax]) in ascending energy."""
    nall = (jmax + 1) ** 2
    lj, lt = np.zeros(nall, np.int32), np.zeros(nall, np.int32)
    le, lb = np.zeros(nall), np.zeros((nall, 2 * jmax + 1))
    nl = lib().ora_asym_basis(C.c_int(jmax), C.c_double(A), C.c_double(B), C.c_double(Cc), C.c_int(max_states),
                              _p(lj), _p(lt), _p(le), _p(lb))
    if nl < 0:
        raise MemoryError("ora_asym_basis")
    return lj[:nl].copy(), lt[:nl].copy(), le[:nl].copy(), lb[:nl].copy()


def asym_states(lev_J, lev_E):
    """State labels of the level-major asymmetric-top basis (M = -J..J inside each level)."""
    e, lev, jq, mq = [], [], [], []
    for l, (J, E) in enumerate(zip(lev_J, lev_E)):
        for M in range(-J, J + 1):
            e.append(E); lev.append(l); jq.append(J); mq.append(M)
    return np.array(e), np.array(lev, np.int32), np.array(jq, np.int32), np.array(mq, np.int32)


def asym_G(lev_J, lev_b, jmax: int, lam: int, mu: int) -> np.ndarray:
    """<J'' tau'' M | f_{lam mu} | J' tau' M> over the level-major states (Eq. 16)."""
    lev_J = np.ascontiguousarray(lev_J, np.int32)
    lev_b = np.ascontiguousarray(lev_b, np.float64)
    n = int(np.sum(2 * lev_J + 1))
    G = np.zeros((n, n))
    lib().ora_asym_G(C.c_int(len(lev_J)), _p(lev_J), _p(lev_b), C.c_int(jmax), C.c_int(lam), C.c_int(mu), C.c_int(n),
                     _p(G))
    return G


def asym_system(p, with_params=False) -> System:
    """Atom + rigid asymmetric top from an AsymTopParams-like object (Eq. 1 basis, Eq. 16 coupling)."""
    lj, lt, le, lb = asym_basis(p.jmax, p.A, p.B, p.C, p.max_states)
    e, lev, jq, mq = asym_states(lj, le)
    G = np.stack([asym_G(lj, lb, p.jmax, int(l), int(m)) for l, m in zip(p.lam, p.mproj)])
    v, ends, dvp, dvpe = diatom_pes(p.coef, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max, with_params)
    s = System(e, lev, jq, mq, G, v, ends, p.mu, p.r_min, p.r_max, dvp, dvpe)
    s.tau = lt
    return s


def spline(y, h, d0, dn) -> np.ndarray:
    y = np.ascontiguousarray(y, np.float64)
    coef = np.zeros((y.shape[0] - 1, 4))
    rc = lib().ora_spline(C.c_int(y.shape[0]), C.c_double(h), _p(y), C.c_double(d0), C.c_double(dn), _p(coef))
    if rc:
        raise ValueError("ora_spline failed")
    return coef


def spline_eval(coef, n_grid, r_min, r_max, R):
    R = np.ascontiguousarray(R, np.float64)
    f, df, d2f = (np.zeros_like(R) for _ in range(3))
    lib().ora_spline_eval(_p(np.ascontiguousarray(coef)), C.c_int(n_grid), C.c_double(r_min), C.c_double(r_max),
                          C.c_int(R.shape[0]), _p(R), _p(f), _p(df), _p(d2f))
    return f, df, d2f


def _trajs(e_coll, b, r0, r_end, dt, init_state, max_steps):
    n = len(e_coll)
    arr = (_Traj * n)()
    for i in range(n):
        arr[i].e_coll = float(e_coll[i])
        arr[i].b = float(b[i])
        arr[i].r0 = float(np.broadcast_to(r0, (n,))[i])
        arr[i].r_end = float(np.broadcast_to(r_end, (n,))[i])
        arr[i].dt = float(np.broadcast_to(dt, (n,))[i])
        arr[i].init_state = int(init_state[i])
        arr[i].max_steps = int(np.broadcast_to(max_steps, (n,))[i])
    return arr


def _results(res, n):
    out = {k: np.array([getattr(res[i], k) for i in range(n)]) for k, _ in _Res._fields_}
    out["steps"] = out["steps"].astype(np.int64)
    out["status"] = out["status"].astype(np.int64)
    return out


def propagate(sys: System, e_coll, b, init_state, r0=30.0, r_end=30.0, dt=5.0, max_steps=1_000_000,
              flags=0, line_speed=None, n_threads=0):
    """Run the RK4 MQCT trajectories; returns (final amplitudes [n_traj][n] complex, result dict)."""
    n_traj = len(e_coll)
    tr = _trajs(e_coll, b, r0, r_end, dt, init_state, max_steps)
    amp = np.zeros((n_traj, sys.n, 2))
    res = (_Res * n_traj)()
    ls = None if line_speed is None else np.ascontiguousarray(line_speed, np.float64)
    d = sys._desc()
    rc = lib().ora_propagate(C.byref(d), tr, C.c_int(n_traj), C.c_int(flags), _p(ls) if ls is not None else None,
                             C.c_int(n_threads), _p(amp), res)
    if rc:
        raise RuntimeError(f"ora_propagate failed ({rc})")
    return amp[..., 0] + 1j * amp[..., 1], _results(res, n_traj)


def tangent(sys: System, e_coll, b, init_state, r0=30.0, r_end=30.0, dt=5.0, max_steps=1_000_000, n_threads=0):
    """Forward-mode derivative of the final populations: returns (amp, dpop [n_traj][P][n], results)."""
    if sys.dvp is None:
        raise ValueError("system has no parameter-derivative tables")
    n_traj = len(e_coll)
    P = sys.dvp.shape[0]
    tr = _trajs(e_coll, b, r0, r_end, dt, init_state, max_steps)
    amp = np.zeros((n_traj, sys.n, 2))
    dpop = np.zeros((n_traj, P, sys.n))
    res = (_Res * n_traj)()
    d = sys._desc()
    rc = lib().ora_tangent(C.byref(d), tr, C.c_int(n_traj), C.c_int(n_threads), _p(amp), _p(dpop), res)
    if rc:
        raise RuntimeError(f"ora_tangent failed ({rc})")
    return amp[..., 0] + 1j * amp[..., 1], dpop, _results(res, n_traj)


def cross_sections(sys: System, pop, weight, group, n_groups) -> np.ndarray:
    """sigma[g][level''] = sum_{t in g} weight_t * sum_{s in level''} pop_t[s]."""
    pop = np.ascontiguousarray(pop, np.float64)
    weight = np.ascontiguousarray(weight, np.float64)
    group = np.ascontiguousarray(group, np.int32)
    sig = np.zeros((n_groups, sys.n_levels))
    lib().ora_cross_sections(C.c_int(sys.n), _p(sys.level), C.c_int(sys.n_levels), C.c_int(pop.shape[0]), _p(pop),
                             _p(weight), _p(group), C.c_int(n_groups), _p(sig))
    return sig


def molmol_states(lev_J, j2s, lev_E1, bconst2):
    """Composite states of Eq. 3 for an asymmetric top (levels l1 with J = lev_J[l1], energies lev_E1)
    and a linear rotor (j2 in j2s, E = bconst2 j2 (j2+1)): for each level l1, each j2, each total j in
    |J - j2| .. J + j2 and m = -j..j.  Level id = l1 * len(j2s) + index of j2.  Returns energy,
    level, j (total), m, l1, j2."""
    e, lev, jq, mq, l1s, j2o = [], [], [], [], [], []
    for l1, (J, E1) in enumerate(zip(lev_J, lev_E1)):
        for i2, a in enumerate(j2s):
            for j in range(abs(int(J) - a), int(J) + a + 1):
                for m in range(-j, j + 1):
                    e.append(E1 + bconst2 * a * (a + 1)); lev.append(l1 * len(j2s) + i2)
                    jq.append(j); mq.append(m); l1s.append(l1); j2o.append(a)
    i32 = lambda x: np.array(x, np.int32)
    return np.array(e), i32(lev), i32(jq), i32(mq), i32(l1s), i32(j2o)


def molmol_G(lev_J, lev_b, jmax1, l1, j2, jt, mt, lam1, mu1, lam2, lam) -> np.ndarray:
    """<n'' m | tau_{lam1 mu1 lam2 lam} | n' m> (Eqs. 13-17) over the composite states."""
    n = len(l1)
    G = np.zeros((n, n))
    a = [np.ascontiguousarray(x, np.int32) for x in (l1, j2, jt, mt, lev_J)]
    lib().ora_molmol_G(C.c_int(n), *(_p(x) for x in a[:4]), _p(a[4]),
                       _p(np.ascontiguousarray(lev_b, np.float64)), C.c_int(jmax1), C.c_int(lam1), C.c_int(mu1),
                       C.c_int(lam2), C.c_int(lam), _p(G))
    return G

