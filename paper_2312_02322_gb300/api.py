"""Thin Python binding of the C ABI in include/mqct.h (argument marshalling only).

Every step of the trajectory path runs in the CUDA library ``_build/libmqct.so``; this
module converts numpy / torch arguments to pointers and back.  torch provides device
memory and streams.  The library must be built (``paper_2312_02322_gb300.build``):
importing the binding without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmqct.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_TRAJ = range(7)
PATH_PLAIN, PATH_FACTORISED = 0, 1
FP64, FP32, BF16X3 = 0, 1, 2
TRAJ_MAX_STEPS, TRAJ_TABLE_RANGE, TRAJ_NONFINITE, TRAJ_TIMEOUT, TRAJ_INVALID = 1, 2, 4, 8, 16
PRESCRIBED_TRAJ = 1  # mqct_system_desc.flags
DECOUPLED_TRAJ = 2

_PATHS = {"plain": PATH_PLAIN, "factorised": PATH_FACTORISED}
_PRECS = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3}


class MQCTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mqct status {status}: {message}")
        self.status = status
        self.message = message


class Desc(C.Structure):
    _fields_ = [
        ("n_states", C.c_int32), ("energy", C.c_void_p), ("level", C.c_void_p), ("j", C.c_void_p),
        ("m", C.c_void_p), ("mu", C.c_double), ("n_terms", C.c_int32), ("G", C.c_void_p),
        ("g_nnz", C.c_int64), ("g_term", C.c_void_p), ("g_row", C.c_void_p), ("g_col", C.c_void_p),
        ("g_val", C.c_void_p), ("n_grid", C.c_int32), ("r_min", C.c_double), ("r_max", C.c_double),
        ("v", C.c_void_p), ("dv_ends", C.c_void_p), ("n_params", C.c_int32), ("dv_dparam", C.c_void_p),
        ("ddv_ends", C.c_void_p), ("path", C.c_int32), ("precision", C.c_int32), ("flags", C.c_int32),
        ("grid_kind", C.c_int32), ("trunc_threshold", C.c_double), ("trunc_r", C.c_double * 2),
        ("adapt_tol", C.c_double), ("adapt_hmax", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [("n_states", C.c_int32), ("n_levels", C.c_int32), ("n_terms", C.c_int32), ("n_grid", C.c_int32),
                ("n_blocks", C.c_int32), ("max_block", C.c_int32), ("path", C.c_int32), ("precision", C.c_int32),
                ("table_nnz", C.c_int64), ("table_bytes", C.c_int64), ("glambda_nnz", C.c_int64),
                ("device_bytes", C.c_int64), ("n_coupling_terms", C.c_int32), ("n_row_tiles", C.c_int32),
                ("tc_kchunks", C.c_int64), ("trunc_dropped", C.c_int64), ("grid_kind", C.c_int32),
                ("reserved", C.c_int32)]


class DiatomParams(C.Structure):
    _fields_ = [("jmax", C.c_int32), ("bconst", C.c_double), ("mu", C.c_double), ("n_terms", C.c_int32),
                ("A", C.c_double * 16), ("beta", C.c_double * 16), ("c6", C.c_double), ("rd", C.c_double),
                ("n_grid", C.c_int32), ("r_min", C.c_double), ("r_max", C.c_double), ("with_params", C.c_int32),
                ("path", C.c_int32), ("precision", C.c_int32), ("grid_kind", C.c_int32),
                ("trunc_threshold", C.c_double), ("trunc_r", C.c_double * 2)]


class AsymParams(C.Structure):
    _fields_ = [("jmax", C.c_int32), ("A", C.c_double), ("B", C.c_double), ("C", C.c_double),
                ("max_states", C.c_int32), ("mu", C.c_double), ("n_terms", C.c_int32), ("lam", C.c_int32 * 64),
                ("mproj", C.c_int32 * 64), ("coef", C.c_double * 64), ("beta", C.c_double * 64), ("c6", C.c_double),
                ("rd", C.c_double), ("n_grid", C.c_int32), ("r_min", C.c_double), ("r_max", C.c_double),
                ("with_params", C.c_int32), ("path", C.c_int32), ("precision", C.c_int32),
                ("tau_out", C.c_void_p)]


class PropagateOpts(C.Structure):
    _fields_ = [("t_start_ns", C.c_void_p), ("t_done_ns", C.c_void_p), ("batch_shape", C.c_void_p),
                ("tc_slots", C.c_void_p)]


GRID_UNIFORM, GRID_LOG = 0, 1


class MolMolParams(C.Structure):
    _fields_ = [("A", C.c_double), ("B", C.c_double), ("C", C.c_double), ("j1max", C.c_int32),
                ("bconst2", C.c_double), ("n_j2", C.c_int32), ("j2", C.c_int32 * 8), ("mu", C.c_double),
                ("n_terms", C.c_int32), ("lam1", C.c_int32 * 64), ("mu1", C.c_int32 * 64), ("lam2", C.c_int32 * 64),
                ("lam", C.c_int32 * 64), ("coef", C.c_double * 64), ("beta", C.c_double * 64), ("c6", C.c_double),
                ("rd", C.c_double), ("n_grid", C.c_int32), ("r_min", C.c_double), ("r_max", C.c_double),
                ("path", C.c_int32), ("precision", C.c_int32)]


class RateDesc(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_energies", C.c_int32), ("n_temps", C.c_int32), ("reserved", C.c_int32),
                ("mu", C.c_double), ("u", C.c_void_p), ("kT", C.c_void_p), ("level_energy", C.c_void_p),
                ("degeneracy", C.c_void_p)]


# Boltzmann constant (hartree per kelvin) and bohr^3 per atomic unit of time in cm^3/s (CODATA 2018)
KB_HARTREE_PER_K = 3.1668115634556e-6
RATE_AU_TO_CM3_S = 0.529177210903e-8 ** 3 / 2.4188843265857e-17

# (slots per CTA, threads) of the FP32 batched kernel for batch_shape = index + 1
BATCH_SHAPES = [(32, 512), (16, 512), (8, 256), (8, 512), (4, 512), (16, 256), (4, 256)]

TRAJ_DTYPE = np.dtype([("e_coll", "<f8"), ("b", "<f8"), ("r0", "<f8"), ("r_end", "<f8"), ("dt", "<f8"),
                       ("init_state", "<i4"), ("max_steps", "<i4"), ("system_idx", "<i4"), ("_pad", "<i4")])
DIAG_DTYPE = np.dtype([("steps", "<i4"), ("status", "<i4"), ("norm_dev", "<f8"), ("energy_dev", "<f8"),
                       ("angmom_dev", "<f8"), ("t_final", "<f8")])
assert TRAJ_DTYPE.itemsize == 56 and DIAG_DTYPE.itemsize == 40

_lock = threading.Lock()
_lib = None


def lib():
    """Load libmqct.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library not built: {LIB_PATH} (run python -m paper_2312_02322_gb300.build)")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.mqct_build_diatom.argtypes = [C.POINTER(DiatomParams), C.POINTER(Desc)]
            L.mqct_build_asym_top.argtypes = [C.POINTER(AsymParams), C.POINTER(Desc)]
            L.mqct_build_molmol.argtypes = [C.POINTER(MolMolParams), C.POINTER(Desc)]
            L.mqct_free_desc.argtypes = [C.POINTER(Desc)]
            L.mqct_free_desc.restype = None
            L.mqct_create_system.argtypes = [C.POINTER(Desc), C.POINTER(vp)]
            L.mqct_destroy_system.argtypes = [vp]
            L.mqct_system_info.argtypes = [vp, C.POINTER(Info)]
            L.mqct_propagate.argtypes = [C.POINTER(vp), i32, vp, i32, vp, vp, vp, vp]
            L.mqct_propagate_ex.argtypes = [C.POINTER(vp), i32, vp, i32, vp, vp, vp, C.POINTER(PropagateOpts), vp]
            L.mqct_cross_sections.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp]
            L.mqct_adjoint.argtypes = [vp, vp, i32, vp, vp, i32, vp, i32, vp, vp]
            L.mqct_rate_coefficients.argtypes = [C.POINTER(RateDesc), vp, vp, vp, vp]
            L.mqct_probe_fma_rate.argtypes = [i32, C.POINTER(C.c_double), vp]
            L.mqct_probe_fma_rate.restype = C.c_int
            L.mqct_probe_op_latency.argtypes = [i32, i32, C.POINTER(C.c_double), vp]
            L.mqct_probe_op_latency.restype = C.c_int
            L.mqct_last_error.restype = C.c_char_p
            L.mqct_last_launch_count.restype = C.c_int64
            L.mqct_version.restype = C.c_char_p
            for f in ("mqct_build_diatom", "mqct_build_asym_top", "mqct_build_molmol", "mqct_create_system", "mqct_destroy_system", "mqct_system_info",
                      "mqct_propagate", "mqct_propagate_ex", "mqct_cross_sections", "mqct_adjoint",
                      "mqct_rate_coefficients"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _check(st: int, allow=()):
    if st != OK and st not in allow:
        msg = lib().mqct_last_error()
        raise MQCTError(st, msg.decode() if msg else "")
    return st


def _ptr(x):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class System:
    """An mqct_system (immutable, owns its device memory).

    Keeps host copies of the state labels so that initial states can be addressed by
    (j, m) label; state indices are the caller order of the description."""

    def __init__(self, desc: Desc, keep=None):
        h = C.c_void_p()
        _check(lib().mqct_create_system(C.byref(desc), C.byref(h)))
        self._h = h
        n = desc.n_states
        self.n = n
        self.j = np.ctypeslib.as_array(C.cast(desc.j, C.POINTER(C.c_int32)), (n,)).copy()
        self.m = np.ctypeslib.as_array(C.cast(desc.m, C.POINTER(C.c_int32)), (n,)).copy()
        self.level = np.ctypeslib.as_array(C.cast(desc.level, C.POINTER(C.c_int32)), (n,)).copy()
        self.energy = np.ctypeslib.as_array(C.cast(desc.energy, C.POINTER(C.c_double)), (n,)).copy()
        self.mu = desc.mu
        self.n_params = desc.n_params
        self._keep = keep
        self._index = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(self.j, self.m))}
        self._lindex = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(self.level, self.m))}
        self.tau = None  # per-level tau label (asymmetric top only)

    @classmethod
    def diatom(cls, p: "_inputs.DiatomParams", path="plain", precision="fp64", with_params=False,
               prescribed=False, grid="uniform", trunc=None, decoupled=False, adapt=None) -> "System":
        """prescribed=True: MQCT_PRESCRIBED_TRAJ, each trajectory follows the time-symmetric straight
        line of impact parameter b and speed sqrt(2 e_coll / mu) for exactly max_steps steps.
        grid="log": MQCT_GRID_LOG tabulation (splines in ln R); trunc=(threshold, R_a, R_b): PLAIN-path
        truncation of |M| <= threshold at both distances (Sec. III); decoupled=True: MQCT_DECOUPLED_TRAJ
        (classical motion in the isotropic potential alone, the amplitudes along it); adapt=(tol, hmax):
        step-doubling adaptive steps between dt and hmax dt (FP64 systems)."""
        dp = DiatomParams()
        dp.jmax, dp.bconst, dp.mu, dp.n_terms = p.jmax, p.bconst, p.mu, p.n_terms
        for i in range(p.n_terms):
            dp.A[i] = float(p.A[i])
            dp.beta[i] = float(p.beta[i])
        dp.c6, dp.rd, dp.n_grid, dp.r_min, dp.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
        dp.with_params = int(bool(with_params))
        dp.path, dp.precision = _PATHS[path], _PRECS[precision]
        dp.grid_kind = {"uniform": GRID_UNIFORM, "log": GRID_LOG}[grid]
        if trunc is not None:
            dp.trunc_threshold, dp.trunc_r[0], dp.trunc_r[1] = (float(x) for x in trunc)
        d = Desc()
        _check(lib().mqct_build_diatom(C.byref(dp), C.byref(d)))
        d.flags = (PRESCRIBED_TRAJ if prescribed else 0) | (DECOUPLED_TRAJ if decoupled else 0)
        if adapt is not None:
            d.adapt_tol, d.adapt_hmax = float(adapt[0]), int(adapt[1])
        try:
            return cls(d)
        finally:
            lib().mqct_free_desc(C.byref(d))

    @staticmethod
    def molmol_params(p: "_inputs.MolMolParams", path="factorised", precision="fp64") -> MolMolParams:
        mp = MolMolParams()
        mp.A, mp.B, mp.C, mp.j1max, mp.bconst2 = p.A, p.B, p.C, p.j1max, p.bconst2
        mp.n_j2 = len(p.j2)
        for i, a in enumerate(p.j2):
            mp.j2[i] = int(a)
        mp.mu, mp.n_terms = p.mu, p.n_terms
        for t, (a, m, b, c) in enumerate(p.terms):
            mp.lam1[t], mp.mu1[t], mp.lam2[t], mp.lam[t] = a, m, b, c
            mp.coef[t], mp.beta[t] = float(p.coef[t]), float(p.beta[t])
        mp.c6, mp.rd, mp.n_grid, mp.r_min, mp.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
        mp.path, mp.precision = _PATHS[path], _PRECS[precision]
        return mp

    @classmethod
    def molmol(cls, p: "_inputs.MolMolParams", path="factorised", precision="fp64") -> "System":
        """Asymmetric top + linear rotor (composite states of Eq. 3, coupling of Eqs. 13-17)."""
        mp = cls.molmol_params(p, path, precision)
        d = Desc()
        _check(lib().mqct_build_molmol(C.byref(mp), C.byref(d)))
        try:
            return cls(d)
        finally:
            lib().mqct_free_desc(C.byref(d))

    @classmethod
    def asym_top(cls, p: "_inputs.AsymTopParams", path="plain", precision="fp64", with_params=False) -> "System":
        ap = AsymParams()
        ap.jmax, ap.A, ap.B, ap.C, ap.max_states, ap.mu = p.jmax, p.A, p.B, p.C, p.max_states, p.mu
        ap.n_terms = p.n_terms
        for t in range(p.n_terms):
            ap.lam[t], ap.mproj[t] = int(p.lam[t]), int(p.mproj[t])
            ap.coef[t], ap.beta[t] = float(p.coef[t]), float(p.beta[t])
        ap.c6, ap.rd, ap.n_grid, ap.r_min, ap.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
        ap.with_params = int(bool(with_params))
        ap.path, ap.precision = _PATHS[path], _PRECS[precision]
        tau = np.zeros((p.jmax + 1) ** 2, np.int32)
        ap.tau_out = tau.ctypes.data
        d = Desc()
        _check(lib().mqct_build_asym_top(C.byref(ap), C.byref(d)))
        try:
            s = cls(d)
        finally:
            lib().mqct_free_desc(C.byref(d))
        s.tau = tau[: int(s.level.max()) + 1].copy()
        return s

    def state(self, j, m) -> int:
        """State index of the (j, m) label (unique for a linear rotor)."""
        return self._index[(int(j), int(m))]

    def level_state(self, level, m) -> int:
        """State index of projection m in the given level."""
        return self._lindex[(int(level), int(m))]

    @property
    def info(self) -> dict:
        inf = Info()
        _check(lib().mqct_system_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    @property
    def handle(self):
        return self._h

    @property
    def n_levels(self) -> int:
        return self.info["n_levels"]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mqct_destroy_system(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_trajs(ts: "_inputs.TrajSet", systems) -> np.ndarray:
    """mqct_traj array for a TrajSet; initial states addressed by their (j, m) labels, or by
    (level, m) when ts.init_by == "level"."""
    systems = systems if isinstance(systems, (list, tuple)) else [systems]
    tr = np.zeros(ts.n, TRAJ_DTYPE)
    tr["e_coll"], tr["b"] = ts.e_coll, ts.b
    tr["r0"], tr["r_end"], tr["dt"], tr["max_steps"] = ts.r0, ts.r_end, ts.dt, ts.max_steps
    sidx = ts.system if len(ts.system) else np.zeros(ts.n, np.int32)
    tr["system_idx"] = sidx
    if ts.init_by == "level":
        tr["init_state"] = [systems[s].level_state(j, m) for s, j, m in zip(sidx, ts.init_j, ts.init_m)]
    else:
        tr["init_state"] = [systems[s].state(j, m) for s, j, m in zip(sidx, ts.init_j, ts.init_m)]
    return tr


def propagate(systems, trajs, want_pop=True, want_amp=False, want_diag=True, device=None, stream=None,
              allow_traj_status=True, batch_shape=0, tc_slots=0, timing=None):
    """Run mqct_propagate_ex.

    trajs: numpy TRAJ_DTYPE array (host) or a torch uint8 CUDA tensor holding the same bytes.
    device=True returns torch CUDA tensors (asynchronous); device=False returns numpy arrays.
    batch_shape / tc_slots: launch-shape options, one value or one per system (0 = automatic,
    see mqct_propagate_opts).
    timing: optional pair (t_start, t_done) of int64 arrays (numpy or CUDA tensors) of length n
    that receive each trajectory's start and finish time on the GPU clock (ns).
    Returns (pop [n][N_max], amp [n][N_max] complex, diag) with None for outputs not requested."""
    systems = systems if isinstance(systems, (list, tuple)) else [systems]
    hs = (C.c_void_p * len(systems))(*[s.handle.value for s in systems])
    nmax = max(s.n for s in systems)
    if isinstance(trajs, np.ndarray):
        n = trajs.shape[0]
    else:
        n = trajs.numel() // TRAJ_DTYPE.itemsize
    if device is None:
        device = not isinstance(trajs, np.ndarray)
    pop = amp = diag = None
    if device:
        import torch

        dev = torch.device("cuda")
        if want_pop:
            pop = torch.empty((n, nmax), dtype=torch.float64, device=dev)
        if want_amp:
            amp = torch.empty((n, nmax, 2), dtype=torch.float64, device=dev)
        if want_diag:
            diag = torch.empty((n * DIAG_DTYPE.itemsize,), dtype=torch.uint8, device=dev)
    else:
        if want_pop:
            pop = np.zeros((n, nmax))
        if want_amp:
            amp = np.zeros((n, nmax, 2))
        if want_diag:
            diag = np.zeros(n, DIAG_DTYPE)
    op = PropagateOpts()
    ns = len(systems)
    shapes = np.ascontiguousarray(np.broadcast_to(np.asarray(batch_shape, np.int32), (ns,)))
    slots = np.ascontiguousarray(np.broadcast_to(np.asarray(tc_slots, np.int32), (ns,)))
    op.batch_shape, op.tc_slots = shapes.ctypes.data, slots.ctypes.data
    if timing is not None:
        op.t_start_ns, op.t_done_ns = _ptr(timing[0]), _ptr(timing[1])
    st = lib().mqct_propagate_ex(hs, len(systems), _ptr(trajs), n, _ptr(pop), _ptr(amp), _ptr(diag), C.byref(op),
                                 _stream(stream))
    _check(st, allow=(ERR_TRAJ,) if allow_traj_status else ())
    if amp is not None and not device:
        amp = amp[..., 0] + 1j * amp[..., 1]
    return pop, amp, diag


def diag_to_numpy(diag) -> np.ndarray:
    if isinstance(diag, np.ndarray):
        return diag
    return diag.cpu().numpy().view(DIAG_DTYPE)


def cross_sections(system: System, pop, weight, group, n_groups: int, stream=None):
    """sigma[g][level] = sum_{t in g} weight_t sum_{s in level} pop_t[s] (device reduction)."""
    n = pop.shape[0]
    if isinstance(pop, np.ndarray):
        pop = np.ascontiguousarray(pop, np.float64)
        weight = np.ascontiguousarray(weight, np.float64)
        group = np.ascontiguousarray(group, np.int32)
        sig = np.zeros((n_groups, system.n_levels))
    else:
        import torch

        sig = torch.empty((n_groups, system.n_levels), dtype=torch.float64, device=pop.device)
    _check(lib().mqct_cross_sections(system.handle, _ptr(pop), _ptr(weight), _ptr(group), n, n_groups, _ptr(sig),
                                     _stream(stream)))
    return sig


def sigma_weights(ts: "_inputs.TrajSet", status=None) -> np.ndarray:
    """Per-trajectory weights of the cross-section quadrature (Sec. III sampling):
    regular midpoint grid 2 pi b db (divided by 2j'+1 when every m' is run), Monte-Carlo
    2 pi b_max b / (trajectories in the group); trajectories with MAX_STEPS / NONFINITE /
    INVALID status get weight 0."""
    if ts.sampling == "regular":
        w = 2.0 * np.pi * ts.b * (ts.b_max / ts.n_b)
        if ts.m_avg == "all":
            w = w / (2 * ts.init_j + 1)
    else:
        counts = np.bincount(ts.group, minlength=ts.n_groups).astype(np.float64)
        w = 2.0 * np.pi * ts.b_max * ts.b / counts[ts.group]
    if status is not None:
        bad = (np.asarray(status) & (TRAJ_MAX_STEPS | TRAJ_NONFINITE | TRAJ_INVALID | TRAJ_TIMEOUT)) != 0
        w = np.where(bad, 0.0, w)
    return w


def last_launch_count() -> int:
    """Kernel launches of the library made by the last propagate / cross-section / adjoint / rate call
    on this thread (mqct_last_launch_count)."""
    return int(lib().mqct_last_launch_count())


def rate_coefficients(sigma, u, level_energy, degeneracy, mu: float, kT, sigma_sym: bool = True, stream=None):
    """Eq. 20 and the Maxwell-Boltzmann rate coefficients of both directions of every pair of levels
    (mqct_rate_coefficients).  sigma[k][a][b] = sigma_{a->b}(U_k) in bohr^2 (numpy or a CUDA tensor);
    u [K], kT [n_T] in hartree; level_energy [L] (hartree), degeneracy [L].  Returns (sigma_sym or
    None, rate) with rate[t][a][b] = k_{a->b}(T_t) in bohr^3 per atomic unit of time, on the
    device of sigma."""
    u = np.ascontiguousarray(u, np.float64)
    kT = np.ascontiguousarray(np.atleast_1d(kT), np.float64)
    E = np.ascontiguousarray(level_energy, np.float64)
    g = np.ascontiguousarray(degeneracy, np.float64)
    K, L = len(u), len(E)
    if tuple(sigma.shape) != (K, L, L) or len(g) != L:
        raise ValueError("sigma must be [K][L][L] with K energies and L levels")
    if isinstance(sigma, np.ndarray):
        sigma = np.ascontiguousarray(sigma, np.float64)
        sym = np.zeros((K, L, L)) if sigma_sym else None
        rate = np.zeros((len(kT), L, L))
    else:
        import torch

        sigma = sigma.contiguous().to(torch.float64)
        sym = torch.empty((K, L, L), dtype=torch.float64, device=sigma.device) if sigma_sym else None
        rate = torch.empty((len(kT), L, L), dtype=torch.float64, device=sigma.device)
    d = RateDesc(L, K, len(kT), 0, float(mu), u.ctypes.data, kT.ctypes.data, E.ctypes.data, g.ctypes.data)
    _check(lib().mqct_rate_coefficients(C.byref(d), _ptr(sigma), _ptr(sym), _ptr(rate), _stream(stream)))
    return sym, rate


def adjoint(system: System, trajs: np.ndarray, weight, group, n_groups: int, dL_dsigma, ckpt: int = 64,
            stream=None) -> np.ndarray:
    """dL/dtheta for L = sum dL_dsigma[g][l] sigma[g][l] by the discrete adjoint of the RK4 map
    (mqct_adjoint); theta are the parameters whose tables the system was built with."""
    weight = np.ascontiguousarray(weight, np.float64)
    group = np.ascontiguousarray(group, np.int32)
    dls = np.ascontiguousarray(dL_dsigma, np.float64)
    out = np.zeros(system.n_params)
    _check(lib().mqct_adjoint(system.handle, _ptr(trajs), trajs.shape[0], _ptr(weight), _ptr(group), n_groups,
                              _ptr(dls), int(ckpt), _ptr(out), _stream(stream)), allow=(ERR_TRAJ,))
    return out


def _diatom_with(p, theta):
    """Copy of a DiatomParams with theta = (A_0..A_{L-1}, beta_0..beta_{L-1})."""
    import copy

    q = copy.copy(p)
    L = p.n_terms
    th = np.asarray(theta, np.float64)
    q.A = th[:L].copy()
    q.beta = th[L:2 * L].copy()
    return q


def cross_section_fn(precision="fp64"):
    """torch.autograd.Function computing the cross sections of a diatom workload as a function
    of theta = (A, beta); backward runs the adjoint kernel (FP64, or the mixed adjoint with
    precision="fp32").

        sigma = CrossSection.apply(theta, params, trajset, ckpt)
    theta: float64 CPU tensor [2L]; returns sigma [n_groups][n_levels] (float64, CPU)."""
    import torch

    class CrossSection(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, params, ts, ckpt=64):
            p = _diatom_with(params, theta.detach().cpu().numpy())
            sys_ = System.diatom(p, path="factorised", precision=precision, with_params=True)
            tr = make_trajs(ts, sys_)
            pop, _, diag = propagate(sys_, tr, device=False)
            w = sigma_weights(ts, diag["status"])
            sig = cross_sections(sys_, pop, w, ts.group, ts.n_groups)
            ctx.sys, ctx.tr, ctx.w, ctx.ts, ctx.ckpt = sys_, tr, w, ts, ckpt
            return torch.from_numpy(sig)

        @staticmethod
        def backward(ctx, g):
            d = adjoint(ctx.sys, ctx.tr, ctx.w, ctx.ts.group, ctx.ts.n_groups, g.detach().cpu().numpy(), ctx.ckpt)
            return torch.from_numpy(d), None, None, None

    return CrossSection


def fma_rate(kind: str = "fp64", stream=None) -> float:
    """Measured FMA throughput of the current GPU in GFLOP/s ("fp64" or "fp32")."""
    out = C.c_double()
    _check(lib().mqct_probe_fma_rate({"fp64": 0, "fp32": 1}[kind], C.byref(out), _stream(stream)))
    return out.value


def op_latency(kind: str = "dfma", warps: int = 1, stream=None) -> float:
    """SM clock cycles per operation of a dependent chain ("dfma", "ffma", "ddiv", "cvt"), with
    `warps` warps of one CTA running chains at once (mqct_probe_op_latency)."""
    out = C.c_double()
    k = {"dfma": 0, "ffma": 1, "ddiv": 2, "cvt": 3}[kind]
    _check(lib().mqct_probe_op_latency(k, int(warps), C.byref(out), _stream(stream)))
    return out.value


def version() -> str:
    return lib().mqct_version().decode()
