"""C-ABI library checks that need no GPU: it loads, exports every declared symbol, its
structs match the binding, and its host-side logic (the built-in system builder, input
validation) behaves.  No compute call is made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2312_02322_gb300 import api, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2312_02322_gb300 import build

    build.build()
    return api.lib()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    names = set()
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(mqct_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "mqct_propagate" in names and "mqct_adjoint" in names and "mqct_cross_sections" in names
    for name in names:
        assert hasattr(L, name), name


def test_version_and_last_error(L):
    assert "sm_103a" in api.version()
    d = api.Desc()
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_INVALID_ARG
    assert b"n_states" in L.mqct_last_error()


def build_desc(jmax=3, path="plain", with_params=False, n_grid=40):
    p = inputs.diatom_pes_params(jmax=jmax, n_grid=n_grid)
    dp = api.DiatomParams()
    dp.jmax, dp.bconst, dp.mu, dp.n_terms = p.jmax, p.bconst, p.mu, p.n_terms
    for i in range(p.n_terms):
        dp.A[i], dp.beta[i] = p.A[i], p.beta[i]
    dp.c6, dp.rd, dp.n_grid, dp.r_min, dp.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
    dp.with_params = int(with_params)
    dp.path = api._PATHS[path]
    d = api.Desc()
    assert api.lib().mqct_build_diatom(C.byref(dp), C.byref(d)) == 0
    return d, p


def dense_G(d):
    n, L = d.n_states, d.n_terms
    G = np.zeros((L, n, n))
    t = np.ctypeslib.as_array(C.cast(d.g_term, C.POINTER(C.c_int32)), (d.g_nnz,))
    r = np.ctypeslib.as_array(C.cast(d.g_row, C.POINTER(C.c_int32)), (d.g_nnz,))
    c = np.ctypeslib.as_array(C.cast(d.g_col, C.POINTER(C.c_int32)), (d.g_nnz,))
    v = np.ctypeslib.as_array(C.cast(d.g_val, C.POINTER(C.c_double)), (d.g_nnz,))
    np.add.at(G, (t, r, c), v)
    return G


def test_builder_coupling_matches_oracle(L, ora):
    """The library's quadrature-built G^lambda (Eq. 15) agrees with the oracle's Racah-formula G."""
    for jmax in (3, 12, 39):
        d, p = build_desc(jmax)
        G = dense_G(d)
        for lam in range(5):
            assert np.max(np.abs(G[lam] - ora.diatom_G(jmax, lam))) < 1e-13
        e = np.ctypeslib.as_array(C.cast(d.energy, C.POINTER(C.c_double)), (d.n_states,))
        e2, lev, jq, mq = ora.diatom_basis(jmax, p.bconst)
        assert np.array_equal(e, e2)
        api.lib().mqct_free_desc(C.byref(d))


def build_asym(p, with_params=False, tau=None):
    ap = api.AsymParams()
    ap.jmax, ap.A, ap.B, ap.C, ap.max_states, ap.mu = p.jmax, p.A, p.B, p.C, p.max_states, p.mu
    ap.n_terms = p.n_terms
    for t in range(p.n_terms):
        ap.lam[t], ap.mproj[t], ap.coef[t], ap.beta[t] = int(p.lam[t]), int(p.mproj[t]), p.coef[t], p.beta[t]
    ap.c6, ap.rd, ap.n_grid, ap.r_min, ap.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
    ap.with_params = int(with_params)
    ap.tau_out = None if tau is None else tau.ctypes.data
    d = api.Desc()
    st = api.lib().mqct_build_asym_top(C.byref(ap), C.byref(d))
    return st, d, ap


def test_asym_builder_matches_oracle_at_full_size(L, ora):
    """Library: Wang classes by Sturm bisection + inverse iteration, G by quadrature of Wigner d
    over beta.  Oracle: Jacobi rotations, G by the Eq. 16 closed form.  Same basis order, labels,
    eigenvector signs and coupling matrices on the N = 1580 workload (28 terms)."""
    p = inputs.asym_pes_params()
    tau = np.zeros((p.jmax + 1) ** 2, np.int32)
    st, d, _ = build_asym(p, tau=tau)
    assert st == 0
    lj, lt, le, lb = ora.asym_basis(p.jmax, p.A, p.B, p.C, p.max_states)
    e2, lev2, jq2, mq2 = ora.asym_states(lj, le)
    n = d.n_states
    assert n == len(e2) == 1580
    arr = lambda ptr, t: np.ctypeslib.as_array(C.cast(ptr, C.POINTER(t)), (n,))
    assert np.allclose(arr(d.energy, C.c_double), e2, rtol=1e-13, atol=0)
    assert np.array_equal(arr(d.level, C.c_int32), lev2)
    assert np.array_equal(arr(d.j, C.c_int32), jq2)
    assert np.array_equal(arr(d.m, C.c_int32), mq2)
    assert np.array_equal(tau[: len(lt)], lt)
    G = dense_G(d)
    for t in range(p.n_terms):
        Go = ora.asym_G(lj, lb, p.jmax, int(p.lam[t]), int(p.mproj[t]))
        assert np.max(np.abs(G[t] - Go)) < 1e-12, (p.lam[t], p.mproj[t])
    v = np.ctypeslib.as_array(C.cast(d.v, C.POINTER(C.c_double)), (p.n_terms, p.n_grid))
    v2, _, _, _ = ora.diatom_pes(p.coef, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max)
    assert np.allclose(v, v2, rtol=1e-14, atol=0)
    api.lib().mqct_free_desc(C.byref(d))


@pytest.mark.parametrize("field,value", [("jmax", 21), ("C", 1.0), ("max_states", 0), ("n_terms", 65)])
def test_asym_builder_validation(L, field, value):
    p = inputs.asym_pes_params(jmax=3, max_states=30, lam_max=2)
    ap_ok = build_asym(p)
    assert ap_ok[0] == 0
    api.lib().mqct_free_desc(C.byref(ap_ok[1]))
    st, d, ap = build_asym(p)
    api.lib().mqct_free_desc(C.byref(d))
    setattr(ap, field, value)
    assert L.mqct_build_asym_top(C.byref(ap), C.byref(d)) == api.ERR_INVALID_ARG
    ap.jmax, ap.C, ap.max_states, ap.n_terms = p.jmax, p.C, p.max_states, p.n_terms
    ap.mproj[1] = 2  # mu > lambda = 1
    assert L.mqct_build_asym_top(C.byref(ap), C.byref(d)) == api.ERR_INVALID_ARG
    assert b"mu <= lambda" in L.mqct_last_error()


def test_builder_pes_matches_oracle(L, ora):
    d, p = build_desc(4, with_params=True, n_grid=60)
    v = np.ctypeslib.as_array(C.cast(d.v, C.POINTER(C.c_double)), (5, 60))
    ends = np.ctypeslib.as_array(C.cast(d.dv_ends, C.POINTER(C.c_double)), (5, 2))
    dvp = np.ctypeslib.as_array(C.cast(d.dv_dparam, C.POINTER(C.c_double)), (10, 5, 60))
    dvpe = np.ctypeslib.as_array(C.cast(d.ddv_ends, C.POINTER(C.c_double)), (10, 5, 2))
    v2, e2, dvp2, dvpe2 = ora.diatom_pes(p.A, p.beta, p.c6, p.rd, 60, p.r_min, p.r_max, with_params=True)
    assert np.allclose(v, v2, rtol=1e-14, atol=0)
    assert np.allclose(ends, e2, rtol=1e-12, atol=1e-30)
    assert np.allclose(dvp, dvp2, rtol=1e-14, atol=0)
    assert np.allclose(dvpe, dvpe2, rtol=1e-12, atol=1e-30)
    api.lib().mqct_free_desc(C.byref(d))


def test_prescribed_flag_needs_fp64(L):
    d, _ = build_desc(2, path="factorised")
    d.flags = api.PRESCRIBED_TRAJ
    d.precision = api.FP32
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_UNSUPPORTED
    assert b"PRESCRIBED" in L.mqct_last_error()
    assert not h.value
    api.lib().mqct_free_desc(C.byref(d))


def test_builder_coupling_matches_oracle_at_paper_size(L, ora):
    """jmax = 446 (N = 199 809, the largest basis the paper-scale tests run): the library's
    Gauss-Legendre Gaunt integrals agree with the oracle's Racah-formula G^lambda to 1e-12 on every
    entry of lambda = 0, 1, 6, 12; entries only the library lists are accidental zeros of the
    Clebsch-Gordan coefficient (below 1e-15), which the oracle drops."""
    p = inputs.sparse_pes_params(jmax=446, lam_max=12)
    dp = api.DiatomParams()
    dp.jmax, dp.bconst, dp.mu, dp.n_terms = p.jmax, p.bconst, p.mu, len(p.A)
    for i in range(len(p.A)):
        dp.A[i], dp.beta[i] = p.A[i], p.beta[i]
    dp.c6, dp.rd, dp.n_grid, dp.r_min, dp.r_max = p.c6, p.rd, p.n_grid, p.r_min, p.r_max
    dp.path, dp.grid_kind = api._PATHS["plain"], api.GRID_LOG
    d = api.Desc()
    assert L.mqct_build_diatom(C.byref(dp), C.byref(d)) == 0
    nnz = d.g_nnz
    get = lambda f, t: np.ctypeslib.as_array(C.cast(getattr(d, f), C.POINTER(t)), (nnz,)).copy()
    t, r, c, v = get("g_term", C.c_int32), get("g_row", C.c_int32), get("g_col", C.c_int32), get("g_val", C.c_double)
    assert d.n_states == 199809
    api.lib().mqct_free_desc(C.byref(d))
    for lam in (0, 1, 6, 12):
        orow, ocol, oval = ora.diatom_G_triplets(446, lam)
        m = t == lam
        kl = r[m].astype(np.int64) * 1_000_000 + c[m]
        ko = orow.astype(np.int64) * 1_000_000 + ocol
        keys = np.union1d(kl, ko)
        vl, vo = np.zeros(keys.size), np.zeros(keys.size)
        vl[np.searchsorted(keys, kl)] = v[m]
        vo[np.searchsorted(keys, ko)] = oval
        assert np.max(np.abs(vl - vo)) < 1e-12, lam
        only_lib = ~np.isin(keys, ko)
        assert not np.any(~np.isin(keys, kl)), lam
        assert np.all(np.abs(vl[only_lib]) < 1e-15), lam


@pytest.mark.parametrize("field,value,needle", [
    ("n_grid", 3, b"n_grid"),
    ("mu", -1.0, b"mu"),
    ("n_terms", 0, b"n_terms"),
    ("path", 7, b"path"),
    ("flags", 6, b"flags"),
])
def test_create_validation_rejects_before_gpu(L, field, value, needle):
    d, _ = build_desc(2)
    setattr(d, field, value)
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_INVALID_ARG
    assert needle in L.mqct_last_error()
    assert not h.value
    setattr(d, "n_grid", 40)
    api.lib().mqct_free_desc(C.byref(d))


def test_create_rejects_coupling_across_m(L):
    n = 2
    e = np.zeros(n)
    lev = np.array([0, 1], np.int32)
    j = np.array([1, 1], np.int32)
    m = np.array([0, 1], np.int32)
    G = np.array([[[0.0, 1.0], [1.0, 0.0]]])
    v = np.zeros((1, 8))
    ends = np.zeros((1, 2))
    d = api.Desc()
    d.n_states, d.energy, d.level, d.j, d.m = n, e.ctypes.data, lev.ctypes.data, j.ctypes.data, m.ctypes.data
    d.mu, d.n_terms, d.G = 100.0, 1, G.ctypes.data
    d.n_grid, d.r_min, d.r_max, d.v, d.dv_ends = 8, 2.0, 30.0, v.ctypes.data, ends.ctypes.data
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_INVALID_ARG
    assert b"different m" in L.mqct_last_error()
    m[1] = 0
    G[0, 0, 1] = 0.5  # not symmetric
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_INVALID_ARG
    assert b"symmetric" in L.mqct_last_error()


def test_create_sums_duplicate_triplets(L):
    """Triplet G: repeated (term, row, column) entries are summed before the symmetry check, so
    (0, 1) given as 0.25 + 0.25 against (1, 0) = 0.5 passes validation (on a machine without a GPU
    the call then stops at the first device allocation), and 0.25 alone is rejected."""
    n = 2
    e = np.zeros(n)
    lev = np.array([0, 1], np.int32)
    j = np.array([1, 1], np.int32)
    m = np.zeros(n, np.int32)
    v = np.zeros((1, 8))
    ends = np.zeros((1, 2))
    term = np.zeros(3, np.int32)
    row = np.array([0, 1, 0], np.int32)
    col = np.array([1, 0, 1], np.int32)
    val = np.array([0.25, 0.5, 0.25])
    d = api.Desc()
    d.n_states, d.energy, d.level, d.j, d.m = n, e.ctypes.data, lev.ctypes.data, j.ctypes.data, m.ctypes.data
    d.mu, d.n_terms, d.G = 100.0, 1, None
    d.g_nnz, d.g_term, d.g_row, d.g_col, d.g_val = 3, term.ctypes.data, row.ctypes.data, col.ctypes.data, val.ctypes.data
    d.n_grid, d.r_min, d.r_max, d.v, d.dv_ends = 8, 2.0, 30.0, v.ctypes.data, ends.ctypes.data
    h = C.c_void_p()
    st = L.mqct_create_system(C.byref(d), C.byref(h))
    assert st != api.ERR_INVALID_ARG, L.mqct_last_error()
    if st == api.OK:
        L.mqct_destroy_system(h)
    d.g_nnz = 2  # (0, 1) = 0.25 only
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == api.ERR_INVALID_ARG
    assert b"symmetric" in L.mqct_last_error()


def test_struct_layouts_match_header(L, tmp_path):
    """Compile a probe against include/mqct.h with gcc and compare sizes and offsets with the binding."""
    import subprocess

    src = tmp_path / "layout.c"
    checks = {
        "mqct_system_desc": (api.Desc, ["n_states", "energy", "mu", "n_terms", "G", "g_nnz", "g_val", "n_grid",
                                        "r_min", "v", "n_params", "ddv_ends", "path", "flags"]),
        "mqct_system_info_t": (api.Info, ["n_states", "table_nnz", "device_bytes", "n_coupling_terms",
                                          "n_row_tiles", "tc_kchunks"]),
        "mqct_diatom_params": (api.DiatomParams, ["jmax", "bconst", "mu", "n_terms", "A", "beta", "c6", "rd",
                                                  "n_grid", "r_min", "with_params", "path", "precision"]),
        "mqct_propagate_opts": (api.PropagateOpts, ["t_start_ns", "t_done_ns", "batch_shape", "tc_slots"]),
        "mqct_asym_params": (api.AsymParams, ["jmax", "A", "B", "C", "max_states", "mu", "n_terms", "lam", "mproj",
                                              "coef", "beta", "c6", "rd", "n_grid", "r_min", "r_max",
                                              "with_params", "path", "precision", "tau_out"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mqct.h"', "int main(void) {"]
    for st, (_, fields) in checks.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append('printf("mqct_traj %zu\\n", sizeof(mqct_traj));')
    for f in api.TRAJ_DTYPE.names[:-1]:
        lines.append(f'printf("mqct_traj.{f} %zu\\n", offsetof(mqct_traj, {f}));')
    lines.append('printf("mqct_diag %zu\\n", sizeof(mqct_diag));')
    for f in api.DIAG_DTYPE.names:
        lines.append(f'printf("mqct_diag.{f} %zu\\n", offsetof(mqct_diag, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)]).decode().split("\n") if l)
    for st, (cls, fields) in checks.items():
        assert int(out[st]) == C.sizeof(cls), st
        for f in fields:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
    assert int(out["mqct_traj"]) == api.TRAJ_DTYPE.itemsize
    for f in api.TRAJ_DTYPE.names[:-1]:
        assert int(out[f"mqct_traj.{f}"]) == api.TRAJ_DTYPE.fields[f][1], f
    assert int(out["mqct_diag"]) == api.DIAG_DTYPE.itemsize
    for f in api.DIAG_DTYPE.names:
        assert int(out[f"mqct_diag.{f}"]) == api.DIAG_DTYPE.fields[f][1], f


@pytest.mark.parametrize("path,prec,grid,thr,status,needle", [
    ("plain", api.FP64, 2, 0.0, api.ERR_INVALID_ARG, b"grid_kind"),
    ("factorised", api.FP32, api.GRID_LOG, 0.0, api.ERR_UNSUPPORTED, b"GRID_LOG"),
    ("factorised", api.BF16X3, api.GRID_LOG, 0.0, api.ERR_UNSUPPORTED, b"GRID_LOG"),
    ("factorised", api.FP64, api.GRID_UNIFORM, 1e-5, api.ERR_UNSUPPORTED, b"truncation"),
    ("plain", api.FP64, api.GRID_UNIFORM, float("nan"), api.ERR_INVALID_ARG, b"trunc_threshold"),
])
def test_grid_and_truncation_validation(L, path, prec, grid, thr, status, needle):
    """The logarithmic grid and the truncation (Sec. III) are rejected where no kernel runs them."""
    d, _ = build_desc(2, path=path)
    d.precision = prec
    d.grid_kind = grid
    d.trunc_threshold = thr
    d.trunc_r[0], d.trunc_r[1] = 6.03, 7.11
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == status
    assert needle in L.mqct_last_error()
    assert not h.value
    api.lib().mqct_free_desc(C.byref(d))


@pytest.mark.parametrize("flags,prec,status,needle", [
    (api.PRESCRIBED_TRAJ | api.DECOUPLED_TRAJ, api.FP64, api.ERR_INVALID_ARG, b"exclude"),
    (api.DECOUPLED_TRAJ, api.FP32, api.ERR_UNSUPPORTED, b"DECOUPLED"),
])
def test_decoupled_flag_validation(L, flags, prec, status, needle):
    d, _ = build_desc(2, path="factorised")
    d.flags = flags
    d.precision = prec
    h = C.c_void_p()
    assert L.mqct_create_system(C.byref(d), C.byref(h)) == status
    assert needle in L.mqct_last_error()
    assert not h.value
    api.lib().mqct_free_desc(C.byref(d))


def _oracle_molmol(ora, p):
    lev_J, lev_E, lev_b = [], [], []
    for J in range(p.j1max + 1):
        E, b = ora.asym_levels(J, p.A, p.B, p.C)
        for e_, bb in zip(E, b):
            row = np.zeros(2 * p.j1max + 1)
            row[p.j1max - J:p.j1max + J + 1] = bb
            lev_J.append(J); lev_E.append(e_); lev_b.append(row)
    lev_J = np.array(lev_J, np.int32)
    e, lev, jt, mt, l1, j2 = ora.molmol_states(lev_J, p.j2, lev_E, p.bconst2)
    G = np.stack([ora.molmol_G(lev_J, np.array(lev_b), p.j1max, l1, j2, jt, mt, *t) for t in p.terms])
    return e, lev, jt, mt, G


@pytest.mark.parametrize("j1max,j2", [(2, (0, 2)), (3, (0, 1, 2))])
def test_molmol_builder_matches_oracle(L, ora, j1max, j2):
    """Asymmetric top + linear rotor: the library's composite states (Eq. 3) and coupling -- its own
    Clebsch-Gordan coefficients by the lowering-operator construction and its one-molecule integrals
    by quadrature -- agree with the oracle's Racah-formula algebra of Eqs. 15-17."""
    p = inputs.molmol_params(j1max=j1max, j2=j2)
    mp = api.System.molmol_params(p)
    d = api.Desc()
    assert L.mqct_build_molmol(C.byref(mp), C.byref(d)) == 0
    n = d.n_states
    arr = lambda ptr, t: np.ctypeslib.as_array(C.cast(ptr, C.POINTER(t)), (n,))
    e, lev, jt, mt, Go = _oracle_molmol(ora, p)
    assert n == len(e)
    assert np.allclose(arr(d.energy, C.c_double), e, rtol=1e-13, atol=0)
    assert np.array_equal(arr(d.level, C.c_int32), lev)
    assert np.array_equal(arr(d.j, C.c_int32), jt)
    assert np.array_equal(arr(d.m, C.c_int32), mt)
    G = dense_G(d)
    for t in range(p.n_terms):
        assert np.max(np.abs(G[t] - Go[t])) < 1e-12, p.terms[t]
    api.lib().mqct_free_desc(C.byref(d))
