"""Adjoint (cross-section gradients with respect to the PES parameters A_l, beta_l):
the GPU discrete adjoint against the oracle's forward tangent of the same RK4 map (1e-8
relative) and against central finite differences of the GPU forward path (1e-5 relative)."""
import numpy as np
import pytest

from paper_2312_02322_gb300 import inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02322_gb300 import api, build

    build.build()
    return api


def case(jmax=3, n_b=3, energies=(700.0,), init_js=(0, 1)):
    return W.small_workload(jmax=jmax, n_b=n_b, energies=energies, init_js=init_js, b_max=7.0, n_grid=120,
                            m_avg="one")


def dsigma_oracle(ora, p, ts, w):
    osys = ora.diatom_system(p.jmax, p.bconst, p.mu, p.A, p.beta, p.c6, p.rd, p.n_grid, p.r_min, p.r_max,
                             with_params=True)
    init = [j * j + j + m for j, m in zip(ts.init_j, ts.init_m)]
    amp, dpop, res = ora.tangent(osys, ts.e_coll, ts.b, init, dt=ts.dt)
    P = dpop.shape[1]
    dsig = np.zeros((P, ts.n_groups, osys.n_levels))
    for t in range(ts.n):
        for s in range(osys.n):
            dsig[:, ts.group[t], osys.level[s]] += w[t] * dpop[t, :, s]
    return dsig


@pytest.mark.parametrize("ckpt", [64, 7])
def test_adjoint_matches_oracle_tangent(mq, ora, ckpt):
    p, ts = case()
    sys_ = mq.System.diatom(p, path="factorised", with_params=True)
    tr = mq.make_trajs(ts, sys_)
    _, _, diag = mq.propagate(sys_, tr, device=False)
    w = mq.sigma_weights(ts, diag["status"])
    rng = np.random.default_rng(3)
    dls = rng.standard_normal((ts.n_groups, sys_.n_levels))
    g = mq.adjoint(sys_, tr, w, ts.group, ts.n_groups, dls, ckpt=ckpt)
    dsig = dsigma_oracle(ora, p, ts, w)
    want = np.einsum("pgl,gl->p", dsig, dls)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(g - want)) < 1e-8 * scale, (g, want)


def test_adjoint_matches_central_differences(mq):
    p, ts = case(jmax=3, n_b=2, energies=(900.0,), init_js=(1,))
    th0 = np.concatenate([p.A, p.beta])
    sys_ = mq.System.diatom(p, path="factorised", with_params=True)
    tr = mq.make_trajs(ts, sys_)
    _, _, diag = mq.propagate(sys_, tr, device=False)
    w = mq.sigma_weights(ts, diag["status"])
    rng = np.random.default_rng(5)
    dls = rng.standard_normal((ts.n_groups, sys_.n_levels))
    g = mq.adjoint(sys_, tr, w, ts.group, ts.n_groups, dls, ckpt=16)

    def loss(th):
        q = mq._diatom_with(p, th)
        s2 = mq.System.diatom(q, path="factorised")
        pop, _, d2 = mq.propagate(s2, mq.make_trajs(ts, s2), device=False)
        return float(np.sum(dls * mq.cross_sections(s2, pop, w, ts.group, ts.n_groups))), d2["steps"]

    for k in range(len(th0)):
        h = 1e-5 * abs(th0[k])
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        lp, sp = loss(tp)
        lm, sm = loss(tm)
        assert np.array_equal(sp, sm) and np.array_equal(sp, diag["steps"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g[k]), 1e-3 * np.max(np.abs(g))), (k, fd, g[k])


def test_autograd_function(mq):
    """CrossSection.backward returns the adjoint's vector-Jacobian product for the upstream
    gradient torch hands it: equal to mqct_adjoint called directly with the same weights, and to
    central differences (h = 1e-5 relative) of the forward through the same function."""
    import torch

    p, ts = case(jmax=2, n_b=2, energies=(800.0,), init_js=(0,))
    CS = mq.cross_section_fn()
    th0 = np.concatenate([p.A, p.beta])
    th = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    sig = CS.apply(th, p, ts, 32)
    wts = torch.arange(sig.numel(), dtype=torch.float64).reshape(sig.shape) - 0.3 * sig.numel()
    L = (sig * wts).sum()
    L.backward()
    assert th.grad is not None and th.grad.shape == th.shape
    # the same VJP through the C ABI directly
    sys_ = mq.System.diatom(p, path="factorised", with_params=True)
    tr = mq.make_trajs(ts, sys_)
    _, _, diag = mq.propagate(sys_, tr, device=False)
    w = mq.sigma_weights(ts, diag["status"])
    direct = mq.adjoint(sys_, tr, w, ts.group, ts.n_groups, wts.numpy(), ckpt=32)
    g = th.grad.numpy()
    assert np.max(np.abs(g - direct)) <= 1e-12 * np.max(np.abs(direct))
    # central differences of the loss through the autograd function's forward
    for k in (0, 1, len(th0) - 1):
        h = 1e-5 * abs(th0[k])
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        lp = float((CS.apply(torch.tensor(tp), p, ts, 32) * wts).sum())
        lm = float((CS.apply(torch.tensor(tm), p, ts, 32) * wts).sum())
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g[k]), 1e-3 * np.max(np.abs(g))), (k, fd, g[k])


def test_mixed_adjoint_matches_fp64_adjoint(mq):
    """The mixed adjoint (FP32 amplitudes and cotangents, compensated step update, FP64 classical
    motion and parameter gradient) against the FP64 adjoint of the same trajectories and weights."""
    p, ts = case(jmax=4, n_b=3, energies=(700.0,), init_js=(0, 1))
    s64 = mq.System.diatom(p, path="factorised", precision="fp64", with_params=True)
    s32 = mq.System.diatom(p, path="factorised", precision="fp32", with_params=True)
    tr = mq.make_trajs(ts, s64)
    _, _, diag = mq.propagate(s64, tr, device=False)
    w = mq.sigma_weights(ts, diag["status"])
    rng = np.random.default_rng(11)
    dls = rng.standard_normal((ts.n_groups, s64.n_levels))
    g64 = mq.adjoint(s64, tr, w, ts.group, ts.n_groups, dls, ckpt=16)
    g32 = mq.adjoint(s32, tr, w, ts.group, ts.n_groups, dls, ckpt=16)
    err = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    assert err < 1e-3, err


def test_adjoint_28_terms_matches_oracle_tangent(mq, ora):
    """More than 16 expansion terms: the atom + asymmetric top with all cos-type terms lam <= 6
    (28 terms, 56 parameters), FP64 adjoint against the oracle's forward tangent (1e-8)."""
    p, ts = W.small_asym_workload(jmax=4, max_states=60, lam_max=6, energies=(1500.0,), n_per_e=3, b_max=6.0)
    ts.r0 = ts.r_end = 14.0
    assert p.n_terms == 28
    sys_ = mq.System.asym_top(p, path="factorised", with_params=True)
    tr = mq.make_trajs(ts, sys_)
    _, _, diag = mq.propagate(sys_, tr, device=False)
    assert np.all(diag["status"] == 0)
    w = mq.sigma_weights(ts, diag["status"])
    rng = np.random.default_rng(12)
    dls = rng.standard_normal((ts.n_groups, sys_.n_levels))
    g = mq.adjoint(sys_, tr, w, ts.group, ts.n_groups, dls, ckpt=32)
    osys = ora.asym_system(p, with_params=True)
    lab = {(int(l), int(m)): i for i, (l, m) in enumerate(zip(osys.level, osys.mq))}
    init = [lab[(int(l), int(m))] for l, m in zip(ts.init_j, ts.init_m)]
    amp, dpop, res = ora.tangent(osys, ts.e_coll, ts.b, init, r0=ts.r0, r_end=ts.r_end, dt=ts.dt)
    assert np.array_equal(res["steps"], diag["steps"])
    want = np.zeros(dpop.shape[1])
    for t in range(ts.n):
        for s in range(osys.n):
            want += w[t] * dpop[t, :, s] * dls[ts.group[t], osys.level[s]]
    assert np.max(np.abs(g - want)) < 1e-8 * np.max(np.abs(want))


def test_adjoint_with_work_vectors_in_global_memory(mq):
    """N = 784 (j <= 27): the FP64 adjoint's work vectors exceed shared memory and live in global
    memory; central differences (h = 1e-5 relative) of the forward path agree to 1e-5."""
    p = W.diatom_pes_params(jmax=27, n_grid=200)
    ts = W.regular_set([3000.0], [0], n_b=2, b_max=6.0, m_avg="one", r0=14.0)
    sys_ = mq.System.diatom(p, path="factorised", with_params=True)
    tr = mq.make_trajs(ts, sys_)
    _, _, diag = mq.propagate(sys_, tr, device=False)
    assert np.all(diag["status"] == 0)
    w = mq.sigma_weights(ts, diag["status"])
    rng = np.random.default_rng(13)
    dls = rng.standard_normal((ts.n_groups, sys_.n_levels))
    g = mq.adjoint(sys_, tr, w, ts.group, ts.n_groups, dls, ckpt=64)
    th0 = np.concatenate([p.A, p.beta])

    def loss(th):
        s2 = mq.System.diatom(mq._diatom_with(p, th), path="factorised")
        pop, _, d2 = mq.propagate(s2, mq.make_trajs(ts, s2), device=False)
        return float(np.sum(dls * mq.cross_sections(s2, pop, w, ts.group, ts.n_groups))), d2["steps"]

    for k in (1, len(p.A) + 1):
        h = 1e-5 * abs(th0[k])
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        lp, sp = loss(tp)
        lm, sm = loss(tm)
        assert np.array_equal(sp, sm) and np.array_equal(sp, diag["steps"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g[k]), 1e-3 * np.max(np.abs(g))), (k, fd, g[k])
