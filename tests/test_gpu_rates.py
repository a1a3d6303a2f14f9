"""GPU parity of the post-processing step (Sec. III, Eq. 20 and the Maxwell-Boltzmann rates)
against the oracle, through the C ABI."""
import numpy as np
import pytest

import paper_2312_02322_gb300.inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mq():
    import torch

    assert torch.cuda.is_available()
    import paper_2312_02322_gb300.api as api

    return api


def _compare(rate, ref, rtol):
    ok = np.isfinite(ref) & (np.abs(ref) > 1e-250)
    assert np.all(np.isfinite(rate))
    err = np.max(np.abs(rate[ok] - ref[ok]) / np.abs(ref[ok]))
    assert err < rtol, err
    # rates the oracle underflows to zero are negligible on the GPU too
    assert np.all(np.abs(rate[~ok]) < 1e-200)


def test_small_all_pairs_match_oracle(mq):
    from oracle import rates as R

    rs = W.rate_set(n_levels=7)
    sym, rate = mq.rate_coefficients(rs.sigma, rs.u, rs.energy, rs.g, rs.mu, rs.kT)
    assert np.allclose(sym, R.sigma_sym(rs.sigma, rs.g), rtol=1e-15, atol=0)
    ref = R.rates(rs.sigma, rs.u, rs.energy, rs.g, rs.mu, rs.kT)
    _compare(rate, ref, 1e-10)


def test_detailed_balance_on_device(mq):
    import torch

    rs = W.rate_set(n_levels=40, seed=3)
    sig = torch.from_numpy(rs.sigma).cuda()
    _, rate = mq.rate_coefficients(sig, rs.u, rs.energy, rs.g, rs.mu, rs.kT, sigma_sym=False)
    k = rate.cpu().numpy()
    E, g = rs.energy, rs.g
    for t, th in enumerate(rs.kT):
        arg = -(E[None, :] - E[:, None]) / th
        ok = (g[:, None] * k[t] > 1e-250) & (k[t].T > 1e-250) & (np.abs(arg) < 600.0)
        lhs = g[:, None] * k[t]
        rhs = g[None, :] * k[t].T * np.exp(np.where(ok, arg, 0.0))
        assert np.max(np.abs(lhs[ok] - rhs[ok]) / lhs[ok]) < 1e-12


def test_paper_scale_sampled(mq):
    """1032 levels (the paper's count of non-degenerate channels), sampled pairs vs the oracle."""
    import torch

    from oracle import rates as R

    rs = W.rate_set(n_levels=1032, seed=9)
    sig = torch.from_numpy(rs.sigma).cuda()
    _, rate = mq.rate_coefficients(sig, rs.u, rs.energy, rs.g, rs.mu, rs.kT, sigma_sym=False)
    k = rate.cpu().numpy()
    rng = np.random.default_rng(1)
    L = rs.energy.size
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, L, (24, 2))] + [(0, L - 1), (L - 1, 0), (5, 5), (0, 1)]
    ref = R.rates(rs.sigma, rs.u, rs.energy, rs.g, rs.mu, rs.kT, pairs=pairs)
    for (a, b) in pairs:
        _compare(k[:, a, b], ref[:, a, b], 1e-10)


def test_edge_cases_match_oracle(mq):
    """Thresholds above U_1 and above U_K, a zero pair, two energies only, tail slopes at both clips."""
    from oracle import rates as R

    u = W.cm(np.array([50.0, 400.0]))
    E = W.cm(np.array([0.0, 300.0, 1500.0, 10.0]))
    g = np.array([1.0, 3.0, 5.0, 7.0])
    sig = np.zeros((2, 4, 4))
    sig[:, 0, 1] = [2.0, 1.0]      # u0 = 150 cm^-1 inside (U_1, U_2); slope ~ -1/3
    sig[:, 1, 0] = [0.5, 0.4]
    sig[:, 0, 2] = [1.0, 1.0]      # u0 = 750 cm^-1 above U_K
    sig[:, 2, 0] = [0.1, 0.3]
    sig[:, 1, 3] = [3.0, 0.01]     # steep fall -> p clipped to -1
    sig[:, 3, 1] = [3.0, 0.02]
    sig[:, 2, 3] = [0.2, 5.0]      # growth -> p = 0
    kT = np.array([10.0, 100.0, 1000.0]) * mq.KB_HARTREE_PER_K
    _, rate = mq.rate_coefficients(sig, u, E, g, 1800.0, kT, sigma_sym=False)
    ref = R.rates(sig, u, E, g, 1800.0, kT)
    assert np.all(rate[:, 1, 2] == 0.0) and np.all(rate[:, 2, 1] == 0.0)
    _compare(rate, ref, 1e-10)


def test_rejections(mq):
    u = np.array([1e-4, 2e-4])
    E = np.zeros(2)
    g = np.ones(2)
    sig = np.ones((2, 2, 2))
    with pytest.raises(mq.MQCTError):
        mq.rate_coefficients(sig, u[::-1].copy(), E, g, 1000.0, [1e-4])
    with pytest.raises(mq.MQCTError):
        mq.rate_coefficients(sig, u, E, g, 1000.0, [0.0])
    with pytest.raises(mq.MQCTError):
        mq.rate_coefficients(sig, u, E, np.array([1.0, 0.0]), 1000.0, [1e-4])
    with pytest.raises(mq.MQCTError):
        mq.rate_coefficients(sig, u, E, g, -1.0, [1e-4])
    with pytest.raises(mq.MQCTError):
        mq.rate_coefficients(np.ones((1, 2, 2)), u[:1].copy(), E, g, 1000.0, [1e-4])
