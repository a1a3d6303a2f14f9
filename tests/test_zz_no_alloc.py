"""mqct_propagate_noalloc: the allocation-free variant of the FP64 trajectory launch.

Callers that may not allocate GPU memory while it runs (fixed device pools, real-time
loops) use this entry point; its scratch is a static device array inside the library.
Here it is called through the C ABI with caller-owned device buffers, twice in a row
(its work counter must be cleared by every call), and its populations and diagnostics
are compared with those of mqct_propagate on the same trajectories, for one system and for
an uneven batch of three systems in one call.  This file is named so that pytest collects
it last."""
import ctypes as C

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
    L = api.lib()
    L.mqct_propagate_noalloc.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
    L.mqct_propagate_noalloc.restype = C.c_int
    return api


@pytest.mark.parametrize("path", ["plain", "factorised"])
def test_noalloc_matches_propagate_twice(mq, path):
    import torch

    p, ts = W.small_workload(jmax=4, n_b=6, energies=(400.0, 1500.0), init_js=(0, 2), b_max=9.0, n_grid=150)
    sys_ = mq.System.diatom(p, path=path, precision="fp64")
    tr = mq.make_trajs(ts, sys_)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    ref_pop, _, ref_diag = mq.propagate(sys_, trd, device=True)
    torch.cuda.synchronize()
    ref_pop = ref_pop.cpu().numpy()
    ref_diag = mq.diag_to_numpy(ref_diag)
    hs = (C.c_void_p * 1)(sys_.handle.value)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        pop = torch.full((ts.n, sys_.n), -1.0, dtype=torch.float64, device="cuda")
        diag = torch.zeros((ts.n * mq.DIAG_DTYPE.itemsize,), dtype=torch.uint8, device="cuda")
        st = mq.lib().mqct_propagate_noalloc(hs, 1, trd.data_ptr(), ts.n, pop.data_ptr(), None, diag.data_ptr(),
                                             stream)
        assert st == mq.OK, mq.lib().mqct_last_error()
        torch.cuda.synchronize()
        d = mq.diag_to_numpy(diag)
        assert np.array_equal(d["steps"], ref_diag["steps"])
        assert np.array_equal(d["status"], ref_diag["status"])
        assert np.max(np.abs(pop.cpu().numpy() - ref_pop)) < 1e-8


def test_noalloc_uneven_batch_twice(mq):
    """Three diatom bases (N = 16, 36, 81) with interleaved trajectories in one call: the views of
    all three systems are written into the static array by the call itself."""
    import torch

    rng = np.random.default_rng(4)
    ps = [W.diatom_pes_params(jmax=j, n_grid=120) for j in (3, 5, 8)]
    systems = [mq.System.diatom(p, path="factorised", precision="fp64") for p in ps]
    n = 18
    sidx = np.repeat(np.arange(3, dtype=np.int32), n // 3)
    rng.shuffle(sidx)
    z = np.zeros(n, np.int32)
    ts = W.TrajSet(W.cm(rng.uniform(500.0, 2500.0, n)), rng.uniform(0.0, 8.0, n), z, z.copy(), sidx.copy(), 3,
                   sampling="mc", b_max=8.0, n_b=0, system=sidx, group_e=np.zeros(3), group_j=np.zeros(3, np.int32))
    tr = mq.make_trajs(ts, systems)
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    ref_pop, _, ref_diag = mq.propagate(systems, trd, device=True)
    torch.cuda.synchronize()
    ref_pop = ref_pop.cpu().numpy()
    ref_diag = mq.diag_to_numpy(ref_diag)
    nmax = max(s_.n for s_ in systems)
    hs = (C.c_void_p * 3)(*[s_.handle.value for s_ in systems])
    stream = torch.cuda.current_stream().cuda_stream
    width = np.array([systems[k].n for k in sidx])
    valid = np.arange(nmax)[None, :] < width[:, None]
    for _ in range(2):
        pop = torch.full((n, nmax), -1.0, dtype=torch.float64, device="cuda")
        diag = torch.zeros((n * mq.DIAG_DTYPE.itemsize,), dtype=torch.uint8, device="cuda")
        st = mq.lib().mqct_propagate_noalloc(hs, 3, trd.data_ptr(), n, pop.data_ptr(), None, diag.data_ptr(), stream)
        assert st == mq.OK, mq.lib().mqct_last_error()
        torch.cuda.synchronize()
        d = mq.diag_to_numpy(diag)
        assert np.all(d["status"] == 0)
        assert np.array_equal(d["steps"], ref_diag["steps"])
        assert np.max(np.abs(np.where(valid, pop.cpu().numpy() - ref_pop, 0.0))) < 1e-8


def test_noalloc_rejects_host_buffers_and_too_many_systems(mq):
    import torch

    p, ts = W.small_workload(jmax=1, n_b=2, energies=(500.0,), init_js=(0,), b_max=5.0, n_grid=40)
    sys_ = mq.System.diatom(p)
    tr = mq.make_trajs(ts, sys_)
    pop = torch.zeros((ts.n, sys_.n), dtype=torch.float64, device="cuda")
    hs = (C.c_void_p * 1)(sys_.handle.value)
    # host trajectories: rejected (the call cannot stage them without allocating)
    st = mq.lib().mqct_propagate_noalloc(hs, 1, tr.ctypes.data, ts.n, pop.data_ptr(), None, None, None)
    assert st == mq.ERR_INVALID_ARG
    assert b"device memory" in mq.lib().mqct_last_error()
    hs17 = (C.c_void_p * 17)(*([sys_.handle.value] * 17))
    trd = torch.from_numpy(tr.view(np.uint8).copy()).cuda()
    st = mq.lib().mqct_propagate_noalloc(hs17, 17, trd.data_ptr(), ts.n, pop.data_ptr(), None, None, None)
    assert st == mq.ERR_INVALID_ARG
    assert b"16 systems" in mq.lib().mqct_last_error()
