"""The allocation-free scoring entry point against the regular one.

rtdetmcd_distances_noalloc exists for callers that cannot allocate device
memory when they score (a sorting line that must not wait on an allocator
between frames, code inside a fixed memory budget).  It keeps its working
state in a fixed device array instead of a workspace.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtd():
    import __graft_entry__ as g
    g.build()
    import paper_1910_05615_gb300 as m
    return m


def _case(seed, n, p):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((n, p)) * 1.5 + 0.5).astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    S = (Q * np.logspace(0, 2, p)) @ Q.T
    return X, rng.standard_normal(p), S


def test_noalloc_matches_regular_entry_point_twice(rtd):
    lib = rtd._load()
    # two calls in a row with different sizes and fits: the shared array must
    # not carry anything over from the first call
    for seed, n, p in ((0, 20_011, 20), (1, 7_003, 5)):
        X, mu, S = _case(seed, n, p)
        Xd = torch.from_numpy(X).cuda()
        for prec in (rtd.RTD_FP64, rtd.RTD_FP32):
            ref = rtd.rtdetmcd_distances(Xd, mu, S, precision=prec)
            out = torch.empty(n, dtype=torch.float32, device="cuda")
            st = lib.rtdetmcd_distances_noalloc(Xd.data_ptr(), n, p, p, mu.ctypes.data, S.ctypes.data,
                                                prec, out.data_ptr(),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == 0
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-6, atol=0)


def test_noalloc_rejects_what_it_cannot_hold(rtd):
    lib = rtd._load()
    X, mu, S = _case(2, 100, 3)
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty(100, dtype=torch.float32, device="cuda")
    # host rows would need staging memory: refused
    st = lib.rtdetmcd_distances_noalloc(X.ctypes.data, 100, 3, 3, mu.ctypes.data, S.ctypes.data, 1,
                                        out.data_ptr(), None)
    assert st == 1
    # p beyond the maximum the fixed array holds: refused
    st = lib.rtdetmcd_distances_noalloc(Xd.data_ptr(), 10, 65, 65, mu.ctypes.data, S.ctypes.data, 1,
                                        out.data_ptr(), None)
    assert st == 1
