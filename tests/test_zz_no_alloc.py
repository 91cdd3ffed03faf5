"""The allocation-free scoring entry point against the regular one.

rtdetmcd_distances_noalloc exists for callers that cannot allocate device
memory when they score (a sorting line that must not wait on an allocator
between frames, code inside a fixed memory budget).  It keeps its working
state in a fixed device array instead of a workspace.  Both entry points run
the same kernels on the same inputs, so their outputs must agree bit for bit.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O

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


def _call(lib, Xd, n, p, mu, S, prec, out):
    return lib.rtdetmcd_distances_noalloc(Xd.data_ptr(), n, p, p, mu.ctypes.data, S.ctypes.data, prec,
                                          out.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _free_bytes():
    return torch.cuda.mem_get_info()[0]     # cudaMemGetInfo


def test_noalloc_matches_regular_entry_point_twice(rtd):
    lib = rtd._load()
    # two calls in a row with different sizes and fits: the shared array must
    # not carry anything over from the first call
    for seed, n, p in ((0, 20_011, 20), (1, 7_003, 5)):
        X, mu, S = _case(seed, n, p)
        Xd = torch.from_numpy(X).cuda()
        plain = O.mahalanobis_d2_plain(X, mu, S)
        for prec, tol in ((rtd.RTD_FP64, 1e-6), (rtd.RTD_FP32, 2e-4)):
            ref = rtd.rtdetmcd_distances(Xd, mu, S, precision=prec)
            out = torch.empty(n, dtype=torch.float32, device="cuda")
            assert _call(lib, Xd, n, p, mu, S, prec, out) == 0
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got, ref.cpu().numpy())
            assert np.max(np.abs(got - plain) / np.maximum(plain, 1e-3)) < tol


def test_noalloc_allocates_nothing(rtd):
    lib = rtd._load()
    n, p = 50_000, 12
    X, mu, S = _case(3, n, p)
    Xd = torch.from_numpy(X).cuda()
    ref = rtd.rtdetmcd_distances(Xd, mu, S, precision=rtd.RTD_FP32)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    assert _call(lib, Xd, n, p, mu, S, rtd.RTD_FP32, out) == 0      # warm: modules loaded
    torch.cuda.synchronize()
    a0, f0 = torch.cuda.memory_allocated(), _free_bytes()
    out.zero_()
    torch.cuda.synchronize()
    assert _call(lib, Xd, n, p, mu, S, rtd.RTD_FP32, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0 and _free_bytes() == f0
    assert torch.equal(out, ref)


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
    # the binding refuses an output it could overrun or misread
    with pytest.raises(ValueError):
        rtd.rtdetmcd_distances_noalloc(Xd, mu, S, out=torch.empty(99, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        rtd.rtdetmcd_distances_noalloc(Xd, mu, S, out=torch.empty(100, dtype=torch.float16, device="cuda"))
    with pytest.raises(ValueError):
        rtd.rtdetmcd_distances_noalloc(Xd, mu, S, out=torch.empty(200, dtype=torch.float32, device="cuda")[::2])
