"""The C-ABI library builds, loads and exports every symbol include/rtdetmcd.h
declares; host-side argument checks and the library's own chi-square
routines (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtdetmcd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1910_05615_gb300 import build as b
    path = b.build()
    import paper_1910_05615_gb300 as m
    L = m._load()
    assert os.path.samefile(path, m.library_path())
    return L


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rtdetmcd_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


def test_chi2_quantile_matches_oracle(lib):
    for p in (1, 2, 3, 5, 8, 20, 40, 64):
        for q in (0.5, 0.6, 0.75, 0.975, 0.99):
            assert lib.rtdetmcd_chi2_quantile(p, q) == pytest.approx(O.chi2_ppf(q, p), rel=1e-12)


def test_status_strings(lib):
    import paper_1910_05615_gb300 as m
    for code in range(8):
        assert m.rtdetmcd_status_string(code) != "unknown status"
    assert m.rtdetmcd_status_string(99) == "unknown status"


def test_workspace_size(lib):
    import paper_1910_05615_gb300 as m
    a = m.rtdetmcd_workspace_size(1_000_000, 20)
    b = m.rtdetmcd_workspace_size(1_000_000, 20, precision=m.RTD_FP64)
    assert 0 < a < b < 4 << 30
    assert m.rtdetmcd_workspace_size(10, 20) == 0          # n <= 2p
    assert m.rtdetmcd_workspace_size(1000, 65) == 0        # p > 64
    assert m.rtdetmcd_diag_size(5, 1) == 8 * (10 + 2 * (75 + 10 + 6) + 3)


@pytest.mark.parametrize("n,p,ld,h,code", [
    (1000, 5, 5, 502, 1),      # h < [(n+p+1)/2] = 503
    (1000, 5, 5, 1000, 1),     # h = n
    (1000, 0, 5, 700, 1),      # p < 1
    (1000, 65, 65, 700, 1),    # p > 64
    (1000, 5, 4, 700, 1),      # ld < p
    (10, 5, 5, 8, 1),          # n <= 2p
    (1000, 5, 5, 700, 5),      # valid, but no workspace
])
def test_fit_rejects_before_device_work(lib, n, p, ld, h, code):
    import paper_1910_05615_gb300 as m
    X = np.zeros((n, max(ld, 1)), np.float32)
    res = m._Result()
    st = lib.rtdetmcd_fit(X.ctypes.data, n, p, ld, h, None, None, 0, None, ctypes.byref(res), None, None)
    assert st == code and res.status == code


def test_fit_rejects_too_many_blocks(lib):
    """An explicit block count above RTD_MAX_BLOCKS = 1024 is refused (the
    rule's own q is capped there instead, reading R10)."""
    import paper_1910_05615_gb300 as m
    n, p = 100_000, 2
    X = np.zeros((n, p), np.float32)
    o = m._Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    for q, code in ((1025, 1), (1024, 5)):     # 5: valid, but no workspace
        o.q_override = q
        res = m._Result()
        st = lib.rtdetmcd_fit(X.ctypes.data, n, p, p, (3 * n) // 4, ctypes.byref(o), None, 0, None,
                              ctypes.byref(res), None, None)
        assert st == code, q
    o.q_override = 1025
    assert lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o)) == 0


@pytest.mark.parametrize("p", [24, 49])
def test_bf16_form_width_range(lib, p):
    """The tensor-core Gram form covers 25 <= p <= 48 only."""
    import paper_1910_05615_gb300 as m
    n = 20_000
    X = np.zeros((n, p), np.float32)
    o = m._Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision = m.RTD_BF16
    res = m._Result()
    st = lib.rtdetmcd_fit(X.ctypes.data, n, p, p, (3 * n) // 4, ctypes.byref(o), None, 0, None,
                          ctypes.byref(res), None, None)
    assert st == 1
    assert lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o)) == 0
    o.precision = m.RTD_FP32
    assert lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o)) > 0


def test_distances_rejects_bad_arguments(lib):
    X = np.zeros((10, 3), np.float32)
    mu = np.zeros(3)
    S = np.eye(3)
    out = np.zeros(10, np.float32)
    st = lib.rtdetmcd_distances(X.ctypes.data, 10, 3, 2, mu.ctypes.data, S.ctypes.data, 1,
                                out.ctypes.data, None, 0, None)
    assert st == 1
    st = lib.rtdetmcd_distances(X.ctypes.data, 10, 3, 3, mu.ctypes.data, S.ctypes.data, 7,
                                out.ctypes.data, None, 0, None)
    assert st == 1


@pytest.mark.parametrize("case", ["mu_only", "zero_diag", "nan_sigma", "nan_mu"])
def test_fit_rejects_bad_warm_start(lib, case):
    """A warm start needs both mu and Sigma, finite, with a positive diagonal;
    anything else is RTD_EINVAL before any device work."""
    import paper_1910_05615_gb300 as m
    n, p, h = 1000, 3, 700
    X = np.zeros((n, p), np.float32)
    mu, S = np.zeros(p), np.eye(p)
    if case == "zero_diag":
        S[1, 1] = 0.0
    elif case == "nan_sigma":
        S[0, 2] = np.nan
    elif case == "nan_mu":
        mu[0] = np.nan
    o = m._Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.init_mu = mu.ctypes.data
    o.init_sigma = None if case == "mu_only" else S.ctypes.data
    res = m._Result()
    st = lib.rtdetmcd_fit(X.ctypes.data, n, p, p, h, ctypes.byref(o), None, 0, None, ctypes.byref(res), None, None)
    assert st == 1 and res.status == 1


@pytest.mark.parametrize("case", ["host_x", "bad_c", "bad_wbit", "p_too_big", "one_row"])
def test_grad_rejects_bad_arguments(lib, case):
    """rtdetmcd_grad wants device rows and subset bytes, c > 0, a bit index
    0..7, 1 <= p <= 64 and n >= 2; anything else is RTD_EINVAL."""
    n, p, c, wbit = 100, 3, 1.2, 1
    if case == "bad_c":
        c = 0.0
    elif case == "bad_wbit":
        wbit = 8
    elif case == "p_too_big":
        p = 65
    elif case == "one_row":
        n = 1
    X = np.zeros((n, p), np.float32)
    w = np.full(n, 2, np.uint8)
    mu, S = np.zeros(p), np.eye(p)
    val = ctypes.c_double(0.0)
    st = lib.rtdetmcd_grad(X.ctypes.data, n, p, p, w.ctypes.data, wbit, mu.ctypes.data, S.ctypes.data, c,
                           1.0, 1.0, ctypes.byref(val), None, None, 0, None)
    assert st == 1
    ws = lib.rtdetmcd_grad_workspace_size(n, p)
    assert (ws == 0) if case == "p_too_big" else (ws > 0 and ws % 256 == 0)


def test_fit_batch_rejects_before_device_work(lib):
    """An invalid frame (here h below [(n+p+1)/2]) stops the whole batch with
    RTD_EINVAL before any device work, and only that frame carries the code."""
    import paper_1910_05615_gb300 as m
    F = 3
    frames = [np.zeros((1000, 5), np.float32) for _ in range(F)]
    Xp = (ctypes.c_void_p * F)(*[a.ctypes.data for a in frames])
    n = (ctypes.c_int64 * F)(1000, 1000, 1000)
    p = (ctypes.c_int32 * F)(5, 5, 5)
    ld = (ctypes.c_int64 * F)(5, 5, 5)
    h = (ctypes.c_int64 * F)(700, 400, 700)
    res = (m._Result * F)()
    st = lib.rtdetmcd_fit_batch(F, Xp, n, p, ld, h, None, None, 0, None, 2, res, None, None)
    assert st == 1
    assert [res[f].status for f in range(F)] == [0, 1, 0]
    one = lib.rtdetmcd_fit_batch_workspace_size(F, n, p, None, 1)
    assert one > 0 and lib.rtdetmcd_fit_batch_workspace_size(F, n, p, None, 2) == 2 * one
    assert lib.rtdetmcd_fit_batch_workspace_size(F, n, p, None, 8) == 3 * one   # at most one slice per frame
    assert lib.rtdetmcd_fit_batch_workspace_size(F, n, p, None, 0) == 0


def test_stage_calls_reject_before_device_work(lib):
    """The stage entry points of a sharded fit refuse ranges outside
    [0, p), [0, q), [0, n) and missing pointers (RTD_EINVAL) before looking
    at the workspace (RTD_EWORKSPACE when it is missing)."""
    n, p, h = 40_000, 3, 30_000
    X = np.zeros((n, p), np.float32)
    q, m = ctypes.c_int32(0), ctypes.c_int64(0)
    assert lib.rtdetmcd_partition(n, p, h, None, ctypes.byref(q), ctypes.byref(m)) == 0
    assert (q.value, m.value) == (3, n // 3)
    assert lib.rtdetmcd_partition(n, p, n, None, ctypes.byref(q), ctypes.byref(m)) == 1   # h = n
    out = np.zeros(4 * p * p + 64)
    uni = np.concatenate([np.zeros(p), np.ones(p)])
    fits = np.zeros(3 * (2 + p + p * p))
    mom = np.zeros(1 + p + p * p)
    x = X.ctypes.data
    std = lambda lo, hi, o: lib.rtdetmcd_standardize(x, n, p, p, h, None, lo, hi, None, 0, None, o)  # noqa: E731
    assert std(0, 0, out.ctypes.data) == 1            # empty column range
    assert std(1, p + 1, out.ctypes.data) == 1
    assert std(0, p, None) == 1
    assert std(0, p, out.ctypes.data) == 5            # valid: only the workspace is missing
    blk = lambda lo, hi, u: lib.rtdetmcd_fit_blocks(x, n, p, p, h, None, u, lo, hi, None, 0, None,  # noqa: E731
                                                   out.ctypes.data)
    assert blk(0, 4, uni.ctypes.data) == 1
    assert blk(2, 1, uni.ctypes.data) == 1
    assert blk(0, 3, None) == 1
    assert blk(3, 3, uni.ctypes.data) == 5
    mo = lambda lo, hi, f: lib.rtdetmcd_reweight_moments(x, n, p, p, h, None, uni.ctypes.data, f, lo, hi,  # noqa
                                                         None, 0, None, out.ctypes.data)
    assert mo(-1, 2, fits.ctypes.data) == 1
    assert mo(0, 2, None) == 1
    assert mo(0, 3, fits.ctypes.data) == 5
    import paper_1910_05615_gb300 as M
    m_res = M._Result()
    fin = lambda lo, hi, mm: lib.rtdetmcd_reweight_finish(x, n, p, p, h, None, uni.ctypes.data,  # noqa: E731
                                                          fits.ctypes.data, mm, lo, hi, None, 0, None,
                                                          ctypes.byref(m_res), None, None)
    assert fin(0, n + 1, mom.ctypes.data) == 1 and m_res.status == 1
    assert fin(0, n, None) == 1
    assert fin(5, n, mom.ctypes.data) == 5
