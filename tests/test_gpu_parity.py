"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs."""
import numpy as np
import pytest

import datagen
import oracle as O
from parity import TOL, compare_fit, rel_center, rel_mat, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtd():
    import __graft_entry__ as g
    g.build()
    import paper_1910_05615_gb300 as m
    return m


def _spd(p, rng, cond=50.0):
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    ev = np.logspace(0, np.log10(cond), p)
    return (Q * ev) @ Q.T


# ----------------------------------------------------------- scoring (Section 6)
@pytest.mark.parametrize("p", [1, 3, 5, 20, 37, 64])
@pytest.mark.parametrize("host", [False, True])
def test_distances(rtd, p, host):
    rng = np.random.default_rng(p)
    n = 5003 + 7 * p
    X = (rng.standard_normal((n, p)) * 2 + 1).astype(np.float32)
    mu = rng.standard_normal(p)
    S = _spd(p, rng)
    ref = O.mahalanobis_d2_plain(X, mu, S)
    src = X if host else torch.from_numpy(X).cuda()
    for prec, tol in ((rtd.RTD_FP64, 1e-6), (rtd.RTD_FP32, 2e-4)):
        d2 = to_np(rtd.rtdetmcd_distances(src, mu, S, precision=prec))
        # FP64 form: exact up to the float32 store of the result
        err = np.max(np.abs(d2 - ref) / np.maximum(ref, 1e-3))
        assert err < tol, (prec, err)


def test_distances_strided(rtd):
    rng = np.random.default_rng(0)
    n, p, ld = 3001, 6, 11
    buf = rng.standard_normal((n, ld)).astype(np.float32)
    X = torch.from_numpy(buf).cuda()[:, :p]
    mu = np.zeros(p)
    S = _spd(p, rng)
    d2 = to_np(rtd.rtdetmcd_distances(X, mu, S, precision=rtd.RTD_FP64))
    ref = O.mahalanobis_d2_plain(buf[:, :p], mu, S)
    assert np.max(np.abs(d2 - ref) / np.maximum(ref, 1e-3)) < 1e-6


def test_flag_bit_exact(rtd):
    rng = np.random.default_rng(1)
    d2 = (rng.chisquare(5, 100_003)).astype(np.float32)
    cut = O.chi2_ppf(0.975, 5)
    d2[:10] = np.float32(cut)                      # exactly at the cutoff: not flagged
    fl, cnt = rtd.rtdetmcd_flag(torch.from_numpy(d2).cuda(), cut)
    ref = d2.astype(np.float64) > cut
    assert np.array_equal(to_np(fl).astype(bool), ref) and cnt == int(ref.sum())
    fl2, cnt2 = rtd.rtdetmcd_flag(d2, cut)         # host buffers
    assert np.array_equal(fl2.astype(bool), ref) and cnt2 == cnt


@pytest.mark.parametrize("p", [1, 4, 20, 37, 64])
@pytest.mark.parametrize("host", [False, True])
def test_score_one_pass(rtd, p, host):
    """Distances, flags and count in one pass (Section 6): the flags equal
    those of the FP64 distances (rows within 2^-9 of the cutoff are decided
    in FP64), the distances match the plain definition, and outside the band
    the FP32 distances are those of rtdetmcd_distances bit for bit."""
    rng = np.random.default_rng(100 + p)
    n = 200_003 + 13 * p
    X = (rng.standard_normal((n, p)) * 1.3 + 0.4).astype(np.float32)
    X[: n // 20] += 4.0
    mu = rng.standard_normal(p) * 0.1
    S = _spd(p, rng, cond=30.0)
    cut = O.chi2_ppf(0.975, p)
    ref = O.mahalanobis_d2_plain(X, mu, S)
    src = X if host else torch.from_numpy(X).cuda()
    for prec, tol in ((rtd.RTD_FP32, 2e-4), (rtd.RTD_FP64, 1e-6)):
        d2, fl, cnt = rtd.rtdetmcd_score(src, mu, S, cut, precision=prec)
        d2, fl = to_np(d2), to_np(fl).astype(bool)
        assert np.max(np.abs(d2 - ref) / np.maximum(ref, 1e-3)) < tol
        decided = np.abs(ref - cut) > 1e-12 * cut
        assert np.array_equal(fl[decided], (ref > cut)[decided]) and cnt == int(fl.sum())
        if prec == rtd.RTD_FP32:
            d2b = to_np(rtd.rtdetmcd_distances(src, mu, S, precision=prec))
            outside = np.abs(d2b.astype(np.float64) - cut) > 2.0 ** -8 * cut
            assert np.array_equal(d2[outside], d2b[outside])
    # flags only, distances only
    _, fl2, cnt2 = rtd.rtdetmcd_score(src, mu, S, cut, d2=False)
    assert cnt2 == cnt and np.array_equal(to_np(fl2).astype(bool), fl)
    d3, fl3, cnt3 = rtd.rtdetmcd_score(src, mu, S, cut, flags=False)
    assert fl3 is None and cnt3 == -1


@pytest.mark.parametrize("p", [1, 4, 20, 37, 64])
def test_score_prepared(rtd, p):
    """A fit prepared once scores two batches with one launch each: the
    distances and flags equal those of rtdetmcd_score bit for bit (the same
    factorisation and pass), in both forms, and the device counter adds up
    both calls' flags."""
    rng = np.random.default_rng(300 + p)
    mu = rng.standard_normal(p) * 0.1
    S = _spd(p, rng, cond=30.0)
    cut = O.chi2_ppf(0.975, p)
    prep = rtd.rtdetmcd_score_prepare(mu, S, cut)
    for prec in (rtd.RTD_FP32, rtd.RTD_FP64):
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        total = 0
        for k in range(2):
            n = 100_003 + 7919 * k
            X = (rng.standard_normal((n, p)) * 1.3 + 0.4).astype(np.float32)
            X[: n // 20] += 4.0
            Xd = torch.from_numpy(X).cuda()
            d2, fl = rtd.rtdetmcd_score_prepared(Xd, prep, precision=prec, count=count)
            d2r, flr, cntr = rtd.rtdetmcd_score(Xd, mu, S, cut, precision=prec)
            assert torch.equal(d2, d2r) and torch.equal(fl, flr)
            total += cntr
            ref = O.mahalanobis_d2_plain(X, mu, S)
            decided = np.abs(ref - cut) > 1e-12 * cut
            assert np.array_equal(to_np(fl).astype(bool)[decided], (ref > cut)[decided])
        torch.cuda.synchronize()
        assert int(count.item()) == total
    if p == 4:   # rows of stride 8, a ragged last group of four rows
        buf = (rng.standard_normal((50_001, 8)) * 1.3).astype(np.float32)
        Xs = torch.from_numpy(buf).cuda()[:, :4]
        d2, fl = rtd.rtdetmcd_score_prepared(Xs, prep)
        ref = O.mahalanobis_d2_plain(buf[:, :4], mu, S)
        assert np.max(np.abs(to_np(d2) - ref) / np.maximum(ref, 1e-3)) < 2e-4
        decided = np.abs(ref - cut) > 1e-12 * cut
        assert np.array_equal(to_np(fl).astype(bool)[decided], (ref > cut)[decided])


def test_score_prepared_rejects(rtd):
    """A scatter that is not positive definite is refused at preparation, and
    the FP32 pass of such a prepared fit writes nothing; host rows, a count
    without flags and a misaligned prepared fit are argument errors."""
    p = 4
    bad = np.eye(p)
    bad[3, 3] = 0.0
    prep = torch.empty(rtd.rtdetmcd_prepared_size(), dtype=torch.uint8, device="cuda")
    with pytest.raises(rtd.RtdError) as e:
        rtd.rtdetmcd_score_prepare(np.zeros(p), bad, out=prep)
    assert e.value.code == 4
    X = torch.randn(5000, p, device="cuda")
    d2 = torch.full((5000,), -7.0, device="cuda")
    fl = torch.full((5000,), 9, dtype=torch.uint8, device="cuda")
    rtd.rtdetmcd_score_prepared(X, prep, d2_out=d2, flags_out=fl)
    torch.cuda.synchronize()
    assert bool((d2 == -7.0).all()) and bool((fl == 9).all())
    good = rtd.rtdetmcd_score_prepare(np.zeros(p), np.eye(p))
    lib = rtd._load()
    Xh = np.zeros((5000, p), np.float32)
    assert lib.rtdetmcd_score_prepared(Xh.ctypes.data, 5000, p, p, good.data_ptr(), rtd.RTD_FP32, d2.data_ptr(),
                                       fl.data_ptr(), None, None) == 1
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert lib.rtdetmcd_score_prepared(X.data_ptr(), 5000, p, p, good.data_ptr(), rtd.RTD_FP32, d2.data_ptr(),
                                       None, cnt.data_ptr(), None) == 1
    assert lib.rtdetmcd_score_prepared(X.data_ptr(), 5000, p, p, good.data_ptr() + 8, rtd.RTD_FP32,
                                       d2.data_ptr(), fl.data_ptr(), None, None) == 1


def test_score_strided_and_rejects(rtd):
    rng = np.random.default_rng(5)
    n, p, ld = 40_001, 6, 11
    buf = rng.standard_normal((n, ld)).astype(np.float32)
    X = torch.from_numpy(buf).cuda()[:, :p]
    S = _spd(p, rng)
    d2, fl, cnt = rtd.rtdetmcd_score(X, np.zeros(p), S, 12.0)
    ref = O.mahalanobis_d2_plain(buf[:, :p], np.zeros(p), S)
    assert np.max(np.abs(to_np(d2) - ref) / np.maximum(ref, 1e-3)) < 2e-4
    assert cnt == int(np.sum(ref > 12.0))
    bad = S.copy()
    bad[0, 0] = -1.0
    with pytest.raises(rtd.RtdError) as e:
        rtd.rtdetmcd_score(X, np.zeros(p), bad, 12.0)
    assert e.value.code == 4


# ------------------------------------------------------------- whole fits
def _fit_both(rtd, fr, form, host=False, **kw):
    X = fr.X if host else torch.from_numpy(fr.X).cuda()
    prec = rtd.RTD_FP32 if form == "fp32" else rtd.RTD_FP64
    got = rtd.rtdetmcd_fit(X, fr.h, precision=prec, subset=True, diag=True, **kw)
    ref = O.fit(fr.X, fr.h, **{k: v for k, v in kw.items() if k in ("omega", "seed", "q")})
    return got, ref


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_fit_small_case(rtd, form):
    """n=10,000, p=5, 10% point outliers at 10 v_min (serial algorithm, q=1)."""
    fr = datagen.small_fp64_case()
    got, ref = _fit_both(rtd, fr, form)
    assert got["q"] == ref.q == 1
    d = got["diag"]
    # the whole-column univariate MCD is FP64 in both forms
    rt = 1e-10
    np.testing.assert_allclose(d["mu_uni"], ref.mu_uni, rtol=rt, atol=rt * 1e-2)
    np.testing.assert_allclose(d["sigma_uni"], ref.s_uni, rtol=rt)
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))
    assert got["n_flagged"] == int(ref.flags.sum())


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_fit_column_of_close_values(rtd, form):
    """A column whose values all share their high 24 key bits (1 + j 2^-23,
    j < 256, in random order, heavy ties) and a column with one value in 30%
    of the rows: long runs of keys that differ only in the lowest digit, and
    long runs of equal keys, in every sort pass."""
    import types
    rng = np.random.default_rng(21)
    n, p = 30_011, 3
    X = rng.standard_normal((n, p)).astype(np.float32)
    X[:, 1] = (1.0 + rng.integers(0, 256, n) * 2.0 ** -23).astype(np.float32)
    X[rng.random(n) < 0.3, 2] = np.float32(0.75)
    fr = types.SimpleNamespace(X=X, h=(3 * n) // 4)
    got, ref = _fit_both(rtd, fr, form, q=3)
    d = got["diag"]
    np.testing.assert_allclose(d["mu_uni"], ref.mu_uni, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(d["sigma_uni"], ref.s_uni, rtol=1e-10)
    ok, rep = compare_fit(got, ref, X, form)
    if not ok:
        pytest.fail(str(rep))


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_fit_blocks(rtd, form):
    """Parallel algorithm: q = 9 blocks of a ragged n (discarded rows)."""
    fr = datagen.contaminated_gaussian(184_331, 5, eps=0.15, kind="shift", shift=6.0, seed=4)
    got, ref = _fit_both(rtd, fr, form)
    assert got["q"] == ref.q == 9 and got["m"] == ref.m
    d = got["diag"]
    for l, b in enumerate(ref.blocks):
        for k in range(2):
            c = d["chains"][2 * l + k]
            oc = b.chains[k]
            # initial scatters S~_k are continuous functions of the data
            assert rel_mat(c["S_init"], b.S[k]) < (1e-4 if form == "fp32" else 1e-8)
            if oc is not None and oc.ok and c["status"] == 0:
                assert rel_mat(c["Sigma"], oc.Sigma) < TOL[form] * 10
        assert d["blocks"][l]["chosen"] == b.chosen
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))


def test_fit_host_buffers(rtd):
    fr = datagen.contaminated_gaussian(20_000, 6, eps=0.2, kind="cluster", shift=6.0, seed=2)
    got, ref = _fit_both(rtd, fr, "fp32", host=True)
    assert isinstance(got["flags"], np.ndarray)
    ok, rep = compare_fit(got, ref, fr.X, "fp32")
    if not ok:
        pytest.fail(str(rep))


# ----------------------------------------------------- full-size workload
@pytest.fixture(scope="module")
def main_case():
    fr = datagen.main_case()
    return fr, O.fit(fr.X, fr.h)


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_fit_main_case(rtd, main_case, form):
    """n=1,000,000, p=20, h=floor(0.75n), 20% cluster outliers (q = 12)."""
    fr, ref = main_case
    X = torch.from_numpy(fr.X).cuda()
    got = rtd.rtdetmcd_fit(X, fr.h, precision=rtd.RTD_FP32 if form == "fp32" else rtd.RTD_FP64,
                           subset=True, diag=True)
    assert got["q"] == ref.q == 12
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))
    for l, b in enumerate(ref.blocks):
        assert got["diag"]["blocks"][l]["chosen"] == b.chosen
        assert got["diag"]["blocks"][l]["kept"] == int(l in ref.kept)
    # the update-based C-step (Section 3.5) is taken: some chain recomputed
    # its Gram from scratch at fewer steps than it ran
    ch = got["diag"]["chains"]
    assert any(c["status"] == 0 and 0 < c["full_recomputes"] < c["steps"] for c in ch)
    assert sum(c["steps"] - c["full_recomputes"] for c in ch) > 0


# ------------------------------------------------------------ edge cases
def test_nonfinite_rows(rtd):
    fr = datagen.contaminated_gaussian(5000, 4, eps=0.0, kind="point", shift=0.0, seed=0)
    X = fr.X.copy()
    X[1234, 2] = np.nan
    with pytest.raises(rtd.RtdError) as e:
        rtd.rtdetmcd_fit(torch.from_numpy(X).cuda(), fr.h)
    assert e.value.code == 2
    X[1234, 2] = np.inf
    r = rtd.rtdetmcd_fit(torch.from_numpy(X).cuda(), fr.h, check=False)
    assert r["status"] == 2


def test_degenerate_column(rtd):
    fr = datagen.contaminated_gaussian(5000, 4, eps=0.0, kind="point", shift=0.0, seed=0)
    X = fr.X.copy()
    X[:3000, 1] = 1.0           # more than half the values equal: zero univariate MCD scale
    with pytest.raises(O.OracleError):
        O.fit(X, fr.h)
    r = rtd.rtdetmcd_fit(torch.from_numpy(X).cuda(), fr.h, check=False)
    assert r["status"] == 4


@pytest.mark.parametrize("form", ["fp32", "fp64"])
@pytest.mark.parametrize("n,p,alpha,seed", [
    (3001, 1, 0.75, 0),        # univariate data
    (9, 3, 0.75, 1),           # the smallest sizes the definition allows here
    (4999, 64, 0.75, 2),       # maximum dimension
    (12_288, 3, 0.5, 3),       # h = [(n+p+1)/2], q = 1 exactly at n = p omega
    (61_447, 2, 0.6, 5),       # q = 7, ragged tail
])
def test_fit_edges(rtd, form, n, p, alpha, seed):
    fr = datagen.contaminated_gaussian(n, p, eps=0.1, kind="point", shift=9.0, seed=seed, alpha=alpha)
    h = max(fr.h, (n + p + 1) // 2)
    try:
        ref = O.fit(fr.X, h)
    except O.OracleError:
        r = rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), h, check=False)
        assert r["status"] != 0
        return
    got = rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), h,
                           precision=rtd.RTD_FP32 if form == "fp32" else rtd.RTD_FP64,
                           subset=True, diag=True)
    assert got["q"] == ref.q
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_fit_block_cap(rtd, form):
    """n / (p omega) = 1250 blocks by eq. partitionsize, capped at 1024
    (reading R10) on both sides: 1024 blocks of 39 rows."""
    fr = datagen.contaminated_gaussian(40_000, 2, eps=0.1, kind="point", shift=9.0, seed=12)
    ref = O.fit(fr.X, fr.h, omega=16)
    assert ref.q == 1024 and ref.m == 39
    got = rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, omega=16, subset=True,
                           precision=rtd.RTD_FP32 if form == "fp32" else rtd.RTD_FP64)
    assert got["q"] == 1024 and got["m"] == 39
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))
    with pytest.raises(rtd.RtdError):
        rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, q=1025)


def test_fit_deterministic(rtd):
    fr = datagen.contaminated_gaussian(50_000, 8, eps=0.2, kind="cluster", shift=7.0, seed=9)
    X = torch.from_numpy(fr.X).cuda()
    a = rtd.rtdetmcd_fit(X, fr.h, subset=True)
    b = rtd.rtdetmcd_fit(X, fr.h, subset=True)
    assert np.array_equal(a["mu"], b["mu"]) and np.array_equal(a["Sigma"], b["Sigma"])
    assert torch.equal(a["flags"], b["flags"]) and torch.equal(a["subset"], b["subset"])


# ------------------------------------------- selection paths of the C-step
@pytest.mark.parametrize("case", ["main", "point"])
def test_select_paths_agree(rtd, main_case, case):
    """The FP32 form's window selection (default), the histogram path at every
    step, and windows of the smallest width (whose misses fall back to the
    histogram path) all take the FP64-exact h_b smallest at every step, so
    they give the same subsets and bitwise the same fits."""
    if case == "main":
        fr = main_case[0]
    else:
        fr = datagen.contaminated_gaussian(120_000, 5, eps=0.1, kind="point", shift=10.0, seed=3)
    X = torch.from_numpy(fr.X).cuda()
    res = {sp: rtd.rtdetmcd_fit(X, fr.h, select_path=sp, subset=True, profile=True) for sp in (0, 1, 2)}
    for sp in (1, 2):
        assert torch.equal(res[sp]["subset"], res[0]["subset"]), sp
        assert np.array_equal(res[sp]["mu"], res[0]["mu"]) and np.array_equal(res[sp]["Sigma"], res[0]["Sigma"])
        assert np.array_equal(res[sp]["mu_raw"], res[0]["mu_raw"])
        assert torch.equal(res[sp]["flags"], res[0]["flags"])
    p0, p1, p2 = (res[sp]["profile"] for sp in (0, 1, 2))
    assert p0["win_steps"] > 0 and p1["win_steps"] == 0
    assert p2["win_steps"] > 0
    assert p0["sel_band"] > 0


@pytest.mark.parametrize("case", ["main", "point", "p37", "p64"])
def test_dist_paths_agree(rtd, main_case, case):
    """The C-step distances on the CUDA cores (FP32 FMAs, the default) and on
    the tensor cores (split-TF32 operands) feed the same FP64-exact
    decisions: the same subsets at every step, so bitwise the same fits."""
    if case == "main":
        fr = main_case[0]
    elif case == "point":
        fr = datagen.contaminated_gaussian(120_000, 5, eps=0.1, kind="point", shift=10.0, seed=3)
    elif case == "p37":
        fr = datagen.contaminated_gaussian(300_000, 37, eps=0.15, kind="cluster", shift=6.0, seed=6)
    else:
        fr = datagen.contaminated_gaussian(200_000, 64, eps=0.1, kind="shift", shift=7.0, seed=4)
    X = torch.from_numpy(fr.X).cuda()
    a = rtd.rtdetmcd_fit(X, fr.h, dist_path=0, subset=True, profile=True)
    b = rtd.rtdetmcd_fit(X, fr.h, dist_path=1, subset=True)
    assert torch.equal(a["subset"], b["subset"])
    assert np.array_equal(a["mu"], b["mu"]) and np.array_equal(a["Sigma"], b["Sigma"])
    assert np.array_equal(a["Sigma_raw"], b["Sigma_raw"]) and torch.equal(a["flags"], b["flags"])
    assert a["profile"]["win_steps"] > 0


@pytest.mark.parametrize("case", ["main", "blocks", "point", "fp64", "bf16", "maxsteps"])
def test_graph_fit_equals_stream_fit(rtd, main_case, case):
    """The fit captured as one CUDA graph with device-side control flow (the
    C-step loop as a conditional WHILE node) issues the same kernels on the
    same data as the stream path: bitwise the same results."""
    kw = {}
    if case == "main":
        fr = main_case[0]
    elif case == "blocks":
        fr = datagen.contaminated_gaussian(184_331, 5, eps=0.15, kind="shift", shift=6.0, seed=4)
    elif case == "point":
        fr = datagen.contaminated_gaussian(120_000, 5, eps=0.1, kind="point", shift=10.0, seed=3)
    elif case == "fp64":
        fr = datagen.contaminated_gaussian(50_000, 8, eps=0.2, kind="cluster", shift=7.0, seed=9)
        kw = {"precision": rtd.RTD_FP64}
    elif case == "bf16":
        fr = datagen.large_case(n=200_003, p=32, seed=5)
        kw = {"precision": rtd.RTD_BF16}
    else:
        fr = datagen.contaminated_gaussian(60_000, 6, eps=0.15, kind="cluster", shift=6.0, seed=21)
        kw = {"max_csteps": 2}
    X = torch.from_numpy(fr.X).cuda()
    a = rtd.rtdetmcd_fit(X, fr.h, subset=True, diag=True, **kw)
    sub = torch.empty(X.shape[0], dtype=torch.uint8, device="cuda")
    d2 = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    fl = torch.empty(X.shape[0], dtype=torch.uint8, device="cuda")
    for rep in range(2):      # the second call relaunches the cached graph
        d2.fill_(-1.0)
        b = rtd.rtdetmcd_fit(X, fr.h, graph=True, subset=True, diag=True, d2_out=d2, flags_out=fl, **kw)
        assert b["status"] == 0 and b["warnings"] == a["warnings"]
        assert np.array_equal(a["mu"], b["mu"]) and np.array_equal(a["Sigma"], b["Sigma"])
        assert np.array_equal(a["Sigma_raw"], b["Sigma_raw"]) and a["csteps_max"] == b["csteps_max"]
        assert torch.equal(a["d2"], d2) and torch.equal(a["flags"], fl)
        assert torch.equal(a["subset"], b["subset"])
        da, db = a["diag"], b["diag"]
        assert [c["steps"] for c in da["chains"]] == [c["steps"] for c in db["chains"]]


@pytest.mark.parametrize("bad", ["nan", "degenerate"])
def test_graph_fit_data_errors(rtd, bad):
    """Data errors end the captured fit on the device (the conditional nodes
    skip the later stages) with the stream path's status."""
    fr = datagen.contaminated_gaussian(5000, 4, eps=0.0, kind="point", shift=0.0, seed=0)
    X = fr.X.copy()
    if bad == "nan":
        X[1234, 2] = np.nan
    else:
        X[:3000, 1] = 1.0
    Xd = torch.from_numpy(X).cuda()
    a = rtd.rtdetmcd_fit(Xd, fr.h, check=False)
    b = rtd.rtdetmcd_fit(Xd, fr.h, graph=True, check=False)
    assert a["status"] == b["status"] == (2 if bad == "nan" else 4)


def test_select_path_rejects_bad_value(rtd):
    fr = datagen.small_fp64_case()
    with pytest.raises(rtd.RtdError):
        rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, select_path=3)


# ------------------------------------------------ warm start (end of Section 4)
@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_warm_start_parity(rtd, form):
    """C-steps of every block from an earlier fit (reading R13), against the
    oracle's warm start from its own full fit."""
    fr = datagen.contaminated_gaussian(60_000, 6, eps=0.15, kind="cluster", shift=6.0, seed=21)
    base = O.fit(fr.X, fr.h)
    ref = O.fit(fr.X, fr.h, init=(base.mu, base.Sigma))
    got = rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, init=(base.mu, base.Sigma),
                           precision=rtd.RTD_FP32 if form == "fp32" else rtd.RTD_FP64, subset=True)
    assert got["q"] == ref.q
    ok, rep = compare_fit(got, ref, fr.X, form)
    if not ok:
        pytest.fail(str(rep))


def test_warm_start_rejects_non_positive_diagonal(rtd):
    fr = datagen.small_fp64_case()
    S = np.eye(fr.X.shape[1])
    S[0, 0] = -1.0
    with pytest.raises(rtd.RtdError):
        rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, init=(np.zeros(fr.X.shape[1]), S))


# ------------------------------ adjoint of steps 8-10 with W held fixed
def _grad_case(rtd, n, p, seed, ld=None):
    fr = datagen.contaminated_gaussian(n, p, eps=0.2, kind="cluster", shift=5.0, seed=seed)
    if ld is None:
        X = torch.from_numpy(fr.X).cuda()
    else:
        buf = np.zeros((n, ld), dtype=np.float32)
        buf[:, :p] = fr.X
        X = torch.from_numpy(buf).cuda()[:, :p]
    fit = rtd.rtdetmcd_fit(X, fr.h, subset=True, d2=False, flags=False)
    W = (to_np(fit["subset"]) >> 1) & 1
    return fr, X, fit, W.astype(bool)


def _grad_err(g, ref):
    """Largest row error relative to the row's gradient norm, with the median
    norm as the floor for rows whose gradient nearly vanishes."""
    nrm = np.linalg.norm(ref, axis=1)
    floor = np.median(nrm)
    return np.max(np.linalg.norm(g - ref, axis=1) / np.maximum(nrm, floor))


@pytest.mark.parametrize("n,p,ld", [(100_000, 20, None), (20_011, 1, None), (30_001, 7, 9), (12_007, 64, None)])
def test_grad_matches_oracle(rtd, n, p, ld):
    """Value and gradient against the oracle's closed forms in FP64 (the
    closed forms are pinned to central differences on the CPU).  Row
    arithmetic in FP32: u = Sigma^-1 r carries about p cond(Sigma)^1/2 eps32,
    so the bar is 1e-4 of each row's gradient norm."""
    fr, X, fit, W = _grad_case(rtd, n, p, seed=40 + p, ld=ld)
    c = fit["c_rew"]
    assert c > 0 and W.sum() == fit["n_reweight"]
    for wl, wr in ((1.0, 1.0), (1.0, 0.0), (0.0, 2.5)):
        val, g = rtd.rtdetmcd_grad(X, fit["subset"], fit["mu"], fit["Sigma"], c, w_logdet=wl, w_rd=wr)
        ref_val = O.fixed_set_objective(fr.X, W, c, wl, wr)
        ref = O.fixed_set_gradient(fr.X, W, c, wl, wr)
        assert abs(val - ref_val) <= 1e-5 * max(abs(ref_val), 1.0), (wl, wr, val, ref_val)
        err = _grad_err(to_np(g), ref)
        assert err < 1e-4, (wl, wr, err)


def test_grad_value_only_and_autograd(rtd):
    fr, X, fit, W = _grad_case(rtd, 50_000, 6, seed=7)
    val, g = rtd.rtdetmcd_grad(X, fit["subset"], fit["mu"], fit["Sigma"], fit["c_rew"], grad=False)
    assert g is None
    Xr = X.clone().requires_grad_(True)
    f = rtd.rtdetmcd_objective(Xr, fr.h, w_logdet=1.0, w_rd=1.0)
    assert abs(float(f) - val) <= 1e-12 * abs(val)
    (3.0 * f).backward()
    ref = O.fixed_set_gradient(fr.X, W, fit["c_rew"])
    assert _grad_err(Xr.grad.cpu().numpy() / 3.0, ref) < 1e-4


def test_grad_sums(rtd):
    """Invariants that hold at any size: the log-det gradient of the rows of W
    sums to zero (log det Sigma is translation invariant) and vanishes off W;
    checked on the 1,000,000 x 20 workload against sampled oracle rows."""
    fr = datagen.main_case()
    X = torch.from_numpy(fr.X).cuda()
    fit = rtd.rtdetmcd_fit(X, fr.h, subset=True, d2=False, flags=False)
    sub = fit["subset"]
    _, g = rtd.rtdetmcd_grad(X, sub, fit["mu"], fit["Sigma"], fit["c_rew"], w_logdet=1.0, w_rd=0.0)
    W = ((sub >> 1) & 1).bool()
    gd = g.double()
    assert float(gd[~W].abs().max()) == 0.0
    s = gd[W].sum(0).abs().max().item()
    assert s <= 1e-3 * gd[W].abs().sum(0).max().item()
    # sampled rows against the closed form u_i 2c/(N-1) with u from the fit
    Wn = W.cpu().numpy()
    N = int(Wn.sum())
    idx = np.flatnonzero(Wn)[:: N // 97][:97]
    Sinv = np.linalg.inv(fit["Sigma"])
    ref = (fr.X[idx].astype(np.float64) - fit["mu"]) @ Sinv * (2.0 * fit["c_rew"] / (N - 1))
    assert _grad_err(g[idx].cpu().numpy(), ref) < 1e-4


def _cotangents(n, p, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(p), rng.standard_normal((p, p)), 0.7, rng.standard_normal(n)


@pytest.mark.parametrize("n,p,ld", [(100_000, 20, None), (30_001, 7, 9), (12_007, 64, None)])
def test_vjp_matches_oracle(rtd, n, p, ld):
    """Vector-Jacobian product of (mu, Sigma, log det Sigma, RD) with W fixed,
    for random cotangents on all four outputs, against the oracle's FP64
    closed forms (pinned to central differences on the CPU)."""
    fr, X, fit, W = _grad_case(rtd, n, p, seed=60 + p, ld=ld)
    c = fit["c_rew"]
    gmu, gS, gld, grd = _cotangents(n, p, p)
    ref = O.fixed_set_vjp(fr.X, W, c, gmu, gS, gld, grd)
    g = rtd.rtdetmcd_vjp(X, fit["subset"], fit["mu"], fit["Sigma"], c, gmu=gmu, gSigma=gS, glogdet=gld,
                         gRD=torch.from_numpy(grd.astype(np.float32)).cuda())
    err = _grad_err(to_np(g), ref)
    assert err < 1e-4, err
    # one output at a time: mu alone, Sigma alone
    g1 = rtd.rtdetmcd_vjp(X, fit["subset"], fit["mu"], fit["Sigma"], c, gmu=gmu)
    assert _grad_err(to_np(g1), O.fixed_set_vjp(fr.X, W, c, gmu=gmu)) < 1e-4
    g2 = rtd.rtdetmcd_vjp(X, fit["subset"], fit["mu"], fit["Sigma"], c, gSigma=gS)
    assert _grad_err(to_np(g2), O.fixed_set_vjp(fr.X, W, c, gSigma=gS)) < 1e-4


def test_fit_outputs_autograd(rtd):
    """torch.autograd through the fit's four outputs: a loss mixing mu,
    Sigma, log det Sigma and the robust distances, against the oracle's VJP
    with the fit's W."""
    fr, X, fit, W = _grad_case(rtd, 40_000, 6, seed=71)
    rng = np.random.default_rng(3)
    a, B, wv = rng.standard_normal(6), rng.standard_normal((6, 6)), rng.standard_normal(40_000)
    Xr = X.clone().requires_grad_(True)
    mu, S, ld, rd = rtd.rtdetmcd_fit_outputs(Xr, fr.h)
    np.testing.assert_array_equal(mu.detach().cpu().numpy(), fit["mu"])
    loss = (mu * torch.from_numpy(a).cuda()).sum() + (S * torch.from_numpy(B).cuda()).sum() + 0.3 * ld \
        + (rd.double() * torch.from_numpy(wv).cuda()).sum()
    loss.backward()
    ref = O.fixed_set_vjp(fr.X, W, fit["c_rew"], a, B, 0.3, wv)
    assert _grad_err(Xr.grad.cpu().numpy(), ref) < 1e-4


def test_adjoint_central_differences_full_fit(rtd):
    """The n = 100,000, p = 20 adjoint check: FP32 forward, torch.autograd
    backward of log det Sigma + sum_i RD_i with the fit's discrete choices
    fixed, against (a) central differences (step 1e-3) of the same quantity
    from the whole fit re-run in the plain FP64 form on each perturbed input,
    on 200 rows whose distances lie away from the h-subset threshold and the
    cutoff, and (b) the oracle's FP64 gradient on every row."""
    fr = datagen.main_case(n=100_000)
    n, p = fr.X.shape
    ref_fit = O.fit(fr.X, fr.h)
    assert ref_fit.q == 1
    X = torch.from_numpy(fr.X).cuda()
    Xr = X.clone().requires_grad_(True)
    mu, S, ld, rd = rtd.rtdetmcd_fit_outputs(Xr, fr.h)
    (ld + rd.double().sum()).backward()
    g = Xr.grad.cpu().numpy().astype(np.float64)
    G = O.fixed_set_gradient(fr.X, ref_fit.W, O.reweight_factor(p))     # c of reading R8
    assert _grad_err(g, G) < 1e-4
    # rows away from both bands of the oracle fit (5% of the threshold)
    ch = ref_fit.blocks[0].chains[ref_fit.blocks[0].chosen]
    Zb = (fr.X.astype(np.float64) - ref_fit.mu_uni) / ref_fit.s_uni
    d2c = O.mahalanobis_d2(Zb, ch.mu, ch.Sigma)
    t = np.sort(d2c)[ref_fit.h_b - 1]
    away = (np.abs(d2c - t) > 0.05 * t) & (np.abs(ref_fit.d2_raw - ref_fit.cutoff_d2) > 0.05 * ref_fit.cutoff_d2)
    rows = np.random.default_rng(5).choice(np.flatnonzero(away), 200, replace=False)
    ks = np.random.default_rng(6).integers(0, p, 200)

    def f64(Xh):
        r = rtd.rtdetmcd_fit(torch.from_numpy(Xh).cuda(), fr.h, precision=rtd.RTD_FP64, subset=True,
                             d2=False, flags=False)
        m = torch.from_numpy(r["mu"]).cuda()
        Sg = torch.from_numpy(r["Sigma"]).cuda()
        Lc = torch.linalg.cholesky(Sg)
        Y = torch.linalg.solve_triangular(Lc, (torch.from_numpy(Xh).cuda().double() - m).T, upper=False)
        val = 2.0 * torch.log(torch.diagonal(Lc)).sum() + Y.square().sum(0).sqrt().sum()
        return float(val), r["subset"].cpu().numpy()

    base_sub = rtd.rtdetmcd_fit(X, fr.h, precision=rtd.RTD_FP64, subset=True)["subset"].cpu().numpy()
    errs, skipped = [], 0
    floor = np.median(np.linalg.norm(G, axis=1))
    for i, k in zip(rows, ks):
        Xp, Xm = fr.X.copy(), fr.X.copy()
        Xp[i, k] = np.float32(fr.X[i, k] + 1e-3)
        Xm[i, k] = np.float32(fr.X[i, k] - 1e-3)
        step = float(Xp[i, k]) - float(Xm[i, k])
        fp, sp = f64(Xp)
        fm, sm = f64(Xm)
        if not (np.array_equal(sp, base_sub) and np.array_equal(sm, base_sub)):
            skipped += 1          # a discrete choice moved: not a point of differentiability
            continue
        fd = (fp - fm) / step
        errs.append(abs(fd - g[i, k]) / max(np.linalg.norm(G[i]), floor))
    assert skipped <= 5 and len(errs) >= 195
    assert max(errs) < 1e-3, max(errs)


def test_grad_rejects_small_set(rtd):
    fr, X, fit, W = _grad_case(rtd, 5_000, 4, seed=3)
    sub = torch.zeros_like(fit["subset"])
    sub[:4] = 2                                   # |W| = p: singular covariance
    with pytest.raises(rtd.RtdError):
        rtd.rtdetmcd_grad(X, sub, fit["mu"], fit["Sigma"], fit["c_rew"])


# --------------------------- split-BF16 form: Grams on the tensor cores
@pytest.mark.parametrize("n,p", [(400_000, 40), (200_003, 25), (200_003, 48)])
def test_bf16_form_parity(rtd, n, p):
    """Start and C-step Grams on tcgen05 (three-way split-BF16 products, FP32
    accumulation in tensor memory, compensated sums every 128 rows), the
    reweighting Gram on the CUDA cores: mu and Sigma (raw and reweighted)
    within 1e-3 relative of the FP64 oracle, and, as for the FP32 form, the
    same final h-subsets, reweighting set and flags outside the 1e-6 tie
    bands."""
    fr = datagen.large_case(n=n, p=p, seed=5)
    ref = O.fit(fr.X, fr.h)
    got = rtd.rtdetmcd_fit(torch.from_numpy(fr.X).cuda(), fr.h, precision=rtd.RTD_BF16, subset=True)
    assert got["q"] == ref.q
    ok, rep = compare_fit(got, ref, fr.X, "bf16")
    rep["logdet"] = abs(got["logdet"] - np.linalg.slogdet(ref.Sigma)[1])
    d2 = to_np(got["d2"]).astype(np.float64)
    rep["d2"] = float(np.max(np.abs(d2 - ref.d2) / np.maximum(ref.d2, 1e-3)))
    print(rep)
    assert ok, rep
    # the tensor-core products carry 24 bits: the fit is as close as the FP32 form's
    assert max(rep["mu"], rep["Sigma"], rep["mu_raw"], rep["Sigma_raw"]) <= 1e-5, rep


def test_bf16_form_matches_fp32_gram(rtd):
    """The tensor-core Gram against the CUDA-core one on the same rows: both
    forms reach the same h-subsets and reweighting set (the FP64 bands decide
    the same rows), so their fits differ by the Gram's rounding only: three-way
    split-BF16 products and FP32 sums on one side, FP32 products and
    compensated sums on the other."""
    fr = datagen.large_case(n=300_000, p=32, seed=9)
    X = torch.from_numpy(fr.X).cuda()
    a = rtd.rtdetmcd_fit(X, fr.h, precision=rtd.RTD_FP32, subset=True)
    b = rtd.rtdetmcd_fit(X, fr.h, precision=rtd.RTD_BF16, subset=True)
    sa, sb = to_np(a["subset"]), to_np(b["subset"])
    rep = {"subset_differ": int(np.sum((sa & 3) != (sb & 3))), "Sigma_raw": rel_mat(b["Sigma_raw"], a["Sigma_raw"]),
           "Sigma": rel_mat(b["Sigma"], a["Sigma"]), "flags_differ": int((a["flags"] != b["flags"]).sum())}
    print(rep)
    assert rep["subset_differ"] == 0 and rep["flags_differ"] == 0, rep
    assert rep["Sigma_raw"] <= 1e-6 and rep["Sigma"] <= 1e-6, rep


# -------------------- many frames of uneven n and p (batched form)
def test_fit_batch_matches_single_fits_and_oracle(rtd):
    """Frames of the many-frames workload (n in [2000, 50000], p in
    {8, 16, 24, 32, 40}, 0-25% point outliers): each batched result equals
    the single-fit result bit for bit, and matches the oracle (FP32 form
    tolerances, q = 1 per frame)."""
    frames = [datagen.batched_frame(f) for f in range(12)]
    Xs = [torch.from_numpy(fr.X).cuda() for fr in frames]
    got = rtd.rtdetmcd_fit_batch(Xs, [fr.h for fr in frames], nstreams=4)
    for f, fr in enumerate(frames):
        one = rtd.rtdetmcd_fit(Xs[f], fr.h)
        g = got[f]
        assert g["status"] == 0 and g["q"] == 1
        assert np.array_equal(g["mu"], one["mu"]) and np.array_equal(g["Sigma"], one["Sigma"])
        assert torch.equal(g["d2"], one["d2"]) and torch.equal(g["flags"], one["flags"])
    for f in (0, 5, 11):
        fr = frames[f]
        ref = O.fit(fr.X, fr.h)
        ok, rep = compare_fit(got[f], ref, fr.X, "fp32", check_subsets=False)
        assert ok, (f, rep)


def test_autotune_keeps_every_value(rtd):
    """The autotuner changes launch shapes only: fits under the tuned shape
    equal the untuned ones bit for bit, and the choice is kept."""
    fr = datagen.contaminated_gaussian(150_000, 12, eps=0.15, kind="cluster", shift=6.0, seed=31)
    X = torch.from_numpy(fr.X).cuda()
    a = rtd.rtdetmcd_fit(X, fr.h, subset=True)
    t = rtd.rtdetmcd_autotune(X, fr.h)
    assert t["candidates"] == 9 and t["ms_best"] > 0 and t["ms_best"] <= t["ms_default"]
    assert rtd.rtdetmcd_tuned(150_000, 12) == {**t, "candidates": 0, "ms_best": 0.0, "ms_default": 0.0}
    for graph in (False, True):
        b = rtd.rtdetmcd_fit(X, fr.h, subset=True, graph=graph)
        assert np.array_equal(a["mu"], b["mu"]) and np.array_equal(a["Sigma"], b["Sigma"])
        assert torch.equal(a["subset"], b["subset"]) and torch.equal(a["flags"], b["flags"])


def test_fit_batch_graph_matches_single_fits(rtd):
    """Many frames, each a captured graph updated in place from frame to frame
    (device-side C-step loop), with per-class autotuning: every result equals
    the single stream fit bit for bit."""
    frames = [datagen.batched_frame(f) for f in range(40, 72)]
    Xs = [torch.from_numpy(fr.X).cuda() for fr in frames]
    got = rtd.rtdetmcd_fit_batch(Xs, [fr.h for fr in frames], nstreams=4, graph=1, autotune=1)
    for f, fr in enumerate(frames):
        one = rtd.rtdetmcd_fit(Xs[f], fr.h)
        g = got[f]
        assert g["status"] == 0
        assert np.array_equal(g["mu"], one["mu"]) and np.array_equal(g["Sigma"], one["Sigma"])
        assert torch.equal(g["d2"], one["d2"]) and torch.equal(g["flags"], one["flags"])


def test_fit_batch_host_frames(rtd):
    frames = [datagen.batched_frame(f) for f in range(20, 26)]
    got = rtd.rtdetmcd_fit_batch([fr.X for fr in frames], [fr.h for fr in frames], nstreams=3)
    for f, fr in enumerate(frames):
        one = rtd.rtdetmcd_fit(fr.X, fr.h)
        assert np.array_equal(got[f]["Sigma"], one["Sigma"])
        assert np.array_equal(got[f]["flags"], one["flags"])
