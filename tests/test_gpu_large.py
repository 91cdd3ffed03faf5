"""GPU: the large-p workload at full size (n = 10,000,000, p = 40, q = 61,
15% mixed contamination) in the FP32 and split-BF16 forms.

The oracle's whole fit is out of reach at this size, so each stage's output
is checked against what the method fixes at any size, recomputed in FP64 on
the host with the oracle's own functions from the GPU's outputs:
  - the standardisation of sampled columns: the oracle's univariate MCD;
  - steps 2-4 for sampled blocks: the chosen chain's final h-subset is the
    h_b smallest distances under that chain's own fit (a C-step fixed point),
    outside the 1e-6 tie band;
  - steps 5-7: the raw fit is the oracle's aggregation (median, KL, keep,
    pool) of the blocks' fits, with the same kept blocks;
  - step 8: the reweighting set is the rows of the blocks within the cutoff
    of the raw fit, outside the tie band;
  - step 9: the reweighted fit is the mean and c_rew-scaled covariance of
    that set (1e-5 relative);
  - step 10: every flag is d2 > cutoff under the reweighted fit outside the
    tie band, and sampled distances match FP64 ones (2e-4 relative).
"""
import numpy as np
import pytest

import datagen
import oracle as O
from parity import TIE, rel_center, rel_mat, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtd():
    import __graft_entry__ as g
    g.build()
    import paper_1910_05615_gb300 as m
    return m


@pytest.fixture(scope="module")
def large():
    fr = datagen.large_case(seed=0)
    return fr, torch.from_numpy(fr.X).cuda()


def _d2_chunks(X, mu, Sigma, rows=None, chunk=1 << 20):
    """FP64 squared distances of the rows of X (or of X[rows]) by the
    oracle's Cholesky form, a chunk of rows at a time."""
    idx = np.arange(X.shape[0]) if rows is None else rows
    out = np.empty(idx.size)
    for a in range(0, idx.size, chunk):
        out[a:a + chunk] = O.mahalanobis_d2(X[idx[a:a + chunk]], mu, Sigma)
    return out


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_large_p_full_size_properties(rtd, large, form):
    fr, Xd = large
    X, h = fr.X, fr.h
    n, p = X.shape
    prec = {"fp32": rtd.RTD_FP32, "bf16": rtd.RTD_BF16}[form]
    f = rtd.rtdetmcd_fit(Xd, h, precision=prec, subset=True, diag=True)
    q, m, hb = f["q"], f["m"], f["h_b"]
    assert (q, m) == (61, n // 61) and f["status"] == 0
    dg = f["diag"]
    mu_uni, s_uni = dg["mu_uni"], dg["sigma_uni"]
    sub = to_np(f["subset"])
    cut = f["cutoff_d2"]
    assert cut == pytest.approx(O.chi2_ppf(0.975, p), rel=1e-12)
    # standardisation (Section 3.1) of sampled columns
    for j in (0, 17, 39):
        u = O.univariate_mcd(X[:, j])
        assert mu_uni[j] == pytest.approx(u.mu, rel=1e-10, abs=1e-12)
        assert s_uni[j] == pytest.approx(np.sqrt(u.s2), rel=1e-10)
    perm = O.partition_permutation(n, 0)
    # steps 2-4 for sampled blocks: the chosen chain's subset is its own fixed point
    for l in (0, 30, 60):
        c = dg["blocks"][l]["chosen"]
        assert c in (0, 1)
        ch = dg["chains"][2 * l + c]
        assert ch["status"] == 0
        rows = perm[l * m:(l + 1) * m]
        Z = (X[rows].astype(np.float64) - mu_uni) / s_uni
        d2l = O.mahalanobis_d2(Z, ch["mu"], ch["Sigma"])
        t = np.sort(d2l)[hb - 1]
        inH = (sub[rows] & 1).astype(bool)
        assert inH.sum() == hb
        away = np.abs(d2l - t) > TIE * t
        assert np.array_equal(inH[away], (d2l <= t)[away])
    # steps 5-7: the oracle's aggregation of the blocks' fits
    c_alpha = O.consistency_factor(h / n, p)
    fits = []
    for l in range(q):
        c = dg["blocks"][l]["chosen"]
        ch = dg["chains"][2 * l + c] if c >= 0 else None
        fits.append(None if ch is None else (ch["mu"], c_alpha * ch["Sigma"]))
    mu_raw_z, S_raw_z, kept, _ = O.aggregate(fits, hb, c_alpha)
    assert sorted(kept) == [l for l in range(q) if dg["blocks"][l]["kept"]]
    D = np.outer(s_uni, s_uni)
    np.testing.assert_allclose(f["mu_raw"], mu_uni + s_uni * mu_raw_z, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(f["Sigma_raw"], S_raw_z * D, rtol=1e-10, atol=1e-12 * np.abs(S_raw_z * D).max())
    # step 8: the reweighting set
    used = perm[: q * m]
    d2_raw = _d2_chunks(X, f["mu_raw"], f["Sigma_raw"], rows=used)
    W = np.zeros(n, bool)
    W[used] = ((sub[used] >> 1) & 1).astype(bool)
    away = np.abs(d2_raw - cut) > TIE * cut
    assert np.array_equal(W[used][away], (d2_raw <= cut)[away])
    # step 9: mean and c_rew-scaled covariance of W
    Xw = X[W].astype(np.float64)
    assert f["n_reweight"] == Xw.shape[0]
    mu_w = Xw.mean(axis=0)
    S_w = O.reweight_factor(p) * np.cov(Xw, rowvar=False, ddof=1)
    del Xw
    assert rel_center(f["mu"], mu_w, S_w) <= 1e-5
    assert rel_mat(f["Sigma"], S_w) <= 1e-5
    # step 10: every flag, and sampled distances
    d2_ref = _d2_chunks(X, f["mu"], f["Sigma"])
    fl = to_np(f["flags"]).astype(bool)
    away = np.abs(d2_ref - cut) > TIE * cut
    assert np.array_equal(fl[away], (d2_ref > cut)[away])
    assert f["n_flagged"] == int(fl.sum())
    S = np.random.default_rng(1).choice(n, 20_000, replace=False)
    d2 = to_np(f["d2"])
    assert np.max(np.abs(d2[S] - d2_ref[S]) / np.maximum(d2_ref[S], 1e-3)) < 2e-4
