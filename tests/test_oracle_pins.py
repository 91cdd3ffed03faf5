"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, brute force, invariants, printed values).  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import datagen
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Section 2.1
def test_chi2_closed_forms():
    # p = 2: F(x) = 1 - exp(-x/2)  =>  quantile = -2 ln(1 - q)
    for q in (0.5, 0.75, 0.975, 0.99):
        assert O.chi2_ppf(q, 2) == pytest.approx(-2.0 * math.log(1.0 - q), rel=1e-12)
    # p = 1: F(x) = erf(sqrt(x/2))
    for x in (0.1, 1.0, 5.023886, 9.0):
        assert O.chi2_cdf(x, 1) == pytest.approx(math.erf(math.sqrt(x / 2)), rel=1e-12)
    # p = 4: F(x) = 1 - exp(-x/2) (1 + x/2)
    for x in (0.5, 3.0, 11.0):
        assert O.chi2_cdf(x, 4) == pytest.approx(1 - math.exp(-x / 2) * (1 + x / 2), rel=1e-12)
    # printed table values (any chi-square table): chi2_{p,0.975}
    assert O.chi2_ppf(0.975, 1) == pytest.approx(5.024, abs=6e-4)
    assert O.chi2_ppf(0.975, 5) == pytest.approx(12.833, abs=6e-4)
    assert O.chi2_ppf(0.975, 20) == pytest.approx(34.170, abs=6e-4)


def test_consistency_factor_closed_form_p2():
    # p = 2: q_a = -2 ln(1-a); F_{chi2_4}(x) = 1 - e^{-x/2}(1 + x/2)
    for a in (0.5, 0.75, 0.9):
        x = -2 * math.log(1 - a)
        expect = a / (1 - math.exp(-x / 2) * (1 + x / 2))
        assert O.consistency_factor(a, 2) == pytest.approx(expect, rel=1e-12)


def test_consistency_factor_truncated_moment_p1():
    # c(a) makes the h-subset variance consistent at N(0,1):
    # 1/c(a) = E[X^2; X^2 <= q_a] / a, integrated here by the trapezoid rule.
    for a in (0.5, 0.75):
        qa = math.sqrt(O.chi2_ppf(a, 1))
        x = np.linspace(-qa, qa, 200001)
        f = x * x * np.exp(-x * x / 2) / math.sqrt(2 * math.pi)
        m2 = np.trapezoid(f, x)
        assert 1.0 / O.consistency_factor(a, 1) == pytest.approx(m2 / a, rel=1e-8)


# ---------------------------------------------------------------- Section 3.1
@pytest.mark.parametrize("seed", range(6))
def test_univariate_mcd_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = 9 + seed % 4
    x = rng.standard_normal(n)
    x[: seed % 3] += 8.0
    mu_b, s2_b = O.univariate_mcd_bruteforce(x)
    u = O.univariate_mcd(x)
    assert u.mu_raw == pytest.approx(mu_b, rel=1e-12, abs=1e-12)
    assert u.s2_raw == pytest.approx(s2_b, rel=1e-10)


def test_univariate_mcd_equivariance():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(5001), 9 + 0.1 * rng.standard_normal(900)])
    u = O.univariate_mcd(x)
    for a, b in ((2.5, -7.0), (-0.3, 4.0)):
        v = O.univariate_mcd(a * x + b)
        assert v.mu == pytest.approx(a * u.mu + b, rel=1e-10, abs=1e-10)
        assert v.s2 == pytest.approx(a * a * u.s2, rel=1e-10)
        assert v.n_w == u.n_w


def test_univariate_mcd_consistency_and_robustness():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(400_000)
    u = O.univariate_mcd(x)
    assert abs(u.mu) < 0.01 and abs(u.s2 - 1.0) < 0.02
    assert abs(u.mu_raw) < 0.02 and abs(u.s2_raw - 1.0) < 0.03
    # 40% far contamination: every far point is rejected by the reweighting,
    # the centre stays put; the scale is inflated only by the consistency
    # factors, which assume clean data.
    y = np.concatenate([x[:240_000], 50 + rng.standard_normal(160_000)])
    v = O.univariate_mcd(y)
    assert v.n_w <= 240_000 and abs(v.mu) < 0.02 and 0.9 < v.s2 < 1.3


# ---------------------------------------------------------------- Section 3.2
def test_wrapping_function():
    g = O.wrap
    # continuity at b (1.541 tanh(0.862*2.5) = 1.5001466) and at c (g(c) = 0)
    assert float(g(np.array([1.5]))[0]) == 1.5
    assert O.WRAP_Q1 * math.tanh(O.WRAP_Q2 * (O.WRAP_C - O.WRAP_B)) == pytest.approx(1.5001466, abs=1e-7)
    assert float(g(np.array([4.0]))[0]) == 0.0
    assert float(g(np.array([5.0]))[0]) == 0.0
    z = np.array([-3.0, -1.0, 0.0, 1.0, 3.0])
    np.testing.assert_array_equal(g(z), -g(-z))
    np.testing.assert_array_equal(g(np.array([-1.0, 1.0])), [-1.0, 1.0])
    # about 85% of N(0,1) values are untouched: P(|Z| <= 1.5) = erf(1.5/sqrt 2)
    assert math.erf(1.5 / math.sqrt(2)) == pytest.approx(0.8664, abs=1e-4)
    x = np.random.default_rng(0).standard_normal(200_000)
    assert np.mean(g(x) == x) == pytest.approx(0.8664, abs=0.004)


def test_gsscm_cutoffs_hand_computed():
    r = np.array([1.0, 8.0, 27.0, 64.0, 125.0])   # r^(2/3) = 1, 4, 9, 16, 25
    A, B = O.gsscm_cutoffs(r)
    assert A == 27.0
    # median 9, |dev| = 8,5,0,7,16 -> MAD 7
    assert B == pytest.approx((9 + 0.6744897501960817 * 1.4826 * 7) ** 1.5, rel=1e-14)
    np.testing.assert_allclose(O.xi_weight(np.array([A, B, 0.5 * (A + B), B + 1]), A, B),
                               [1.0, 0.0, 0.5, 0.0], rtol=0, atol=1e-15)


def test_gsscm_unit_weights_reduce_to_second_moment():
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((2001, 3))
    r = np.sqrt((Z * Z).sum(1))
    A, B = O.gsscm_cutoffs(r)
    w = O.xi_weight(r, A, B)
    keep = w == 1.0
    assert keep.sum() >= 1000           # at least the half below the median
    S2 = O.start_gsscm(Z)
    direct = sum(w[i] ** 2 * np.outer(Z[i], Z[i]) for i in range(Z.shape[0])) / Z.shape[0]
    np.testing.assert_allclose(S2, direct, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- Section 3.3
def test_refine_diagonal_start_reduces_to_univariate():
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((3001, 3)) * np.array([3.0, 1.0, 0.4]) + np.array([0.2, -1.0, 0.5])
    st = O.refine(Z, np.diag([9.0, 1.0, 0.16]))
    for j in range(3):
        u = O.univariate_mcd(Z[:, j])
        assert st.Sigma[j, j] == pytest.approx(u.s2, rel=1e-10)
        assert st.mu[j] == pytest.approx(u.mu, rel=1e-9, abs=1e-12)
    assert np.max(np.abs(st.Sigma - np.diag(np.diag(st.Sigma)))) < 1e-12


def test_refine_drops_ill_conditioned():
    Z = np.random.default_rng(0).standard_normal((500, 3))
    assert O.refine(Z, np.diag([1.0, 1.0, 0.5e-3])) is None
    assert O.refine(Z, np.diag([1.0, 1.0, 2e-3])) is not None


# ---------------------------------------------------------------- Section 3.4
def test_cholesky_distance_and_logdet():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 6))
    S = A @ A.T + 6 * np.eye(6)
    X = rng.standard_normal((50, 6))
    mu = rng.standard_normal(6)
    brute = np.array([(x - mu) @ np.linalg.inv(S) @ (x - mu) for x in X])
    np.testing.assert_allclose(O.mahalanobis_d2(X, mu, S), brute, rtol=1e-11)
    assert O.logdet(S) == pytest.approx(math.log(np.linalg.det(S)), rel=1e-12)
    assert O.kappa1(np.diag([1.0, 10.0, 100.0])) == pytest.approx(100.0)


# ------------------------------------------------------ C-step (Section 2.1)
@pytest.mark.parametrize("seed", range(4))
def test_cstep_determinant_non_increasing(seed):
    fr = datagen.contaminated_gaussian(3000, 4, eps=0.2, kind="shift", shift=4.0, seed=seed)
    f = O.fit(fr.X, fr.h)
    for b in f.blocks:
        for ch in b.chains:
            if ch is not None and ch.ok:
                assert np.all(np.diff(ch.logdets) <= 1e-12), ch.logdets


def test_cstep_fixed_point_of_exact_mcd():
    rng = np.random.default_rng(7)
    X = np.vstack([rng.standard_normal((11, 2)), 6 + rng.standard_normal((3, 2))])
    h = 10
    mu, C, H = O.exact_mcd(X, h)
    ch = O.csteps(X, mu, C, h)
    # step 1 reproduces H, step 2 confirms it (no H_old before step 1)
    assert ch.ok and np.array_equal(ch.H, H) and ch.steps == 2
    assert ch.logdets[0] == ch.logdets[1]


def test_exact_mcd_bounds_rt_detmcd():
    for seed in range(3):
        rng = np.random.default_rng(seed)
        X = np.vstack([rng.standard_normal((11, 2)) @ np.array([[1, 0.6], [0, 0.8]]),
                       np.array([12.0, -9.0]) + 0.3 * rng.standard_normal((3, 2))])
        h = 10
        mu_e, C_e, H_e = O.exact_mcd(X, h)
        f = O.fit(X, h)
        ch = f.blocks[0].chains[f.blocks[0].chosen]
        ld_rt = np.linalg.slogdet(ch.Sigma * np.outer(f.s_uni, f.s_uni))[1]  # X units
        ld_ex = np.linalg.slogdet(C_e)[1]
        assert ld_rt >= ld_ex - 1e-12
        # clean cluster + far outliers: the deterministic fit finds the optimum
        assert np.array_equal(ch.H, H_e)


# ---------------------------------------------------------------- Section 3.5
@pytest.mark.parametrize("seed", range(3))
def test_update_cstep_equals_recompute(seed):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((400, 5)) + 3.0
    h = 300
    H_old = np.zeros(400, bool)
    H_old[rng.choice(400, h, replace=False)] = True
    H_new = H_old.copy()
    flip_in = rng.choice(np.flatnonzero(~H_old), 17, replace=False)
    flip_out = rng.choice(np.flatnonzero(H_old), 17, replace=False)
    H_new[flip_in] = True
    H_new[flip_out] = False
    mu_o, Lam_o = O.subset_estimates(Z, H_old)
    mu_u, Lam_u, hh = O.update_cstep(Z, mu_o, Lam_o, h, H_old, H_new)
    mu_r, Lam_r = O.subset_estimates(Z, H_new)
    assert hh == h
    np.testing.assert_allclose(mu_u, mu_r, rtol=1e-12)
    np.testing.assert_allclose(Lam_u, Lam_r, rtol=1e-10)
    # det(Lambda + delta u v^T) = (1 + delta v^T Lambda^-1 u) det(Lambda)
    u, v = rng.standard_normal(5), rng.standard_normal(5)
    for delta in (+1, -1):
        lhs = np.linalg.det(Lam_r + delta * np.outer(u, v))
        rhs = (1 + delta * v @ np.linalg.solve(Lam_r, u)) * np.linalg.det(Lam_r)
        assert lhs == pytest.approx(rhs, rel=1e-10)


# ---------------------------------------------------------------- Section 4
def test_block_count_table4():
    rows = [l.split() for l in open(os.path.join(GOLD, "table4_block_counts.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) > 40
    for lg, om, p, q in rows:
        assert O.block_count(2 ** int(lg), int(p), int(om)) == int(q), (lg, om, p)


def test_partition_permutation():
    for n in (1, 2, 3, 17, 1000, 4097):
        perm = O.partition_permutation(n, 5)
        assert np.array_equal(np.sort(perm), np.arange(n))
    a = O.partition_permutation(5000, 0)
    b = O.partition_permutation(5000, 1)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, O.partition_permutation(5000, 0))
    # looks random: the first block holds about its share of the first half
    assert abs(np.mean(a[:1000] < 2500) - 0.5) < 0.06


def test_kl_deviation_properties():
    rng = np.random.default_rng(0)
    A = np.diag([1.0, 2.0, 0.5])
    B = np.diag([2.0, 1.0, 0.25])
    expect = sum(r - 1 - math.log(r) for r in (0.5, 2.0, 2.0))
    assert O.kl_cov(A, B) == pytest.approx(expect, rel=1e-12)
    assert O.kl_cov(B, A) != pytest.approx(O.kl_cov(A, B))
    M = rng.standard_normal((4, 4))
    S = M @ M.T + np.eye(4)
    assert O.kl_deviation(np.ones(4), S, np.ones(4), S) == pytest.approx(0.0, abs=1e-12)
    a, b = rng.standard_normal(4), rng.standard_normal(4)
    assert O.kl_deviation(a, S, b, S) == pytest.approx((a - b) @ np.linalg.solve(S, a - b), rel=1e-12)
    assert O.kl_deviation(a, 2 * S, b, S) > 0


def test_bennett_pool_equals_union():
    rng = np.random.default_rng(4)
    c = 1.3
    parts = [rng.standard_normal((n, 3)) + rng.standard_normal(3) for n in (50, 80, 65)]
    fits = [(P.mean(0), c * np.cov(P, rowvar=False, ddof=1), P.shape[0]) for P in parts]
    mu, S, n = O.pool(fits, c)
    U = np.vstack(parts)
    assert n == U.shape[0]
    np.testing.assert_allclose(mu, U.mean(0), rtol=1e-12)
    np.testing.assert_allclose(S, c * np.cov(U, rowvar=False, ddof=1), rtol=1e-11)


# ------------------------------------------------------ invariants of the fit
def _transform_case():
    fr = datagen.contaminated_gaussian(4000, 4, eps=0.1, kind="point", shift=8.0, seed=3)
    return fr.X.astype(np.float64), fr.h


def test_fit_equivariance_sign_scale_shift_permutation():
    X, h = _transform_case()
    f = O.fit(X, h)
    P = np.array([2, 0, 3, 1])
    s = np.array([2.0, -0.5, 1.0, -4.0])          # powers of two: exact in FP
    b = np.array([10.0, -3.0, 0.25, 7.0])
    Y = (X[:, P] * s) + b
    g = O.fit(Y, h)
    np.testing.assert_allclose(g.mu, f.mu[P] * s + b, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(g.Sigma, f.Sigma[np.ix_(P, P)] * np.outer(s, s), rtol=1e-8, atol=1e-10)
    assert np.array_equal(g.flags, f.flags)
    np.testing.assert_allclose(g.d2, f.d2, rtol=1e-8)


def test_cstep_affine_equivariance():
    X, h = _transform_case()
    rng = np.random.default_rng(9)
    A = rng.standard_normal((4, 4)) + 3 * np.eye(4)
    b = rng.standard_normal(4)
    mu0 = np.median(X, axis=0)
    S0 = np.cov(X[:1500], rowvar=False)
    c1 = O.csteps(X, mu0, S0, h)
    c2 = O.csteps(X @ A.T + b, A @ mu0 + b, A @ S0 @ A.T, h)
    assert np.array_equal(c1.H, c2.H) and c1.steps == c2.steps


def test_clean_gaussian_consistency():
    fr = datagen.contaminated_gaussian(200_000, 5, eps=0.0, kind="point", shift=0.0, seed=1)
    f = O.fit(fr.X, fr.h)
    assert np.max(np.abs(f.Sigma - fr.R)) < 0.03
    assert np.max(np.abs(f.mu)) < 0.02
    assert abs(f.flags.mean() - 0.025) < 0.003
    assert np.max(np.abs(f.Sigma_raw - fr.R)) < 0.05


def test_outliers_detected_small_case():
    fr = datagen.small_fp64_case()
    f = O.fit(fr.X, fr.h)
    assert f.q == 1
    assert np.all(f.flags[fr.outlier])
    assert not np.any(f.subset_mask()[fr.outlier])
    assert O.kl_cov(f.Sigma, fr.R) < 0.02


# ------------------------------------------------ warm start (end of Section 4)
def test_warm_start_scale_free_and_runs_one_chain():
    """R13: C-steps rank distances, which a positive factor on the warm
    scatter does not change; the standardisation by the warm diagonal
    absorbs it.  So the fit from (mu, 4 Sigma) equals the fit from
    (mu, Sigma), and each block runs exactly one chain."""
    fr = datagen.contaminated_gaussian(6000, 4, eps=0.15, kind="cluster", shift=6.0, seed=11)
    base = O.fit(fr.X, fr.h, q=3)
    a = O.fit(fr.X, fr.h, q=3, init=(base.mu, base.Sigma))
    b = O.fit(fr.X, fr.h, q=3, init=(base.mu, 4.0 * base.Sigma))
    np.testing.assert_allclose(a.mu, b.mu, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a.Sigma, b.Sigma, rtol=1e-10, atol=1e-12)
    assert np.array_equal(a.flags, b.flags)
    for blk in a.blocks:
        assert blk.chains[1] is None and blk.chains[0] is not None and blk.chosen == 0


def test_warm_start_from_separated_optimum_keeps_it():
    """On well-separated data the exact MCD optimum is a C-step fixed point
    (A7 theorem); a warm start at the optimum's (mean, covariance) with q=1
    stays on the optimal h-subset."""
    rng = np.random.default_rng(5)
    X = np.vstack([rng.standard_normal((12, 2)), rng.standard_normal((4, 2)) * 0.3 + 40.0])
    h = 9
    mu_e, S_e, H_e = O.exact_mcd(X, h)[:3]
    f = O.fit(X, h, q=1, init=(mu_e, S_e))
    assert np.array_equal(f.blocks[0].chains[0].H, H_e)


# -------------------------------- adjoint of steps 8-10 with W fixed (Section 4)
def test_fixed_set_gradient_matches_central_differences():
    """The closed-form gradient against central differences of the fixed-set
    objective (step 1e-5 in FP64), on every coordinate of a few rows inside
    and outside W."""
    rng = np.random.default_rng(2)
    n, p = 300, 4
    X = rng.standard_normal((n, p)) @ np.diag([1.0, 2.0, 0.5, 1.5])
    W = np.zeros(n, bool)
    W[rng.permutation(n)[:200]] = True
    c = 1.2
    G = O.fixed_set_gradient(X, W, c, w_logdet=0.7, w_rd=1.3)
    eps = 1e-5
    for i in [0, 7, 50, 123, 299]:
        for k in range(p):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, k] += eps
            Xm[i, k] -= eps
            fd = (O.fixed_set_objective(Xp, W, c, 0.7, 1.3) - O.fixed_set_objective(Xm, W, c, 0.7, 1.3)) / (2 * eps)
            assert fd == pytest.approx(G[i, k], rel=1e-6, abs=1e-7)


def test_fixed_set_gradient_logdet_sums_to_zero_and_is_scale_covariant():
    """log det Sigma is translation invariant (the W-gradient sums to 0) and
    log det (a^2 Sigma) changes by a constant, so its gradient scales by 1/a."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((120, 3))
    W = rng.random(120) < 0.7
    g1 = O.fixed_set_gradient(X, W, 1.0, w_logdet=1.0, w_rd=0.0)
    np.testing.assert_allclose(g1.sum(axis=0), 0.0, atol=1e-12)
    g2 = O.fixed_set_gradient(3.0 * X, W, 1.0, w_logdet=1.0, w_rd=0.0)
    np.testing.assert_allclose(g2, g1 / 3.0, rtol=1e-12, atol=1e-14)


def test_fixed_set_vjp_matches_central_differences():
    """The VJP of (mu, Sigma, log det Sigma, RD) with W fixed against central
    differences of the contracted outputs (step 1e-5 in FP64), for random
    cotangents on all four outputs, on rows inside and outside W."""
    rng = np.random.default_rng(12)
    n, p = 200, 3
    X = rng.standard_normal((n, p)) @ np.array([[1.0, 0.3, 0.0], [0.0, 2.0, 0.5], [0.0, 0.0, 0.7]])
    W = rng.random(n) < 0.7
    c = 1.15
    gmu = rng.standard_normal(p)
    gS = rng.standard_normal((p, p))
    gld = 0.8
    gRD = rng.standard_normal(n)

    def L(Xv):
        mu, S, ld, rd = O.fixed_set_outputs(Xv, W, c)
        return gmu @ mu + np.sum(gS * S) + gld * ld + gRD @ rd

    G = O.fixed_set_vjp(X, W, c, gmu, gS, gld, gRD)
    eps = 1e-5
    for i in [0, 3, 17, 88, 150, 199]:
        for k in range(p):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, k] += eps
            Xm[i, k] -= eps
            fd = (L(Xp) - L(Xm)) / (2 * eps)
            assert fd == pytest.approx(G[i, k], rel=1e-6, abs=1e-7), (i, k)


def test_fixed_set_vjp_reduces_to_scalar_objective_gradient():
    """gRD = w_rd on every row, g_logdet = w_ld, gmu = gSigma = 0 is the scalar
    objective w_ld log det Sigma + w_rd sum RD."""
    rng = np.random.default_rng(13)
    X = rng.standard_normal((150, 4))
    W = rng.random(150) < 0.8
    a = O.fixed_set_vjp(X, W, 1.3, g_logdet=0.6, gRD=np.full(150, 1.7))
    b = O.fixed_set_gradient(X, W, 1.3, w_logdet=0.6, w_rd=1.7)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)
