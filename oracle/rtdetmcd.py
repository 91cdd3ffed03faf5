"""RT-DetMCD oracle: plain, slow, float64 (test infrastructure only).

Every function cites the passage of arXiv 1910.05615 it restates.  Section
numbers are the paper's: Section 2.1 (MCD, C-step, reweighting), Section 3.1
(univariate MCD standardisation), Section 3.2 (wrapping and GSSCM starts),
Section 3.3 (refinement), Section 3.4 (Cholesky distances and the condition
monitor), Section 3.5 (update-based C-step), Section 4 (blocks, aggregation,
parallel reweighting), Section 5 (block-count rule, eq. partitionsize).

Readings where the paper is silent or ambiguous (each is also listed in the
project's design notes):
  R1  c(alpha) = alpha / F_{chi2_{p+2}}(chi2_{p,alpha})  (Croux-Haesbroeck
      consistency factor, cited but not printed in Section 2.1).
  R2  univariate reweighted MCD: raw window variance uses denominator h-1 and
      c(alpha~) with p=1; reweighting keeps (x-mu0)^2/s0^2 <= chi2_{1,0.975};
      the reweighted variance uses denominator n_w-1 times
      c_rew = 0.975 / F_{chi2_3}(chi2_{1,0.975}).
  R3  GSSCM cutoffs: A = median ||z||; B = (m3 + Phi^-1(0.75)*1.4826*MAD3)^1.5
      with m3, MAD3 the median and raw MAD of ||z||^(2/3).  Medians of even
      counts are the mean of the two middle values.
  R4  random partition: the Feistel/SplitMix64 permutation in
      `partition_permutation`; q = 1 uses the identity order.
  R5  condition monitor uses the exact kappa_1 = ||S||_1 ||S^-1||_1 (the paper
      uses Higham's estimator of the same quantity).  If the very first
      C-step of a start is refused the start yields no fit.
  R6  C-step subsets: distances sorted ascending, ties to the lower position
      within the block.  Iterate until H_new = H_old or 100 steps.
  R7  pooling (Section 4 step 7) pools the actual h-subsets: counts h_b and
      sscp (h_b-1) Sigma_l / c(alpha); Sigma_raw = c(alpha) Lambda/(n-1).
  R8  reweighted scatter multiplied by c_rew = 0.975/F_{chi2_{p+2}}(chi2_{p,0.975})
      (reweight_consistency=1, default).  0 gives the literal plain covariance;
      2 uses c(|W|/n) at the fraction of rows kept.
  R9  KL of Section 4 step 6 uses log|det(A B^-1)| (A may be indefinite).
  R10 block count q = max(floor(n/(p omega)), 1) capped at QMAX = 1024 blocks
      (the paper caps q by the number of CPU cores instead); an explicit q
      above QMAX is refused.
  R11 step 4 keeps start 1 when the two determinants tie ("<="); two starts
      that reach the same h-subset tie exactly.
  R13 warm start (end of Section 4): a run's final (mu, Sigma) as the input
      to step 3 of the next; blocks kept, steps 1-2 and the univariate
      standardisation skipped, Z standardised by the warm fit's centre and
      diagonal, one chain per block.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
from scipy import stats
from scipy.linalg import solve_triangular

KAPPA_MAX = 1000.0          # Section 3.3 step 2 and Section 3.4
OMEGA = 4096                # Section 5, default omega = 2^12
QMAX = 1024                 # largest number of blocks (reading R10)
WRAP_B, WRAP_C = 1.5, 4.0   # Section 3.2, eq. wrapping
WRAP_Q1, WRAP_Q2 = 1.541, 0.862
CUTOFF_Q = 0.975            # Section 2.1
MAX_CSTEPS = 100
PHI_INV_075 = 0.6744897501960817   # standard normal 0.75 quantile
MAD_CONST = 1.4826


class OracleError(ValueError):
    pass


# ----------------------------------------------------------------------------
# Distribution constants (Section 2.1)
# ----------------------------------------------------------------------------
def chi2_ppf(q: float, p: int) -> float:
    return float(stats.chi2.ppf(q, p))


def chi2_cdf(x: float, p: int) -> float:
    return float(stats.chi2.cdf(x, p))


def consistency_factor(alpha: float, p: int) -> float:
    """c(alpha) of eq. mcdraw (reading R1)."""
    return alpha / chi2_cdf(chi2_ppf(alpha, p), p + 2)


def reweight_factor(p: int, q: float = CUTOFF_Q) -> float:
    """Consistency factor of the reweighted scatter (reading R8)."""
    return q / chi2_cdf(chi2_ppf(q, p), p + 2)


# ----------------------------------------------------------------------------
# Section 3.1: univariate reweighted MCD
# ----------------------------------------------------------------------------
@dataclass
class UniMCD:
    mu: float          # reweighted location
    s2: float          # reweighted scale^2
    mu_raw: float
    s2_raw: float
    j: int             # start of the minimum-variance window in sorted order
    n_w: int           # rows kept by the reweighting


def univariate_mcd(x, cutoff_q: float = CUTOFF_Q) -> UniMCD:
    """Univariate reweighted MCD with coverage h~ = [n/2] + 1 (Section 3.1).

    Sort, then slide over the contiguous h~-windows of the sorted values,
    keeping the window of smallest variance (first one on ties).  The window
    sums are taken as differences of running sums of values shifted by the
    middle order statistic.  Raw and reweighted estimates per reading R2.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        raise OracleError("univariate MCD needs n >= 2")
    h = n // 2 + 1
    s = np.sort(x)
    c = s[n // 2]
    d = s - c
    P1 = np.concatenate(([0.0], np.cumsum(d)))
    P2 = np.concatenate(([0.0], np.cumsum(d * d)))
    j = np.arange(n - h + 1)
    S1 = P1[j + h] - P1[j]
    S2 = P2[j + h] - P2[j]
    var = (S2 - S1 * S1 / h) / (h - 1)
    jstar = int(np.argmin(var))
    mu0 = c + S1[jstar] / h
    s2_0 = consistency_factor(h / n, 1) * var[jstar]
    if not s2_0 > 0.0:
        raise OracleError("univariate MCD: zero scale (more than half the "
                          "values are equal)")
    keep = (x - mu0) ** 2 / s2_0 <= chi2_ppf(cutoff_q, 1)
    xw = x[keep]
    n_w = xw.size
    mu = float(xw.mean())
    s2 = reweight_factor(1, cutoff_q) * float(np.sum((xw - mu) ** 2)) / (n_w - 1)
    return UniMCD(mu, s2, float(mu0), float(s2_0), jstar, int(n_w))


def univariate_mcd_bruteforce(x):
    """Raw univariate MCD by enumerating every h~-subset (tiny n only)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    h = n // 2 + 1
    best = None
    for H in itertools.combinations(range(n), h):
        v = x[list(H)].var(ddof=1)
        if best is None or v < best[0]:
            best = (v, x[list(H)].mean())
    return best[1], consistency_factor(h / n, 1) * best[0]


# ----------------------------------------------------------------------------
# Section 4 (random partition) and Section 5 (eq. partitionsize)
# ----------------------------------------------------------------------------
def block_count(n: int, p: int, omega: int = OMEGA) -> int:
    """q = max(floor(n / (p omega)), 1)   (eq. partitionsize), at most QMAX
    (reading R10)."""
    return min(max(n // (p * omega), 1), QMAX)


_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(z):
    """SplitMix64 output function (Steele, Lea, Flood 2014), on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def partition_permutation(n: int, seed: int) -> np.ndarray:
    """Random order of the rows for the block partition (reading R4).

    A 4-round balanced Feistel network on k-bit integers (k the smallest even
    number >= 2 with 2^k >= n) whose round function is SplitMix64 keyed by
    SplitMix64(seed + r), restricted to [0, n) by cycle walking.  Position t of
    the permuted order holds row perm[t].
    """
    k = 2
    while (1 << k) < n:
        k += 2
    half = k // 2
    mask = np.uint64((1 << half) - 1)
    hs = np.uint64(half)
    keys = [splitmix64(np.uint64((seed + r) & 0xFFFFFFFFFFFFFFFF))
            for r in range(4)]

    def one_pass(t):
        L = t >> hs
        R = t & mask
        for r in range(4):
            L, R = R, L ^ (splitmix64(keys[r] ^ R) & mask)
        return (L << hs) | R

    t = np.arange(n, dtype=np.uint64)
    y = one_pass(t)
    bad = y >= np.uint64(n)
    while bad.any():
        y[bad] = one_pass(y[bad])
        bad = y >= np.uint64(n)
    return y.astype(np.int64)


# ----------------------------------------------------------------------------
# Section 3.2: the two initial estimators
# ----------------------------------------------------------------------------
def wrap(z):
    """Wrapping function g of eq. wrapping (b=1.5, c=4, q1=1.541, q2=0.862)."""
    z = np.asarray(z, dtype=np.float64)
    a = np.abs(z)
    mid = WRAP_Q1 * np.tanh(WRAP_Q2 * (WRAP_C - a)) * np.sign(z)
    return np.where(a <= WRAP_B, z, np.where(a <= WRAP_C, mid, 0.0))


def start_wrap(Z) -> np.ndarray:
    """S~_1: classical covariance (denominator n-1) of the wrapped data."""
    return np.cov(wrap(Z), rowvar=False, ddof=1).reshape(Z.shape[1], Z.shape[1])


def gsscm_cutoffs(r):
    """(A, B) of the linearly redescending xi (reading R3)."""
    r = np.asarray(r, dtype=np.float64)
    A = float(np.median(r))
    r23 = r ** (2.0 / 3.0)
    m3 = float(np.median(r23))
    mad3 = float(np.median(np.abs(r23 - m3)))
    B = (m3 + PHI_INV_075 * MAD_CONST * mad3) ** 1.5
    return A, float(B)


def xi_weight(r, A, B):
    """Linearly redescending weight xi(r) of Section 3.2."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    out[r <= A] = 1.0
    mid = (r > A) & (r <= B)
    out[mid] = (B - r[mid]) / (B - A)
    return out


def start_gsscm(Z) -> np.ndarray:
    """S~_2 = (1/n) sum xi^2(||z_i||) z_i z_i^T   (eq. LR), z not re-centred."""
    Z = np.asarray(Z, dtype=np.float64)
    r = np.sqrt(np.sum(Z * Z, axis=1))
    A, B = gsscm_cutoffs(r)
    w = xi_weight(r, A, B) ** 2
    return (Z * w[:, None]).T @ Z / Z.shape[0]


# ----------------------------------------------------------------------------
# Section 3.3: refinement
# ----------------------------------------------------------------------------
@dataclass
class Start:
    mu: np.ndarray
    Sigma: np.ndarray
    V: np.ndarray
    lam: np.ndarray
    D: np.ndarray


def refine(Z, S, kappa_max: float = KAPPA_MAX):
    """Refine an initial scatter S (Section 3.3).  Returns None when
    lambda_1/lambda_p exceeds kappa_max (the start is dropped)."""
    Z = np.asarray(Z, dtype=np.float64)
    lam, V = np.linalg.eigh(S)
    order = np.argsort(-lam, kind="stable")
    lam, V = lam[order], V[:, order]
    if not lam[-1] > 0.0 or lam[0] / lam[-1] > kappa_max:
        return None
    T = Z @ V
    D = np.array([univariate_mcd(T[:, j]).s2 for j in range(T.shape[1])])
    Sigma = (V * D) @ V.T
    S_mhalf = (V * D ** -0.5) @ V.T
    S_half = (V * D ** 0.5) @ V.T
    Zt = Z @ S_mhalf
    mut = np.array([univariate_mcd(Zt[:, j]).mu for j in range(Zt.shape[1])])
    return Start(S_half @ mut, Sigma, V, lam, D)


# ----------------------------------------------------------------------------
# Sections 2.1, 3.4: C-steps with Cholesky distances and condition monitor
# ----------------------------------------------------------------------------
def kappa1(S) -> float:
    """||S||_1 ||S^-1||_1 (exact; reading R5)."""
    return float(np.abs(S).sum(axis=0).max() * np.abs(np.linalg.inv(S)).sum(axis=0).max())


def mahalanobis_d2(Z, mu, Sigma) -> np.ndarray:
    """d^2 = ||L^-1 (z - mu)||^2 with Sigma = L L^T (Section 3.4)."""
    L = np.linalg.cholesky(Sigma)
    Y = solve_triangular(L, (np.asarray(Z, np.float64) - mu).T, lower=True)
    return np.sum(Y * Y, axis=0)


def mahalanobis_d2_plain(X, mu, Sigma) -> np.ndarray:
    """d^2 = (x - mu)^T Sigma^-1 (x - mu) by a linear solve (Section 2.1)."""
    C = np.asarray(X, np.float64) - mu
    return np.einsum("ij,ij->i", C, np.linalg.solve(Sigma, C.T).T)


def csubset(d2, h: int) -> np.ndarray:
    """H_new: the h smallest distances, ties to the lower position (R6)."""
    order = np.argsort(d2, kind="stable")
    H = np.zeros(d2.size, dtype=bool)
    H[order[:h]] = True
    return H


def subset_estimates(Z, H):
    """Mean and sscp of an h-subset (eqs. cstep4a, cstep4b)."""
    Zh = Z[H]
    mu = Zh.mean(axis=0)
    C = Zh - mu
    return mu, C.T @ C


@dataclass
class Chain:
    mu: np.ndarray | None = None        # final centre
    Sigma: np.ndarray | None = None     # final Lambda/(h-1), no c(alpha)
    H: np.ndarray | None = None         # final h-subset (bool over block rows)
    steps: int = 0
    status: str = "converged"
    logdets: list = field(default_factory=list)

    @property
    def ok(self):
        return self.H is not None


def csteps(Z, mu, Sigma, h: int, kappa_max: float = KAPPA_MAX,
           max_steps: int = MAX_CSTEPS) -> Chain:
    """Iterate C-steps from (mu, Sigma) until the h-subset repeats.

    Each step: condition monitor on Sigma_old (Section 3.4), distances via
    Cholesky, sort, first h, new mean and covariance (Section 2.1).
    """
    Z = np.asarray(Z, dtype=np.float64)
    ch = Chain()
    prev = None
    for _ in range(max_steps):
        try:
            np.linalg.cholesky(Sigma)
        except np.linalg.LinAlgError:
            ch.status = "illcond"
            break
        if kappa1(Sigma) >= kappa_max:
            ch.status = "illcond"
            break
        d2 = mahalanobis_d2(Z, mu, Sigma)
        H = csubset(d2, h)
        mu_new, Lam = subset_estimates(Z, H)
        Sigma_new = Lam / (h - 1)
        ch.steps += 1
        ch.logdets.append(float(np.linalg.slogdet(Sigma_new)[1]))
        same = prev is not None and np.array_equal(H, prev)
        mu, Sigma, prev = mu_new, Sigma_new, H
        if same:
            break
    else:
        ch.status = "maxiter"
    if ch.steps == 0:
        return ch
    ch.mu, ch.Sigma, ch.H = mu, Sigma, prev
    return ch


def update_cstep(Z, mu, Lam, h: int, H_old, H_new):
    """Update-based C-step of Section 3.5, applied sequentially.

    Swaps are taken alternately (one entering, one leaving, ascending row
    order within each list) so that the running count stays in {h, h+1}.
    Returns (mu_new, Lambda_new, h).
    """
    Z = np.asarray(Z, dtype=np.float64)
    mu = np.array(mu, dtype=np.float64)
    Lam = np.array(Lam, dtype=np.float64)
    enter = list(np.flatnonzero(H_new & ~H_old))
    leave = list(np.flatnonzero(H_old & ~H_new))
    seq = []
    for a, b in itertools.zip_longest(enter, leave):
        if a is not None:
            seq.append((a, +1))
        if b is not None:
            seq.append((b, -1))
    for i, delta in seq:
        h = h + delta
        u = Z[i] - mu
        mu = mu + (delta / h) * u
        v = Z[i] - mu
        Lam = Lam + delta * np.outer(u, v)
    return mu, Lam, h


# ----------------------------------------------------------------------------
# Section 2.1: exact raw MCD by enumeration (tiny n only)
# ----------------------------------------------------------------------------
def exact_mcd(X, h: int):
    """Exact raw MCD: the h-subset whose covariance has least determinant.
    Returns (mu, covariance (h-1 denominator, no c(alpha)), H)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    best = None
    for H in itertools.combinations(range(n), h):
        Xh = X[list(H)]
        C = np.cov(Xh, rowvar=False, ddof=1).reshape(X.shape[1], X.shape[1])
        ld = np.linalg.slogdet(C)
        val = ld[1] if ld[0] > 0 else -np.inf
        if best is None or val < best[0]:
            best = (val, Xh.mean(axis=0), C, H)
    mask = np.zeros(n, dtype=bool)
    mask[list(best[3])] = True
    return best[1], best[2], mask


# ----------------------------------------------------------------------------
# Section 4 steps 5-7: aggregation
# ----------------------------------------------------------------------------
def kl_deviation(a, A, b, B) -> float:
    """KL[(a,A),(b,B)] of eq. KL (reading R9 for the log-determinant)."""
    Binv = np.linalg.inv(B)
    M = A @ Binv
    p = A.shape[0]
    logabsdet = np.linalg.slogdet(M)[1]
    d = np.asarray(a) - np.asarray(b)
    return float(np.trace(M) - p - logabsdet + d @ Binv @ d)


def kl_cov(A, B) -> float:
    """KL(A, B) without centres (Section 5 accuracy measure)."""
    p = A.shape[0]
    return kl_deviation(np.zeros(p), A, np.zeros(p), B)


def entrywise_median(arrs):
    return np.median(np.stack(arrs, axis=0), axis=0)


def pool(fits, c_alpha: float):
    """Single-pass (Bennett) pooling of Section 4 step 7 (reading R7).
    fits: list of (mu, Sigma_with_c, count)."""
    mu_p = np.array(fits[0][0], dtype=np.float64)
    n_p = fits[0][2]
    Lam_p = (n_p - 1) * fits[0][1] / c_alpha
    for mu, S, cnt in fits[1:]:
        d = mu - mu_p
        Lam = (cnt - 1) * S / c_alpha
        Lam_p = Lam_p + Lam + np.outer(d, d) * (n_p * cnt / (n_p + cnt))
        mu_p = (n_p * mu_p + cnt * mu) / (n_p + cnt)
        n_p = n_p + cnt
    return mu_p, c_alpha * Lam_p / (n_p - 1), n_p


# ----------------------------------------------------------------------------
# The whole method (Section 4, steps 1-10)
# ----------------------------------------------------------------------------
@dataclass
class Block:
    rows: np.ndarray                # original row indices, in block order
    S: list                         # [S~_1, S~_2]
    starts: list                    # [Start | None, Start | None]
    chains: list                    # [Chain | None, Chain | None]
    chosen: int = -1                # 0 / 1, -1 when the block has no fit
    mu: np.ndarray | None = None    # raw block fit (Z units)
    Sigma: np.ndarray | None = None  # c(alpha) * Lambda/(h_b - 1)  (Z units)


@dataclass
class Fit:
    mu: np.ndarray            # reweighted centre, X units
    Sigma: np.ndarray         # reweighted scatter, X units
    mu_raw: np.ndarray
    Sigma_raw: np.ndarray
    d2: np.ndarray            # final squared robust distances, all n rows
    flags: np.ndarray         # d2 > chi2_{p,0.975}
    d2_raw: np.ndarray        # squared distances to the raw fit (block rows)
    W: np.ndarray             # reweighting set (bool over all n; False on
                              # discarded rows)
    mu_uni: np.ndarray
    s_uni: np.ndarray
    q: int
    m: int
    h_b: int
    perm: np.ndarray
    blocks: list
    kept: list                # blocks kept by step 7
    kl: np.ndarray
    c_alpha: float
    cutoff_d2: float
    mu_z: np.ndarray
    Sigma_z: np.ndarray
    mu_raw_z: np.ndarray
    Sigma_raw_z: np.ndarray

    def subset_mask(self) -> np.ndarray:
        """Final h-subsets of the chosen chains, as a bool mask over rows."""
        out = np.zeros(self.d2.size, dtype=bool)
        for b in self.blocks:
            if b.chosen >= 0:
                out[b.rows[b.chains[b.chosen].H]] = True
        return out


def validate(n: int, p: int, h: int):
    """Section 2.1: [(n+p+1)/2] <= h < n and n > 2p."""
    if p < 1 or n <= 2 * p:
        raise OracleError("need p >= 1 and n > 2p")
    if not ((n + p + 1) // 2 <= h < n):
        raise OracleError("need [(n+p+1)/2] <= h < n")


def choose_start(chains) -> int:
    """Section 4 step 4: of the starts whose C-steps gave a fit, the one with
    the lower determinant; start 1 on ties (reading R11).  Returns 0, 1, or
    -1 when neither start gave a fit."""
    ok = [k for k in range(2) if chains[k] is not None and chains[k].ok]
    if not ok:
        return -1
    if len(ok) == 1:
        return ok[0]
    ld = [np.linalg.slogdet(chains[k].Sigma)[1] for k in range(2)]
    return 0 if ld[0] <= ld[1] else 1


def aggregate(fits, h_b: int, c_alpha: float):
    """Section 4 steps 5-7 from the block fits: fits[l] = (mu_l, c(alpha)
    Sigma_l) in Z units, or None for a block without a fit.  Entrywise
    median of the fitted blocks, KL deviation of each from it, keep the
    ceil(q_f/2) closest (stable order by KL), pool their h_b-subsets
    (reading R7).  With one block (q = 1) the raw fit is that block's.
    Returns (mu_raw, Sigma_raw, kept, kl); kl lists the fitted blocks."""
    fitted = [l for l in range(len(fits)) if fits[l] is not None]
    if not fitted:
        raise OracleError("every start of every block was ill-conditioned")
    if len(fits) == 1:
        return fits[0][0], fits[0][1], [0], np.zeros(1)
    mu_med = entrywise_median([fits[l][0] for l in fitted])
    S_med = entrywise_median([fits[l][1] for l in fitted])
    kl = np.array([kl_deviation(mu_med, S_med, fits[l][0], fits[l][1]) for l in fitted])
    order = np.argsort(kl, kind="stable")
    kept = [fitted[i] for i in order[: (len(fitted) + 1) // 2]]
    mu_raw, Sigma_raw, _ = pool([(fits[l][0], fits[l][1], h_b) for l in kept], c_alpha)
    return mu_raw, Sigma_raw, kept, kl


def block_start_unit(args):
    """Steps 1-3 of Section 4 for one start k of one block: the initial
    scatter S~_k (Section 3.2), its refinement (Section 3.3) and the C-steps
    (Sections 2.1, 3.4).  Returns (S~_k, Start | None, Chain | None).  The
    paper runs each block on its own thread; `fit` may map these units over
    host processes."""
    Zl, k, h_b, kappa_max, max_steps = args
    Sk = start_wrap(Zl) if k == 0 else start_gsscm(Zl)
    st = refine(Zl, Sk, kappa_max)
    if st is None:
        return Sk, None, None
    return Sk, st, csteps(Zl, st.mu, st.Sigma, h_b, kappa_max, max_steps)


def _column_mcd(args):
    x, cutoff_q = args
    return univariate_mcd(x, cutoff_q)


def fit(X, h: int, *, omega: int = OMEGA, seed: int = 0,
        kappa_max: float = KAPPA_MAX, cutoff_q: float = CUTOFF_Q,
        max_steps: int = MAX_CSTEPS, q: int | None = None,
        reweight_consistency: int = 1, init=None, map_fn=map) -> Fit:
    """init = (mu, Sigma) in X units: warm start (end of Section 4: the final
    estimate of a run as the input to step 3 of the next).  Reading R13:
    the blocks are kept (step 3 runs per block), steps 1-2 and the
    univariate standardisation are skipped; Z is standardised by the warm
    fit's own centre and diagonal, and each block runs one chain, from the
    warm fit.

    map_fn (default: the builtin map) evaluates the independent units, the
    column univariate MCDs and the (block, start) units of steps 1-3, in
    order; a process pool's map runs them on several host cores with the
    same results."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    validate(n, p, h)
    if q is not None and not 1 <= q <= QMAX:
        raise OracleError("need 1 <= q <= QMAX blocks (reading R10)")
    if init is not None:
        mu_uni = np.asarray(init[0], dtype=np.float64).reshape(p)
        S_init = np.asarray(init[1], dtype=np.float64).reshape(p, p)
        if not (np.all(np.isfinite(mu_uni)) and np.all(np.isfinite(S_init)) and np.all(np.diag(S_init) > 0)):
            raise OracleError("warm start needs a finite centre and a positive diagonal")
        s_uni = np.sqrt(np.diag(S_init))
    else:
        # Section 3.1 and Section 4 (eq. standardization): whole-X univariate MCD.
        uni = list(map_fn(_column_mcd, [(X[:, j], cutoff_q) for j in range(p)]))
        mu_uni = np.array([u.mu for u in uni])
        s_uni = np.sqrt(np.array([u.s2 for u in uni]))
    Z = (X - mu_uni) / s_uni
    # Section 4: random partition into q blocks of m rows (eq. partitionsize).
    if q is None:
        q = block_count(n, p, omega)
    m = n // q
    perm = np.arange(n) if q == 1 else partition_permutation(n, seed)
    h_b = h if q == 1 else (h * m) // n
    if h_b <= p:
        raise OracleError("block subset size h_b must exceed p")
    alpha = h / n
    c_alpha = consistency_factor(alpha, p)
    blocks = []
    if init is None:
        # Steps 1-3 for every (block, start): initial scatter, refinement,
        # C-steps; independent units.
        units = list(map_fn(block_start_unit,
                            [(Z[perm[l * m:(l + 1) * m]], k, h_b, kappa_max, max_steps)
                             for l in range(q) for k in range(2)]))
    for l in range(q):
        rows = perm[l * m:(l + 1) * m]
        if init is not None:
            # warm start: step 3 only, from the warm fit (Z units)
            S = [None, None]
            starts = [None, None]
            Sz = S_init / np.outer(s_uni, s_uni)
            chains = [csteps(Z[rows], np.zeros(p), Sz, h_b, kappa_max, max_steps), None]
        else:
            S = [units[2 * l][0], units[2 * l + 1][0]]
            starts = [units[2 * l][1], units[2 * l + 1][1]]
            chains = [units[2 * l][2], units[2 * l + 1][2]]
        b = Block(rows, S, starts, chains)
        b.chosen = choose_start(chains)
        if b.chosen >= 0:
            ch = chains[b.chosen]
            b.mu, b.Sigma = ch.mu, c_alpha * ch.Sigma
        blocks.append(b)
    mu_raw, Sigma_raw, kept, kl = aggregate(
        [(b.mu, b.Sigma) if b.chosen >= 0 else None for b in blocks], h_b, c_alpha)
    # Steps 8-9: reweighting over the rows of all blocks.
    cutoff_d2 = chi2_ppf(cutoff_q, p)
    used = perm[: q * m]
    d2_raw = np.full(n, np.nan)
    d2_raw[used] = mahalanobis_d2(Z[used], mu_raw, Sigma_raw)
    W = np.zeros(n, dtype=bool)
    W[used] = d2_raw[used] <= cutoff_d2
    Zw = Z[W]
    mu_z = Zw.mean(axis=0)
    Sigma_z = np.cov(Zw, rowvar=False, ddof=1).reshape(p, p)
    if reweight_consistency == 1:
        Sigma_z = reweight_factor(p, cutoff_q) * Sigma_z
    elif reweight_consistency == 2:
        Sigma_z = consistency_factor(Zw.shape[0] / n, p) * Sigma_z
    # Step 10: final distances and flags for every row.
    d2 = mahalanobis_d2(Z, mu_z, Sigma_z)
    flags = d2 > cutoff_d2
    # Back to X units: mu_x = mu_uni + D mu_z, Sigma_x = D Sigma_z D.
    D = s_uni
    return Fit(mu=mu_uni + D * mu_z, Sigma=Sigma_z * np.outer(D, D),
               mu_raw=mu_uni + D * mu_raw, Sigma_raw=Sigma_raw * np.outer(D, D),
               d2=d2, flags=flags, d2_raw=d2_raw, W=W, mu_uni=mu_uni,
               s_uni=s_uni, q=q, m=m, h_b=h_b, perm=perm, blocks=blocks,
               kept=kept, kl=kl, c_alpha=c_alpha, cutoff_d2=cutoff_d2,
               mu_z=mu_z, Sigma_z=Sigma_z, mu_raw_z=mu_raw,
               Sigma_raw_z=Sigma_raw)


def logdet(S) -> float:
    """log det via Cholesky: 2 sum log L_jj (Section 3.4)."""
    return float(2.0 * np.sum(np.log(np.diag(np.linalg.cholesky(S)))))




# ----------------------------------------------------------------------------
# Adjoint of Section 4 steps 8-10 with the reweighting set W fixed
# ----------------------------------------------------------------------------
def fixed_set_objective(X, W, c, w_logdet=1.0, w_rd=1.0):
    """f(X) = w_logdet log det Sigma + w_rd sum_j RD_j, with mu = mean of the
    rows in W, Sigma = c * (sample covariance of W, denominator |W|-1) and
    RD_j = sqrt((x_j - mu)^T Sigma^-1 (x_j - mu)) over all rows (steps 8-10
    with W held fixed)."""
    X = np.asarray(X, dtype=np.float64)
    Xw = X[W]
    mu = Xw.mean(axis=0)
    S = c * np.cov(Xw, rowvar=False, ddof=1).reshape(X.shape[1], X.shape[1])
    L = np.linalg.cholesky(S)
    Y = solve_triangular(L, (X - mu).T, lower=True)
    rd = np.sqrt(np.sum(Y * Y, axis=0))
    return w_logdet * float(2.0 * np.sum(np.log(np.diag(L)))) + w_rd * float(rd.sum())


def fixed_set_gradient(X, W, c, w_logdet=1.0, w_rd=1.0):
    """Gradient of fixed_set_objective with respect to X, from the closed
    forms: with r_i = x_i - mu, u_i = Sigma^-1 r_i, N = |W|,
      d log det Sigma / d x_i = [i in W] 2 c/(N-1) u_i   (Sigma^-1 = S_W^-1 / c),
      d sum RD / d x_i = u_i/RD_i + [i in W] (g/N + 2 c/(N-1) G r_i),
      g = -sum_j u_j/RD_j,   G = -1/2 sum_j u_j u_j^T / RD_j.
    Rows with RD_i = 0 take the zero subgradient of their own term."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=bool)
    N = int(W.sum())
    Xw = X[W]
    mu = Xw.mean(axis=0)
    S = c * np.cov(Xw, rowvar=False, ddof=1).reshape(X.shape[1], X.shape[1])
    Sinv = np.linalg.inv(S)
    R = X - mu
    U = R @ Sinv
    rd = np.sqrt(np.einsum("ij,ij->i", R, U))
    inv = np.where(rd > 0, 1.0 / np.where(rd > 0, rd, 1.0), 0.0)
    g = -(U * inv[:, None]).sum(axis=0)
    G = -0.5 * (U * inv[:, None]).T @ U
    grad = w_rd * U * inv[:, None]
    grad[W] += w_rd * (g / N + (2.0 * c / (N - 1)) * (R[W] @ G))
    grad[W] += w_logdet * (2.0 * c / (N - 1)) * U[W]
    return grad


def fixed_set_outputs(X, W, c):
    """(mu, Sigma, log det Sigma, RD) of the reweighted fit with the set W
    held fixed (steps 8-10): mu = mean of W, Sigma = c * (covariance of W,
    denominator |W| - 1), RD over all rows."""
    X = np.asarray(X, dtype=np.float64)
    Xw = X[np.asarray(W, dtype=bool)]
    mu = Xw.mean(axis=0)
    S = c * np.cov(Xw, rowvar=False, ddof=1).reshape(X.shape[1], X.shape[1])
    L = np.linalg.cholesky(S)
    Y = solve_triangular(L, (X - mu).T, lower=True)
    return mu, S, float(2.0 * np.sum(np.log(np.diag(L)))), np.sqrt(np.sum(Y * Y, axis=0))


def fixed_set_vjp(X, W, c, gmu=None, gSigma=None, g_logdet=0.0, gRD=None):
    """d/dX of gmu.mu + <gSigma, Sigma> + g_logdet log det Sigma + gRD.RD for
    the outputs of fixed_set_outputs, from the chain rule.  With
    r_i = x_i - mu, u_i = Sigma^-1 r_i, omega_i = gRD_i / RD_i, N = |W|:
      the cotangents reaching mu and Sigma through RD and log det are
        gmu_t = gmu - sum_j omega_j u_j,
        G_t   = sym(gSigma) + g_logdet Sigma^-1 - 1/2 sum_j omega_j u_j u_j^T
      (dRD_j/dmu = -u_j/RD_j, dRD_j/dSigma = -u_j u_j^T/(2 RD_j),
      dlogdet/dSigma = Sigma^-1); then d mu/dx_i = [i in W] I/N and
      dSigma = c/(N-1) sum_W (dx r^T + r dx^T), so
        grad_i = omega_i u_i + [i in W] (gmu_t / N + 2 c/(N-1) G_t r_i).
    Rows with RD_i = 0 take the zero subgradient of their own term."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=bool)
    n, p = X.shape
    N = int(W.sum())
    mu, S, _, rd = fixed_set_outputs(X, W, c)
    Sinv = np.linalg.inv(S)
    R = X - mu
    U = R @ Sinv
    gmu = np.zeros(p) if gmu is None else np.asarray(gmu, dtype=np.float64)
    gS = np.zeros((p, p)) if gSigma is None else np.asarray(gSigma, dtype=np.float64)
    gRD = np.zeros(n) if gRD is None else np.asarray(gRD, dtype=np.float64)
    om = np.where(rd > 0, gRD / np.where(rd > 0, rd, 1.0), 0.0)
    gmu_t = gmu - (U * om[:, None]).sum(axis=0)
    G_t = 0.5 * (gS + gS.T) + g_logdet * Sinv - 0.5 * (U * om[:, None]).T @ U
    grad = U * om[:, None]
    grad[W] += gmu_t / N + (2.0 * c / (N - 1)) * (R[W] @ G_t)
    return grad


__all__ = [name for name in dir() if not name.startswith("_")]
