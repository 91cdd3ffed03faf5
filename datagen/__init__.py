"""Seeded synthetic inputs for RT-DetMCD (shared by the oracle tests, the GPU
tests and bench.py).

This module only draws random numbers and shapes them into data sets; it holds
none of the method's arithmetic.  The recipes follow the simulation design of
the paper (Section 5): clean rows from a Gaussian N(0, R) with unit diagonal,
contamination placed along the last eigenvector v of R, as point, cluster or
shift outliers.  R is a seeded random correlation matrix with a prescribed
condition number, drawn with scipy's random_correlation (the Davies-Higham
Givens construction).  Rows are returned as float32 row-major; the oracle and
the CUDA path both read those exact float32 values.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Frame:
    X: np.ndarray          # (n, p) float32, C-contiguous
    R: np.ndarray          # (p, p) float64 true correlation matrix
    v_min: np.ndarray      # (p,) unit eigenvector of R's smallest eigenvalue
    outlier: np.ndarray    # (n,) bool, True on contaminated rows
    h: int                 # floor(alpha * n)
    recipe: str


def random_correlation(p: int, cond: float, rng: np.random.Generator):
    """Random correlation matrix with eigenvalues log-spaced in [1, cond],
    rescaled to sum p (so the diagonal can be one).  Returns (R, v_min)."""
    from scipy.stats import random_correlation as _rc

    if p == 1:
        return np.ones((1, 1)), np.ones(1)
    ev = np.logspace(0.0, np.log10(cond), p)
    ev = ev * (p / ev.sum())
    R = _rc.rvs(ev, random_state=rng)
    R = 0.5 * (R + R.T)
    np.fill_diagonal(R, 1.0)
    w, V = np.linalg.eigh(R)
    v = V[:, 0]
    return R, v / np.linalg.norm(v)


def contaminated_gaussian(n: int, p: int, *, eps: float, kind: str,
                          shift: float, seed: int, cond: float = 100.0,
                          cluster_sd: float = 0.1, alpha: float = 0.75,
                          kind2: str | None = None, shift2: float = 0.0,
                          eps2: float = 0.0) -> Frame:
    """n rows of N(0, R) with floor(eps*n) rows replaced by outliers.

    kind = "point"   : every outlier equals shift * v_min (bitwise identical rows)
           "cluster" : outliers ~ N(shift * v_min, cluster_sd^2 I)
           "shift"   : outliers ~ N(shift * v_min, R)
    An optional second contamination (kind2, shift2, eps2) is placed on other
    rows.  Outlier positions are a seeded random subset.
    """
    rng = np.random.default_rng(seed)
    R, v = random_correlation(p, cond, rng)
    C = np.linalg.cholesky(R)
    X = rng.standard_normal((n, p)) @ C.T
    out = np.zeros(n, dtype=bool)
    n1 = int(np.floor(eps * n))
    n2 = int(np.floor(eps2 * n)) if kind2 else 0
    pos = rng.choice(n, n1 + n2, replace=False)

    def fill(idx, kd, sh):
        if kd == "point":
            X[idx] = sh * v
        elif kd == "cluster":
            X[idx] = sh * v + cluster_sd * rng.standard_normal((len(idx), p))
        elif kd == "shift":
            X[idx] = sh * v + rng.standard_normal((len(idx), p)) @ C.T
        else:
            raise ValueError(kd)

    if n1:
        fill(pos[:n1], kind, shift)
    if n2:
        fill(pos[n1:], kind2, shift2)
    out[pos] = True
    Xf = np.ascontiguousarray(X, dtype=np.float32)
    h = int(np.floor(alpha * n))
    recipe = (f"N(0,R) n={n} p={p} cond(R)={cond:g} seed={seed}; "
              f"{eps:.0%} {kind} outliers at {shift:g}*v_min"
              + (f" sd={cluster_sd:g}" if kind == "cluster" else "")
              + (f"; {eps2:.0%} {kind2} at {shift2:g}*v_min" if n2 else "")
              + f"; h=floor({alpha:g} n)")
    return Frame(Xf, R, v, out, h, recipe)


def small_fp64_case(seed: int = 0) -> Frame:
    """n=10,000, p=5, h=floor(0.75n); 10% point outliers at distance 10 along
    v_min; cond(R)=100."""
    return contaminated_gaussian(10_000, 5, eps=0.10, kind="point", shift=10.0,
                                 seed=seed)


def main_case(seed: int = 0, n: int = 1_000_000, p: int = 20) -> Frame:
    """n=1,000,000, p=20, h=floor(0.75n); 20% cluster outliers
    N(5 v_min, 0.1^2 I); cond(R)=100."""
    return contaminated_gaussian(n, p, eps=0.20, kind="cluster", shift=5.0,
                                 seed=seed, cluster_sd=0.1)


def large_case(seed: int = 0, n: int = 10_000_000, p: int = 40) -> Frame:
    """n=10,000,000, p=40; 7.5% point outliers at 8 v_min and 7.5% cluster
    N(5 v_min, 0.1^2 I)."""
    return contaminated_gaussian(n, p, eps=0.075, kind="point", shift=8.0,
                                 seed=seed, kind2="cluster", shift2=5.0,
                                 eps2=0.075)


def batched_frame(f: int) -> Frame:
    """Frame f of the many-frames workload: n ~ U[2000, 50000],
    p ~ U{8,16,24,32,40}, 0-25% point outliers at 10 v_min, seed f."""
    rng = np.random.default_rng(10_000 + f)
    n = int(rng.integers(2000, 50001))
    p = int(rng.choice([8, 16, 24, 32, 40]))
    eps = float(rng.uniform(0.0, 0.25))
    return contaminated_gaussian(n, p, eps=eps, kind="point", shift=10.0,
                                 seed=f)


def a09_case(n: int, p: int, eps: float, kind: str, gamma: float,
             seed: int, cluster_sd: float = 0.05, alpha: float = 0.5) -> Frame:
    """The paper's A09 design (Section 5): Sigma_jk = (-0.9)^|j-k|, outliers
    at gamma * v with v the last eigenvector scaled so v' Sigma^-1 v = p."""
    rng = np.random.default_rng(seed)
    j = np.arange(p)
    S = (-0.9) ** np.abs(j[:, None] - j[None, :])
    w, V = np.linalg.eigh(S)
    v = V[:, 0]
    v = v * np.sqrt(p / (v @ np.linalg.solve(S, v)))
    C = np.linalg.cholesky(S)
    X = rng.standard_normal((n, p)) @ C.T
    n1 = int(np.floor(eps * n))
    pos = rng.choice(n, n1, replace=False)
    if kind == "point":
        X[pos] = gamma * v
    elif kind == "cluster":
        X[pos] = gamma * v + cluster_sd * rng.standard_normal((n1, p))
    elif kind == "shift":
        X[pos] = gamma * v + rng.standard_normal((n1, p)) @ C.T
    out = np.zeros(n, dtype=bool)
    out[pos] = True
    # alpha = 0.5 is the most robust choice, h = [(n+p+1)/2] (Section 2.1).
    h = (n + p + 1) // 2 if alpha == 0.5 else int(np.floor(alpha * n))
    return Frame(np.ascontiguousarray(X, dtype=np.float32), S,
                 v / np.linalg.norm(v), out, h,
                 f"A09 n={n} p={p} {eps:.0%} {kind} gamma={gamma:g}")
