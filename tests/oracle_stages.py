"""The four stages of a sharded fit computed by the oracle, with the
interface of the CUDA stage backend: lets the sharding logic (ranges,
all-gathers, moment sums) run on CPU processes and be compared with the
oracle's unsharded fit.  Test infrastructure only."""
import numpy as np

import oracle as O


class OracleStages:
    def __init__(self, X, h, *, omega=O.OMEGA, q=None, seed=0, kappa_max=O.KAPPA_MAX, cutoff_q=O.CUTOFF_Q,
                 max_steps=O.MAX_CSTEPS):
        self.X = np.asarray(X, dtype=np.float64)
        self.n, self.p = self.X.shape
        self.h = int(h)
        self.q = q if q is not None else O.block_count(self.n, self.p, omega)
        self.m = self.n // self.q
        self.seed, self.kappa_max, self.cutoff_q, self.max_steps = seed, kappa_max, cutoff_q, max_steps
        self.perm = np.arange(self.n) if self.q == 1 else O.partition_permutation(self.n, seed)
        self.h_b = self.h if self.q == 1 else (self.h * self.m) // self.n
        self.c_alpha = O.consistency_factor(self.h / self.n, self.p)
        self.cutoff_d2 = O.chi2_ppf(cutoff_q, self.p)

    def partition(self):
        return self.q, self.m

    def _z(self, uni):
        p = self.p
        return (self.X - uni[:p]) / uni[p:]

    def standardize(self, lo, hi):
        u = [O.univariate_mcd(self.X[:, j], self.cutoff_q) for j in range(lo, hi)]
        return 0, np.array([[x.mu for x in u], [np.sqrt(x.s2) for x in u]]).reshape(2, hi - lo)

    def fit_blocks(self, uni, lo, hi):
        p, m = self.p, self.m
        Z = self._z(uni)
        recs = np.zeros((hi - lo, 2 + p + p * p))
        for i, l in enumerate(range(lo, hi)):
            Zl = Z[self.perm[l * m:(l + 1) * m]]
            chains = [O.block_start_unit((Zl, k, self.h_b, self.kappa_max, self.max_steps))[2] for k in (0, 1)]
            c = O.choose_start(chains)
            recs[i, 0] = c
            if c >= 0:
                ch = chains[c]
                recs[i, 1] = np.linalg.slogdet(ch.Sigma)[1]
                recs[i, 2:2 + p] = ch.mu
                recs[i, 2 + p:] = ch.Sigma.ravel()
        return 0, recs

    def _raw(self, fits):
        p = self.p
        blk = [None if r[0] < 0 else (r[2:2 + p], self.c_alpha * r[2 + p:].reshape(p, p)) for r in fits]
        mu_raw, Sigma_raw, _, _ = O.aggregate(blk, self.h_b, self.c_alpha)
        return mu_raw, Sigma_raw

    def reweight_moments(self, uni, fits, lo, hi):
        """Count, sum and cross-products (about 0, Z units) of the rows of
        blocks [lo, hi) within the cutoff of the raw fit."""
        Z = self._z(uni)
        mu_raw, Sigma_raw = self._raw(fits)
        rows = self.perm[lo * self.m:hi * self.m]
        Zr = Z[rows]
        Zw = Zr[O.mahalanobis_d2(Zr, mu_raw, Sigma_raw) <= self.cutoff_d2]
        return 0, np.concatenate([[float(Zw.shape[0])], Zw.sum(axis=0), (Zw.T @ Zw).ravel()])

    def reweight_finish(self, uni, fits, moments, lo, hi):
        p = self.p
        mu_uni, s_uni = uni[:p], uni[p:]
        N, s, S = moments[0], moments[1:1 + p], moments[1 + p:].reshape(p, p)
        mu_z = s / N
        Sigma_z = O.reweight_factor(p, self.cutoff_q) * (S - N * np.outer(mu_z, mu_z)) / (N - 1)
        mu_raw, Sigma_raw = self._raw(fits)
        Z = self._z(uni)
        d2 = O.mahalanobis_d2(Z[lo:hi], mu_z, Sigma_z)
        flags = d2 > self.cutoff_d2
        D = np.outer(s_uni, s_uni)
        return 0, {"mu": mu_uni + s_uni * mu_z, "Sigma": Sigma_z * D, "mu_raw": mu_uni + s_uni * mu_raw,
                   "Sigma_raw": Sigma_raw * D, "n_reweight": int(round(N)), "n_flagged": int(flags.sum()),
                   "d2": d2, "flags": flags.astype(np.uint8), "rows": (lo, hi)}
