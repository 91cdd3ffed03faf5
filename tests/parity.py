"""Comparison helpers of the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (stated in the project's design notes):
  FP32 form: mu and Sigma within 1e-5 relative (max-abs over max-abs of the
             oracle), same final h-subsets and flags outside the tie bands.
  FP64 form: 1e-9 relative.
  Split-BF16 form: mu and Sigma within 1e-3 relative, the same subsets and
             flags outside the tie bands.
Tie bands: rows whose oracle distance lies within 1e-6 relative of the h-th
distance of their block (subsets) or of the cutoff (flags) are excluded.
"""
import numpy as np

import oracle as O

TOL = {"fp32": 1e-5, "fp64": 1e-9, "bf16": 1e-3}
TIE = 1e-6


def rel_mat(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_center(mu_a, mu_b, Sigma):
    scale = np.sqrt(np.max(np.diag(Sigma)))
    return float(np.max(np.abs(np.asarray(mu_a) - np.asarray(mu_b))) / scale)


def subset_band(ref, rel=TIE):
    """Rows (original order) whose final-chain distance is within `rel` of
    the h_b-th distance of their block (needs ref.Zrows, set by compare_fit)."""
    band = np.zeros(ref.d2.size, dtype=bool)
    for b in ref.blocks:
        if b.chosen < 0:
            continue
        ch = b.chains[b.chosen]
        d2 = O.mahalanobis_d2(ref.Zrows(b.rows), ch.mu, ch.Sigma)
        t = np.sort(d2)[ref.h_b - 1]
        band[b.rows] = np.abs(d2 - t) <= rel * t
    return band


def flag_band(ref, rel=TIE):
    return np.abs(ref.d2 - ref.cutoff_d2) <= rel * ref.cutoff_d2


def to_np(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a
    return a.detach().cpu().numpy()


def compare_fit(got, ref, X, form, check_subsets=True):
    """Assert parity of a GPU fit with the oracle fit `ref` of the rows X."""
    tol = TOL[form]
    Z = (np.asarray(X, np.float64) - ref.mu_uni) / ref.s_uni
    ref.Zrows = lambda rows: Z[rows]
    report = {
        "mu": rel_center(got["mu"], ref.mu, ref.Sigma),
        "Sigma": rel_mat(got["Sigma"], ref.Sigma),
        "mu_raw": rel_center(got["mu_raw"], ref.mu_raw, ref.Sigma_raw),
        "Sigma_raw": rel_mat(got["Sigma_raw"], ref.Sigma_raw),
    }
    fl = to_np(got["flags"]).astype(bool)
    fb = flag_band(ref)
    report["flag_mismatch"] = int(np.sum((fl != ref.flags) & ~fb))
    report["flag_band"] = int(fb.sum())
    if check_subsets and got.get("subset") is not None:
        sb = to_np(got["subset"])
        band = subset_band(ref)
        report["subset_mismatch"] = int(np.sum(((sb & 1).astype(bool) != ref.subset_mask()) & ~band))
        wb = np.zeros_like(band)
        used = ref.perm[: ref.q * ref.m]
        wb[used] = np.abs(ref.d2_raw[used] - ref.cutoff_d2) <= TIE * ref.cutoff_d2
        report["W_mismatch"] = int(np.sum((((sb >> 1) & 1).astype(bool) != ref.W) & ~wb))
    ok = (report["mu"] <= tol and report["Sigma"] <= tol and report["mu_raw"] <= tol
          and report["Sigma_raw"] <= tol and report["flag_mismatch"] == 0
          and report.get("subset_mismatch", 0) == 0 and report.get("W_mismatch", 0) == 0)
    return ok, report
