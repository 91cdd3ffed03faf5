"""GB300 (sm_103a) RT-DetMCD engine: Python binding of the C ABI in
include/rtdetmcd.h.

The functions below only marshal arguments (tensor pointers, strides, the
current CUDA stream, a workspace tensor) and call the CUDA library; every
step of the method runs in its kernels.  Importing this module fails loudly
if the library has not been built (`paper_1910_05615_gb300.build.build()`).

Method: De Ketelaere, Hubert, Raymaekers, Rousseeuw, Vranckx, "Real-time
outlier detection for large datasets by RT-DetMCD" (arXiv 1910.05615).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

__all__ = [
    "RTD_FP32", "RTD_FP64", "RTD_BF16", "RtdError", "library_path", "rtdetmcd_fit", "rtdetmcd_distances",
    "rtdetmcd_flag", "rtdetmcd_distances_noalloc", "rtdetmcd_chi2_quantile", "rtdetmcd_status_string", "rtdetmcd_workspace_size",
    "rtdetmcd_diag_size", "rtdetmcd_distances_workspace_size", "parse_diag", "rtdetmcd_grad",
    "rtdetmcd_grad_workspace_size", "rtdetmcd_objective", "rtdetmcd_fit_batch",
    "rtdetmcd_fit_batch_workspace_size", "rtdetmcd_vjp", "rtdetmcd_fit_outputs", "rtdetmcd_score",
    "rtdetmcd_score_workspace_size", "rtdetmcd_autotune", "rtdetmcd_tuned", "rtdetmcd_partition",
    "rtdetmcd_standardize", "rtdetmcd_fit_blocks", "rtdetmcd_reweight_moments", "rtdetmcd_reweight_finish",
    "rtdetmcd_prepared_size", "rtdetmcd_score_prepare", "rtdetmcd_score_prepared",
]

RTD_FP64 = 0
RTD_FP32 = 1
RTD_BF16 = 2     # FP32 form with the Grams on the tensor cores (25 <= p <= 48)
RTD_MAX_P = 64

STATUS = {0: "RTD_OK", 1: "RTD_EINVAL", 2: "RTD_ENONFINITE", 3: "RTD_EILLCOND", 4: "RTD_EDEGENERATE",
          5: "RTD_EWORKSPACE", 6: "RTD_ECUDA", 7: "RTD_EINTERNAL"}


class RtdError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("omega", ctypes.c_int32),
                ("q_override", ctypes.c_int32), ("max_csteps", ctypes.c_int32),
                ("cutoff_q", ctypes.c_double), ("kappa_max", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("reweight_consistency", ctypes.c_int32),
                ("select_path", ctypes.c_int32), ("subset_out", ctypes.c_void_p),
                ("diag_out", ctypes.c_void_p), ("profile", ctypes.c_void_p),
                ("init_mu", ctypes.c_void_p), ("init_sigma", ctypes.c_void_p),
                ("dist_path", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("win_rows", ctypes.c_int32), ("sel_ctas", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ms_best", ctypes.c_double), ("ms_default", ctypes.c_double)]


STAGES = ["partition", "univariate", "starts", "refine", "cstep_prep", "cstep_dist",
          "cstep_select", "cstep_update", "aggregate", "reweight", "final", "sort"]


class _Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("bytes", ctypes.c_double * len(STAGES)),
                ("launches", ctypes.c_int64 * len(STAGES)), ("csteps", ctypes.c_int32),
                ("win_steps", ctypes.c_int32), ("win_miss", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sel_cand", ctypes.c_int64), ("sel_band", ctypes.c_int64),
                ("flops", ctypes.c_double * len(STAGES))]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("warnings", ctypes.c_int32),
                ("p", ctypes.c_int32), ("q", ctypes.c_int32),
                ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("h", ctypes.c_int64), ("h_b", ctypes.c_int64),
                ("mu", ctypes.c_double * RTD_MAX_P), ("sigma", ctypes.c_double * (RTD_MAX_P * RTD_MAX_P)),
                ("mu_raw", ctypes.c_double * RTD_MAX_P),
                ("sigma_raw", ctypes.c_double * (RTD_MAX_P * RTD_MAX_P)),
                ("logdet", ctypes.c_double), ("logdet_raw", ctypes.c_double),
                ("cutoff_d2", ctypes.c_double), ("n_flagged", ctypes.c_int64),
                ("n_reweight", ctypes.c_int64), ("csteps_max", ctypes.c_int32),
                ("chains_ok", ctypes.c_int32), ("c_rew", ctypes.c_double)]


def library_path() -> str:
    return _build_mod.LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"RT-DetMCD CUDA library not built ({path}); run "
                          "paper_1910_05615_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
    lib.rtdetmcd_default_options.argtypes = [ctypes.POINTER(_Options)]
    lib.rtdetmcd_workspace_size.argtypes = [i64, i32, ctypes.POINTER(_Options)]
    lib.rtdetmcd_workspace_size.restype = sz
    lib.rtdetmcd_diag_size.argtypes = [i32, i32]
    lib.rtdetmcd_diag_size.restype = sz
    lib.rtdetmcd_fit.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), vp, sz, vp,
                                 ctypes.POINTER(_Result), vp, vp]
    lib.rtdetmcd_fit.restype = i32
    lib.rtdetmcd_distances_workspace_size.argtypes = [i64, i32]
    lib.rtdetmcd_distances_workspace_size.restype = sz
    lib.rtdetmcd_distances.argtypes = [vp, i64, i32, i64, vp, vp, i32, vp, vp, sz, vp]
    lib.rtdetmcd_distances.restype = i32
    lib.rtdetmcd_score_workspace_size.argtypes = [i64, i32]
    lib.rtdetmcd_score_workspace_size.restype = sz
    lib.rtdetmcd_score.argtypes = [vp, i64, i32, i64, vp, vp, dbl, i32, vp, vp, ctypes.POINTER(i64), vp, sz, vp]
    lib.rtdetmcd_score.restype = i32
    lib.rtdetmcd_prepared_size.argtypes = []
    lib.rtdetmcd_prepared_size.restype = sz
    lib.rtdetmcd_score_prepare.argtypes = [vp, vp, i32, dbl, vp, vp]
    lib.rtdetmcd_score_prepare.restype = i32
    lib.rtdetmcd_score_prepared.argtypes = [vp, i64, i32, i64, vp, i32, vp, vp, vp, vp]
    lib.rtdetmcd_score_prepared.restype = i32
    lib.rtdetmcd_distances_noalloc.argtypes = [vp, i64, i32, i64, vp, vp, i32, vp, vp]
    lib.rtdetmcd_distances_noalloc.restype = i32
    P64, P32 = ctypes.POINTER(i64), ctypes.POINTER(i32)
    lib.rtdetmcd_partition.argtypes = [i64, i32, i64, ctypes.POINTER(_Options), ctypes.POINTER(i32),
                                       ctypes.POINTER(i64)]
    lib.rtdetmcd_partition.restype = i32
    lib.rtdetmcd_standardize.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), i32, i32, vp, sz, vp,
                                         vp]
    lib.rtdetmcd_standardize.restype = i32
    lib.rtdetmcd_fit_blocks.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), vp, i32, i32, vp, sz,
                                        vp, vp]
    lib.rtdetmcd_fit_blocks.restype = i32
    lib.rtdetmcd_reweight_moments.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), vp, vp, i32, i32,
                                              vp, sz, vp, vp]
    lib.rtdetmcd_reweight_moments.restype = i32
    lib.rtdetmcd_reweight_finish.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), vp, vp, vp, i64,
                                             i64, vp, sz, vp, ctypes.POINTER(_Result), vp, vp]
    lib.rtdetmcd_reweight_finish.restype = i32
    lib.rtdetmcd_fit_batch_workspace_size.argtypes = [i32, P64, P32, vp, i32]
    lib.rtdetmcd_fit_batch_workspace_size.restype = sz
    lib.rtdetmcd_fit_batch.argtypes = [i32, ctypes.POINTER(vp), P64, P32, P64, P64, vp, vp, sz, vp, i32,
                                       vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.rtdetmcd_fit_batch.restype = i32
    lib.rtdetmcd_grad_workspace_size.argtypes = [i64, i32]
    lib.rtdetmcd_grad_workspace_size.restype = sz
    lib.rtdetmcd_grad.argtypes = [vp, i64, i32, i64, vp, i32, vp, vp, dbl, dbl, dbl, ctypes.POINTER(dbl), vp,
                                  vp, sz, vp]
    lib.rtdetmcd_grad.restype = i32
    lib.rtdetmcd_vjp.argtypes = [vp, i64, i32, i64, vp, i32, vp, vp, dbl, vp, vp, dbl, vp, vp, vp, sz, vp]
    lib.rtdetmcd_vjp.restype = i32
    lib.rtdetmcd_flag.argtypes = [vp, i64, dbl, vp, ctypes.POINTER(i64), vp, sz, vp]
    lib.rtdetmcd_flag.restype = i32
    lib.rtdetmcd_autotune.argtypes = [vp, i64, i32, i64, i64, ctypes.POINTER(_Options), vp, sz, vp,
                                      ctypes.POINTER(_Tuning)]
    lib.rtdetmcd_autotune.restype = i32
    lib.rtdetmcd_tuned.argtypes = [i64, i32, ctypes.POINTER(_Options), ctypes.POINTER(_Tuning)]
    lib.rtdetmcd_tuned.restype = i32
    lib.rtdetmcd_chi2_quantile.argtypes = [i32, dbl]
    lib.rtdetmcd_chi2_quantile.restype = dbl
    lib.rtdetmcd_status_string.argtypes = [i32]
    lib.rtdetmcd_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


# ------------------------------------------------------------ marshalling
def _torch():
    import torch
    return torch


def _rows(X):
    """(pointer, n, p, ld, device_or_None, keepalive) of a float32 row-major
    array: a torch tensor (cuda or cpu) or a numpy array."""
    torch = _torch()
    if isinstance(X, torch.Tensor):
        if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
            raise ValueError("X must be a 2-D float32 tensor with unit column stride")
        dev = X.device if X.is_cuda else None
        return X.data_ptr(), X.shape[0], X.shape[1], X.stride(0), dev, X
    A = np.asarray(X)
    if A.dtype != np.float32 or A.ndim != 2 or A.strides[1] != 4:
        A = np.ascontiguousarray(A, dtype=np.float32)
    return A.ctypes.data, A.shape[0], A.shape[1], A.strides[0] // 4, None, A


def _stream_ptr(device, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if device is None:
        return ctypes.c_void_p(0)
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _workspace(nbytes, device):
    torch = _torch()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


def _out(n, dtype, device):
    if device is None:
        return np.empty(n, dtype=dtype)
    torch = _torch()
    tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.float64: torch.float64}[dtype]
    return torch.empty(n, dtype=tdt, device=device)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def rtdetmcd_workspace_size(n, p, precision=RTD_FP32, omega=4096, q=0):
    lib = _load()
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision, o.omega, o.q_override = precision, omega, q
    return lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o))


def rtdetmcd_diag_size(p, q):
    return _load().rtdetmcd_diag_size(p, q)


def rtdetmcd_distances_workspace_size(n, p):
    return _load().rtdetmcd_distances_workspace_size(n, p)


def rtdetmcd_chi2_quantile(p, q=0.975):
    return _load().rtdetmcd_chi2_quantile(p, q)


def rtdetmcd_status_string(code):
    return _load().rtdetmcd_status_string(code).decode()


def rtdetmcd_fit(X, h, *, precision=RTD_FP32, omega=4096, q=0, seed=0, max_csteps=100,
                 cutoff_q=0.975, kappa_max=1000.0, reweight_consistency=1, select_path=0, dist_path=0,
                 graph=False, init=None, d2=True, flags=True, subset=False, diag=False, profile=False,
                 stream=None, workspace=None, d2_out=None, flags_out=None, check=True):
    """RT-DetMCD fit of the rows of X (float32, row-major) with coverage h.

    X on a CUDA device: outputs are CUDA tensors on the same device.  X in
    host memory (numpy array or CPU tensor, pinned or not): the library
    copies it in and returns host (numpy) outputs.  Returns a dict with the
    reweighted and raw fits (X units, float64 numpy), the flags and squared
    distances, and optional per-row subset bits and diagnostics.
    """
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision, o.omega, o.q_override, o.seed = precision, omega, q, seed
    o.max_csteps, o.cutoff_q, o.kappa_max = max_csteps, cutoff_q, kappa_max
    o.reweight_consistency = reweight_consistency
    o.select_path = select_path
    o.dist_path = dist_path
    o.graph = 1 if graph else 0
    if init is not None:   # warm start: (mu, Sigma) of an earlier fit, X units
        init_mu = np.ascontiguousarray(init[0], dtype=np.float64).reshape(-1)
        init_sigma = np.ascontiguousarray(init[1], dtype=np.float64).reshape(-1)
        if init_mu.size != p or init_sigma.size != p * p:
            raise ValueError("init must be (mu of length p, Sigma of shape p x p)")
        o.init_mu, o.init_sigma = init_mu.ctypes.data, init_sigma.ctypes.data
    ws_need = lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o))
    if ws_need == 0:
        raise RtdError(1, "invalid n, p or options")
    ws = workspace if workspace is not None else _workspace(ws_need, dev)
    if d2_out is None:
        d2_out = _out(n, np.float32, dev) if d2 else None
    fl_out = flags_out
    if fl_out is None:
        fl_out = _out(n, np.uint8, dev) if flags else None
    sub_out = _out(n, np.uint8, dev) if subset else None
    o.subset_out = _ptr(sub_out)
    qq = q if q else max(min(n // (p * omega), 1024), 1)
    dg = _out(lib.rtdetmcd_diag_size(p, qq) // 8, np.float64, dev) if diag else None
    o.diag_out = _ptr(dg)
    prof = _Profile() if profile else None
    o.profile = ctypes.cast(ctypes.pointer(prof), ctypes.c_void_p) if profile else None
    res = _Result()
    st = lib.rtdetmcd_fit(ptr, n, p, ld, h, ctypes.byref(o), ws.data_ptr(), ws.numel(),
                          _stream_ptr(dev, stream), ctypes.byref(res), _ptr(d2_out), _ptr(fl_out))
    del keep
    if st != 0 and check:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    pp = p
    out = {
        "status": st, "warnings": res.warnings, "n": res.n, "p": res.p, "q": res.q, "m": res.m,
        "h": res.h, "h_b": res.h_b,
        "mu": np.array(res.mu[:pp]), "Sigma": np.array(res.sigma[:pp * pp]).reshape(pp, pp),
        "mu_raw": np.array(res.mu_raw[:pp]),
        "Sigma_raw": np.array(res.sigma_raw[:pp * pp]).reshape(pp, pp),
        "logdet": res.logdet, "logdet_raw": res.logdet_raw, "cutoff_d2": res.cutoff_d2,
        "n_flagged": res.n_flagged, "n_reweight": res.n_reweight, "csteps_max": res.csteps_max,
        "chains_ok": res.chains_ok, "c_rew": res.c_rew, "d2": d2_out, "flags": fl_out, "subset": sub_out,
    }
    if diag:
        a = dg.cpu().numpy() if not isinstance(dg, np.ndarray) else dg
        out["diag"] = parse_diag(a, pp, res.q)
    if profile:
        out["profile"] = {"csteps": prof.csteps, "win_steps": prof.win_steps, "win_miss": prof.win_miss,
                          "sel_cand": prof.sel_cand, "sel_band": prof.sel_band, "stages": {
            name: {"ms": prof.ms[i], "bytes": prof.bytes[i], "launches": prof.launches[i], "flops": prof.flops[i]}
            for i, name in enumerate(STAGES)}}
    return out


# ------------------------------------------------- the fit in stages
def _stage_options(lib, precision=RTD_FP32, omega=4096, q=0, seed=0, max_csteps=100, cutoff_q=0.975,
                   kappa_max=1000.0, reweight_consistency=1, select_path=0, dist_path=0):
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision, o.omega, o.q_override, o.seed = precision, omega, q, seed
    o.max_csteps, o.cutoff_q, o.kappa_max = max_csteps, cutoff_q, kappa_max
    o.reweight_consistency, o.select_path, o.dist_path = reweight_consistency, select_path, dist_path
    o.graph = 0
    return o


def _f64(a, size, name):
    """(pointer, keepalive) of a float64 array of `size` values: a numpy
    array or a contiguous torch tensor (host or device)."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != size:
            raise ValueError(f"{name} must be a contiguous float64 tensor of {size} values")
        return a.data_ptr(), a
    A = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if A.size != size:
        raise ValueError(f"{name} must hold {size} values")
    return A.ctypes.data, A


def _stage_ws(lib, n, p, o, dev, workspace):
    need = lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o))
    if need == 0:
        raise RtdError(1, "invalid n, p or options")
    return workspace if workspace is not None else _workspace(need, dev)


def _status(lib, st, check):
    if st != 0 and check:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())


def rtdetmcd_partition(n, p, h, **options):
    """(q, m): block count and rows per block of the partition (Section 4)."""
    lib = _load()
    o = _stage_options(lib, **options)
    q, m = ctypes.c_int32(0), ctypes.c_int64(0)
    st = lib.rtdetmcd_partition(n, p, h, ctypes.byref(o), ctypes.byref(q), ctypes.byref(m))
    _status(lib, st, True)
    return q.value, m.value


def rtdetmcd_standardize(X, h, col_lo, col_hi, *, stream=None, workspace=None, check=True, **options):
    """Univariate MCD of columns [col_lo, col_hi): float64 (2, k) array of
    locations and scales (host numpy).  Returns (status, array)."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    o = _stage_options(lib, **options)
    ws = _stage_ws(lib, n, p, o, dev, workspace)
    k = max(col_hi - col_lo, 0)
    out = np.zeros((2, k), dtype=np.float64)
    st = lib.rtdetmcd_standardize(ptr, n, p, ld, h, ctypes.byref(o), col_lo, col_hi, ws.data_ptr(), ws.numel(),
                                  _stream_ptr(dev, stream), out.ctypes.data)
    del keep
    _status(lib, st, check)
    return st, out


def rtdetmcd_fit_blocks(X, h, uni, blk_lo, blk_hi, *, stream=None, workspace=None, check=True, **options):
    """Steps 2-4 of blocks [blk_lo, blk_hi) given uni = (mu_uni, s_uni):
    float64 (blk_hi - blk_lo, 2 + p + p^2) block-fit records (host numpy).
    Returns (status, records)."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    o = _stage_options(lib, **options)
    ws = _stage_ws(lib, n, p, o, dev, workspace)
    up, ukeep = _f64(uni, 2 * p, "uni")
    k = max(blk_hi - blk_lo, 0)
    out = np.zeros((k, 2 + p + p * p), dtype=np.float64)
    st = lib.rtdetmcd_fit_blocks(ptr, n, p, ld, h, ctypes.byref(o), up, blk_lo, blk_hi, ws.data_ptr(), ws.numel(),
                                 _stream_ptr(dev, stream), out.ctypes.data)
    del keep, ukeep
    _status(lib, st, check)
    return st, out


def rtdetmcd_reweight_moments(X, h, uni, fits, blk_lo, blk_hi, *, stream=None, workspace=None, check=True,
                              **options):
    """Steps 5-7 from all q block-fit records, then the reweighting moments
    (count, sum, centred cross-products) of the rows of blocks
    [blk_lo, blk_hi): float64 (1 + p + p^2,) host array.  Returns (status,
    moments)."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    o = _stage_options(lib, **options)
    q, _ = rtdetmcd_partition(n, p, h, **options)
    ws = _stage_ws(lib, n, p, o, dev, workspace)
    up, ukeep = _f64(uni, 2 * p, "uni")
    fp, fkeep = _f64(fits, q * (2 + p + p * p), "fits")
    out = np.zeros(1 + p + p * p, dtype=np.float64)
    st = lib.rtdetmcd_reweight_moments(ptr, n, p, ld, h, ctypes.byref(o), up, fp, blk_lo, blk_hi, ws.data_ptr(),
                                       ws.numel(), _stream_ptr(dev, stream), out.ctypes.data)
    del keep, ukeep, fkeep
    _status(lib, st, check)
    return st, out


def rtdetmcd_reweight_finish(X, h, uni, fits, moments, row_lo, row_hi, *, d2=True, flags=True, stream=None,
                             workspace=None, check=True, **options):
    """Step 9 from the summed moments, then step 10 for rows [row_lo, row_hi).
    Returns (status, dict) with the reweighted and raw fits (X units) and the
    rows' squared distances and flags (on X's device, or numpy for host X);
    n_flagged counts those rows."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    o = _stage_options(lib, **options)
    q, _ = rtdetmcd_partition(n, p, h, **options)
    ws = _stage_ws(lib, n, p, o, dev, workspace)
    up, ukeep = _f64(uni, 2 * p, "uni")
    fp, fkeep = _f64(fits, q * (2 + p + p * p), "fits")
    mp_, mkeep = _f64(moments, 1 + p + p * p, "moments")
    k = max(row_hi - row_lo, 0)
    d2_out = _out(k, np.float32, dev) if d2 else None
    fl_out = _out(k, np.uint8, dev) if flags else None
    res = _Result()
    st = lib.rtdetmcd_reweight_finish(ptr, n, p, ld, h, ctypes.byref(o), up, fp, mp_, row_lo, row_hi, ws.data_ptr(),
                                      ws.numel(), _stream_ptr(dev, stream), ctypes.byref(res), _ptr(d2_out),
                                      _ptr(fl_out))
    del keep, ukeep, fkeep, mkeep
    _status(lib, st, check)
    return st, {
        "status": st, "warnings": res.warnings, "n": res.n, "p": res.p, "q": res.q, "m": res.m, "h": res.h,
        "h_b": res.h_b, "mu": np.array(res.mu[:p]), "Sigma": np.array(res.sigma[:p * p]).reshape(p, p),
        "mu_raw": np.array(res.mu_raw[:p]), "Sigma_raw": np.array(res.sigma_raw[:p * p]).reshape(p, p),
        "logdet": res.logdet, "logdet_raw": res.logdet_raw, "cutoff_d2": res.cutoff_d2,
        "n_flagged": res.n_flagged, "n_reweight": res.n_reweight, "c_rew": res.c_rew,
        "rows": (row_lo, row_hi), "d2": d2_out, "flags": fl_out,
    }


def _tuning_dict(t):
    return {"win_rows": t.win_rows, "sel_ctas": t.sel_ctas, "candidates": t.candidates, "ms_best": t.ms_best,
            "ms_default": t.ms_default}


def rtdetmcd_autotune(X, h, *, precision=RTD_FP32, graph=True, dist_path=0, select_path=0, stream=None,
                      workspace=None, **opts):
    """Time the candidate launch shapes of the C-step distance pass and the
    window selection on fits of the rows X (a CUDA tensor) and keep the
    fastest for later fits of this class; returns the choice."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    if dev is None:
        raise ValueError("rtdetmcd_autotune needs X on a CUDA device")
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision, o.graph, o.dist_path, o.select_path = precision, 1 if graph else 0, dist_path, select_path
    for k, v in opts.items():
        setattr(o, k, v)
    ws = workspace if workspace is not None else _workspace(lib.rtdetmcd_workspace_size(n, p, ctypes.byref(o)), dev)
    t = _Tuning()
    st = lib.rtdetmcd_autotune(ptr, n, p, ld, h, ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream_ptr(dev, stream),
                               ctypes.byref(t))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return _tuning_dict(t)


def rtdetmcd_tuned(n, p, *, precision=RTD_FP32, dist_path=0, select_path=0):
    """The tuned launch shape kept for fits of this size, or None."""
    lib = _load()
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision, o.dist_path, o.select_path = precision, dist_path, select_path
    t = _Tuning()
    return _tuning_dict(t) if lib.rtdetmcd_tuned(n, p, ctypes.byref(o), ctypes.byref(t)) else None


def rtdetmcd_fit_batch_workspace_size(frames, nstreams=8, precision=RTD_FP32):
    """Workspace bytes of rtdetmcd_fit_batch for these frames (2-D arrays or
    tensors, only their shapes are used)."""
    lib = _load()
    F = len(frames)
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision = precision
    n = (ctypes.c_int64 * F)(*[int(X.shape[0]) for X in frames])
    p = (ctypes.c_int32 * F)(*[int(X.shape[1]) for X in frames])
    return lib.rtdetmcd_fit_batch_workspace_size(F, n, p, ctypes.byref(o), nstreams)


def rtdetmcd_fit_batch(frames, hs, *, precision=RTD_FP32, nstreams=8, d2=True, flags=True, stream=None,
                       workspace=None, check=True, **opts):
    """Independent fits of many frames of uneven n and p (each frame a 2-D
    float32 array or tensor, all on the same CUDA device or all in host
    memory), run concurrently on `nstreams` streams.  Returns a list of
    per-frame dicts (reweighted and raw fits, counts, status, d2 and flags)."""
    lib = _load()
    F = len(frames)
    if F < 1 or len(hs) != F:
        raise ValueError("need one h per frame")
    rows = [_rows(Xf) for Xf in frames]
    devs = {r[4] for r in rows}
    if len(devs) != 1:
        raise ValueError("frames must all be on one CUDA device or all in host memory")
    dev = rows[0][4]
    o = _Options()
    lib.rtdetmcd_default_options(ctypes.byref(o))
    o.precision = precision
    for k, v in opts.items():
        setattr(o, k, v)
    Xp = (ctypes.c_void_p * F)(*[r[0] for r in rows])
    n = (ctypes.c_int64 * F)(*[r[1] for r in rows])
    p = (ctypes.c_int32 * F)(*[r[2] for r in rows])
    ld = (ctypes.c_int64 * F)(*[r[3] for r in rows])
    h = (ctypes.c_int64 * F)(*[int(x) for x in hs])
    need = lib.rtdetmcd_fit_batch_workspace_size(F, n, p, ctypes.byref(o), nstreams)
    if need == 0:
        raise RtdError(1, "invalid frame shape, options or stream count")
    ws = workspace if workspace is not None else _workspace(need, dev)
    d2s = [_out(r[1], np.float32, dev) for r in rows] if d2 else None
    fls = [_out(r[1], np.uint8, dev) for r in rows] if flags else None
    d2p = (ctypes.c_void_p * F)(*[_ptr(a) for a in d2s]) if d2 else None
    flp = (ctypes.c_void_p * F)(*[_ptr(a) for a in fls]) if flags else None
    res = (_Result * F)()
    st = lib.rtdetmcd_fit_batch(F, Xp, n, p, ld, h, ctypes.byref(o), ws.data_ptr(), ws.numel(),
                                _stream_ptr(dev, stream), nstreams, res, d2p, flp)
    del rows
    if st != 0 and check:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    out = []
    for f in range(F):
        r, pp = res[f], p[f]
        out.append({
            "status": r.status, "n": r.n, "p": r.p, "q": r.q, "h": r.h,
            "mu": np.array(r.mu[:pp]), "Sigma": np.array(r.sigma[:pp * pp]).reshape(pp, pp),
            "mu_raw": np.array(r.mu_raw[:pp]), "Sigma_raw": np.array(r.sigma_raw[:pp * pp]).reshape(pp, pp),
            "logdet": r.logdet, "cutoff_d2": r.cutoff_d2, "n_flagged": r.n_flagged, "n_reweight": r.n_reweight,
            "csteps_max": r.csteps_max, "c_rew": r.c_rew,
            "d2": d2s[f] if d2 else None, "flags": fls[f] if flags else None})
    return out


def parse_diag(a, p, q):
    """Unpack the diagnostics record documented at rtdetmcd_diag_size."""
    a = np.asarray(a, dtype=np.float64)
    rec = 3 * p * p + 2 * p + 6
    d = {"mu_uni": a[:p].copy(), "sigma_uni": a[p:2 * p].copy(), "chains": [], "blocks": []}
    for c in range(2 * q):
        r = a[2 * p + c * rec: 2 * p + (c + 1) * rec]
        t = r[3 * p * p + 2 * p:]
        d["chains"].append({
            "S_init": r[:p * p].reshape(p, p), "Sigma_start": r[p * p:2 * p * p].reshape(p, p),
            "mu_start": r[2 * p * p:2 * p * p + p], "Sigma": r[2 * p * p + p:3 * p * p + p].reshape(p, p),
            "mu": r[3 * p * p + p:3 * p * p + 2 * p], "logdet": t[0], "steps": int(t[1]),
            "status": int(t[2]), "full_recomputes": int(t[3]), "last_swaps": int(t[4]), "kappa1": t[5]})
    b = a[2 * p + 2 * q * rec:]
    for l in range(q):
        d["blocks"].append({"chosen": int(b[3 * l]), "kl": b[3 * l + 1], "kept": int(b[3 * l + 2])})
    return d


def rtdetmcd_distances(X, mu, Sigma, *, precision=RTD_FP32, stream=None, workspace=None):
    """Squared robust distances of the rows of X to the fit (mu, Sigma)."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    ws = workspace if workspace is not None else _workspace(lib.rtdetmcd_distances_workspace_size(n, p), dev)
    d2 = _out(n, np.float32, dev)
    st = lib.rtdetmcd_distances(ptr, n, p, ld, mu.ctypes.data, S.ctypes.data, precision, _ptr(d2),
                                ws.data_ptr(), ws.numel(), _stream_ptr(dev, stream))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return d2


def rtdetmcd_score_workspace_size(n, p):
    return _load().rtdetmcd_score_workspace_size(n, p)


def rtdetmcd_score(X, mu, Sigma, cutoff_d2=None, *, precision=RTD_FP32, d2=True, flags=True, stream=None,
                   workspace=None):
    """Distances, flags (d2 > cutoff_d2) and their count for the rows of X
    against the fit (mu, Sigma) in one streaming pass.  cutoff_d2 defaults to
    chi2_{p,0.975}.  Returns (d2 or None, flags or None, n_flagged)."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
    S = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(-1)
    if mu.size != p or S.size != p * p:
        raise ValueError("mu must have p entries and Sigma p x p")
    cut = rtdetmcd_chi2_quantile(p, 0.975) if cutoff_d2 is None else float(cutoff_d2)
    ws = workspace if workspace is not None else _workspace(lib.rtdetmcd_score_workspace_size(n, p), dev)
    d2o = _out(n, np.float32, dev) if d2 else None
    flo = _out(n, np.uint8, dev) if flags else None
    cnt = ctypes.c_int64(0)
    st = lib.rtdetmcd_score(ptr, n, p, ld, mu.ctypes.data, S.ctypes.data, cut, precision, _ptr(d2o), _ptr(flo),
                            ctypes.byref(cnt), ws.data_ptr(), ws.numel(), _stream_ptr(dev, stream))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return d2o, flo, cnt.value


def rtdetmcd_prepared_size():
    return _load().rtdetmcd_prepared_size()


def rtdetmcd_score_prepare(mu, Sigma, cutoff_d2=None, *, device=None, stream=None, out=None):
    """Factorise the fit (mu, Sigma; X units) once for scoring many batches
    (Section 6): returns the prepared fit, a uint8 CUDA tensor (or fills
    `out`).  Raises RtdError if Sigma is not positive definite."""
    torch = _torch()
    lib = _load()
    mu_c = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
    p = mu_c.size
    S_c = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(p, p)
    if cutoff_d2 is None:
        cutoff_d2 = rtdetmcd_chi2_quantile(p, 0.975)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    prep = out if out is not None else torch.empty(lib.rtdetmcd_prepared_size(), dtype=torch.uint8, device=dev)
    st = lib.rtdetmcd_score_prepare(mu_c.ctypes.data, S_c.ctypes.data, p, float(cutoff_d2), prep.data_ptr(),
                                    _stream_ptr(prep.device, stream))
    _status(lib, st, True)
    return prep


def rtdetmcd_score_prepared(X, prepared, *, precision=RTD_FP32, d2=True, flags=True, count=None, stream=None,
                            d2_out=None, flags_out=None):
    """Score the rows of X (a CUDA tensor) against a prepared fit with one
    kernel launch and no wait: returns (d2, flags) CUDA tensors (None where
    not asked for).  `count` (int64 CUDA tensor of one element, nullable)
    receives the number of flagged rows added to its value."""
    lib = _load()
    ptr, n, p, ld, dev, keep = _rows(X)
    if dev is None:
        raise ValueError("rtdetmcd_score_prepared needs X on a CUDA device")
    if d2_out is None and d2:
        d2_out = _out(n, np.float32, dev)
    if flags_out is None and flags:
        flags_out = _out(n, np.uint8, dev)
    if count is not None and (count.dtype != _torch().int64 or count.numel() != 1 or not count.is_cuda):
        raise ValueError("count must be a one-element int64 CUDA tensor")
    st = lib.rtdetmcd_score_prepared(ptr, n, p, ld, prepared.data_ptr(), precision, _ptr(d2_out), _ptr(flags_out),
                                     _ptr(count), _stream_ptr(dev, stream))
    del keep
    _status(lib, st, True)
    return d2_out, flags_out


def rtdetmcd_distances_noalloc(X, mu, Sigma, *, precision=RTD_FP32, out=None, stream=None):
    """Squared distances like rtdetmcd_distances, for callers that cannot
    allocate when they score: no workspace, the library uses a fixed device
    array instead.  X (and out, if given) must be CUDA tensors."""
    lib = _load()
    torch = _torch()
    ptr, n, p, ld, dev, keep = _rows(X)
    if dev is None:
        raise ValueError("rtdetmcd_distances_noalloc needs X on a CUDA device")
    if out is not None:
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        if out.device != dev or out.numel() < n:
            raise ValueError("out must be on X's device and hold at least n = %d values" % n)
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
    S = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(-1)
    if mu.size != p or S.size != p * p:
        raise ValueError("mu must have p entries and Sigma p x p")
    d2 = out if out is not None else _out(n, np.float32, dev)
    with torch.cuda.device(dev):
        st = lib.rtdetmcd_distances_noalloc(ptr, n, p, ld, mu.ctypes.data, S.ctypes.data, precision, _ptr(d2),
                                            _stream_ptr(dev, stream))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return d2


def rtdetmcd_grad_workspace_size(n, p):
    return _load().rtdetmcd_grad_workspace_size(n, p)


def rtdetmcd_grad(X, wset, mu, Sigma, c, *, wbit=1, w_logdet=1.0, w_rd=1.0, grad=True, stream=None,
                  workspace=None):
    """Value and gradient in X of w_logdet log det Sigma + w_rd sum_i RD_i with
    the reweighting set W (bit `wbit` of wset) held fixed (Section 4 steps
    8-10).  X and wset are CUDA tensors; mu, Sigma = c S_W the fit of W.
    Returns (value, grad) with grad an n x p CUDA tensor, or None."""
    lib = _load()
    torch = _torch()
    ptr, n, p, ld, dev, keep = _rows(X)
    if dev is None or not (isinstance(wset, torch.Tensor) and wset.is_cuda):
        raise ValueError("rtdetmcd_grad needs X and wset on a CUDA device")
    if wset.dtype != torch.uint8 or wset.numel() != n or not wset.is_contiguous():
        raise ValueError("wset must be a contiguous uint8 tensor of n bytes")
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    if mu.size != p or S.size != p * p:
        raise ValueError("mu must have p entries and Sigma p x p")
    ws = workspace if workspace is not None else _workspace(lib.rtdetmcd_grad_workspace_size(n, p), dev)
    g = torch.empty((n, p), dtype=torch.float32, device=dev) if grad else None
    val = ctypes.c_double(0.0)
    st = lib.rtdetmcd_grad(ptr, n, p, ld, wset.data_ptr(), wbit, mu.ctypes.data, S.ctypes.data, float(c),
                           float(w_logdet), float(w_rd), ctypes.byref(val), _ptr(g), ws.data_ptr(), ws.numel(),
                           _stream_ptr(dev, stream))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return val.value, g


def rtdetmcd_vjp(X, wset, mu, Sigma, c, *, gmu=None, gSigma=None, glogdet=0.0, gRD=None, wbit=1, stream=None,
                 workspace=None):
    """d/dX of gmu.mu + <gSigma, Sigma> + glogdet log det Sigma + gRD.RD for
    the reweighted fit (mu, Sigma = c S_W, RD over all rows) with the set W
    (bit `wbit` of wset) held fixed.  X, wset and gRD are CUDA tensors; gmu,
    gSigma host arrays or tensors (None = zero).  Returns the n x p gradient
    (CUDA float32)."""
    lib = _load()
    torch = _torch()
    ptr, n, p, ld, dev, keep = _rows(X)
    if dev is None or not (isinstance(wset, torch.Tensor) and wset.is_cuda):
        raise ValueError("rtdetmcd_vjp needs X and wset on a CUDA device")
    if wset.dtype != torch.uint8 or wset.numel() != n or not wset.is_contiguous():
        raise ValueError("wset must be a contiguous uint8 tensor of n bytes")
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
    S = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(-1)
    if mu.size != p or S.size != p * p:
        raise ValueError("mu must have p entries and Sigma p x p")

    def host(a, size):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size != size:
            raise ValueError("cotangent of the wrong size")
        return a

    gm, gs = host(gmu, p), host(gSigma, p * p)
    grd = None
    if gRD is not None:
        if not (isinstance(gRD, torch.Tensor) and gRD.is_cuda and gRD.device == dev) or gRD.numel() != n:
            raise ValueError("gRD must be a CUDA tensor of n values on X's device")
        grd = gRD.detach().to(torch.float32).contiguous()
    ws = workspace if workspace is not None else _workspace(lib.rtdetmcd_grad_workspace_size(n, p), dev)
    g = torch.empty((n, p), dtype=torch.float32, device=dev)
    st = lib.rtdetmcd_vjp(ptr, n, p, ld, wset.data_ptr(), wbit, mu.ctypes.data, S.ctypes.data, float(c),
                          gm.ctypes.data if gm is not None else None, gs.ctypes.data if gs is not None else None,
                          float(glogdet), _ptr(grd), g.data_ptr(), ws.data_ptr(), ws.numel(),
                          _stream_ptr(dev, stream))
    del keep
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return g


_outputs_fn = None


def rtdetmcd_fit_outputs(X, h, **fit_kwargs):
    """Differentiable outputs (mu, Sigma, logdet, RD) of the reweighted fit of
    the rows of X (a CUDA float32 tensor): mu (p) and Sigma (p x p) float64,
    logdet a 0-d float64, RD (n) float32, all on X's device.  The forward
    pass runs rtdetmcd_fit; the backward pass holds the fit's discrete
    choices (the h-subsets and the reweighting set W) fixed and applies
    rtdetmcd_vjp to the incoming cotangents of all four outputs."""
    global _outputs_fn
    torch = _torch()
    if _outputs_fn is None:
        class _Outputs(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Xt, hh, kw):
                fit = rtdetmcd_fit(Xt.detach(), hh, d2=True, flags=False, subset=True, **kw)
                ctx.save_for_backward(Xt, fit["subset"])
                ctx.fit = (fit["mu"], fit["Sigma"], fit["c_rew"])
                dev = Xt.device
                mu = torch.tensor(fit["mu"], dtype=torch.float64, device=dev)
                S = torch.tensor(fit["Sigma"], dtype=torch.float64, device=dev)
                ld = torch.tensor(fit["logdet"], dtype=torch.float64, device=dev)
                return mu, S, ld, fit["d2"].clamp_min(0).sqrt()

            @staticmethod
            def backward(ctx, gmu, gS, gld, grd):
                Xt, sub = ctx.saved_tensors
                mu, S, c = ctx.fit
                g = rtdetmcd_vjp(Xt.detach(), sub, mu, S, c, gmu=gmu, gSigma=gS,
                                 glogdet=float(gld) if gld is not None else 0.0, gRD=grd)
                return g, None, None

        _outputs_fn = _Outputs
    return _outputs_fn.apply(X, h, fit_kwargs)


_objective_fn = None


def rtdetmcd_objective(X, h, *, w_logdet=1.0, w_rd=1.0, **fit_kwargs):
    """Differentiable scalar w_logdet log det Sigma + w_rd sum_i RD_i of the
    reweighted fit of the rows of X (a CUDA float32 tensor).  The forward
    pass runs rtdetmcd_fit; the backward pass holds its reweighting set W
    fixed (the set is a discrete choice) and applies rtdetmcd_grad.  Returns
    a 0-d float64 tensor on X's device."""
    global _objective_fn
    torch = _torch()
    if _objective_fn is None:
        class _Objective(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Xt, hh, wl, wr, kw):
                fit = rtdetmcd_fit(Xt.detach(), hh, d2=False, flags=False, subset=True, **kw)
                val, _ = rtdetmcd_grad(Xt.detach(), fit["subset"], fit["mu"], fit["Sigma"], fit["c_rew"],
                                       w_logdet=wl, w_rd=wr, grad=False)
                ctx.save_for_backward(Xt, fit["subset"])
                ctx.fit = (fit["mu"], fit["Sigma"], fit["c_rew"], wl, wr)
                return torch.tensor(val, dtype=torch.float64, device=Xt.device)

            @staticmethod
            def backward(ctx, gout):
                Xt, sub = ctx.saved_tensors
                mu, S, c, wl, wr = ctx.fit
                _, g = rtdetmcd_grad(Xt.detach(), sub, mu, S, c, w_logdet=wl, w_rd=wr, grad=True)
                return g * gout.to(torch.float32), None, None, None, None

        _objective_fn = _Objective
    return _objective_fn.apply(X, h, float(w_logdet), float(w_rd), fit_kwargs)


def rtdetmcd_flag(d2, cutoff_d2, *, stream=None, workspace=None):
    """flags = d2 > cutoff_d2 and their count."""
    lib = _load()
    torch = _torch()
    if isinstance(d2, torch.Tensor) and d2.is_cuda:
        dev, ptr, n = d2.device, d2.data_ptr(), d2.numel()
    else:
        d2 = np.ascontiguousarray(d2, dtype=np.float32)
        dev, ptr, n = None, d2.ctypes.data, d2.size
    fl = _out(n, np.uint8, dev)
    ws = workspace if workspace is not None else _workspace(n * 5 + 1024, dev)
    cnt = ctypes.c_int64(0)
    st = lib.rtdetmcd_flag(ptr, n, float(cutoff_d2), _ptr(fl), ctypes.byref(cnt), ws.data_ptr(),
                           ws.numel(), _stream_ptr(dev, stream))
    if st != 0:
        raise RtdError(st, lib.rtdetmcd_status_string(st).decode())
    return fl, cnt.value
