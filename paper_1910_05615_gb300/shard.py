"""One RT-DetMCD fit sharded over the processes of a torch.distributed group
(one GPU per process).

Section 4 runs every block on its own thread and exchanges only small
summaries between the steps; the sharded fit keeps that structure:

  1. columns: process r fits the univariate MCD of its ceil(p/G) columns
     (Section 3.1, eq. standardization); all-gather of 2 values per column;
  2. blocks:  process r runs steps 2-4 on its ceil(q/G) consecutive blocks of
     the random partition; all-gather of the q block fits
     (2 + p + p^2 values each);
  3. steps 5-7 (median, KL, keep, pool) run on every process from the same q
     fits, so every process holds the same raw fit; the step-8 distances of
     its own blocks' rows give the reweighting moments (count, sum, centred
     cross-products: 1 + p + p^2 values), summed over the processes;
  4. step 9 from the summed moments on every process, then step 10 on its
     ceil(n/G) consecutive original rows.

Every process holds all of X (rows and columns).  The exchanges are
collectives of the group's backend: NCCL on CUDA tensors, gloo on host
tensors.  A stage's status is combined over the processes (largest code)
before the next stage, so every process raises the same error and none is
left waiting in a collective.

The stage computations come from a backend object (default: the C ABI's
stage calls on this process's GPU, `CudaStages`); it has no CPU fallback.
"""
from dataclasses import dataclass

import numpy as np

from . import (RTD_FP32, RtdError, rtdetmcd_fit_blocks, rtdetmcd_partition, rtdetmcd_reweight_finish,
               rtdetmcd_reweight_moments, rtdetmcd_standardize, rtdetmcd_status_string)


@dataclass(frozen=True)
class ShardRanges:
    """Half-open ranges of one process: columns, blocks, original rows."""
    cols: tuple
    blocks: tuple
    rows: tuple


def shard_range(total: int, world: int, rank: int) -> tuple:
    """Consecutive shares of ceil(total / world); trailing processes may get
    an empty range."""
    k = -(-total // world)
    lo = min(rank * k, total)
    return lo, min(lo + k, total)


def shard_ranges(n: int, p: int, q: int, world: int, rank: int) -> ShardRanges:
    return ShardRanges(shard_range(p, world, rank), shard_range(q, world, rank), shard_range(n, world, rank))


class CudaStages:
    """The stage calls of the C ABI (rtdetmcd_standardize, _fit_blocks,
    _reweight_moments, _reweight_finish) on the rows X (a CUDA tensor, or
    host rows copied in by every call), with one workspace for all calls."""

    def __init__(self, X, h, *, precision=RTD_FP32, omega=4096, q=0, seed=0, max_csteps=100, cutoff_q=0.975,
                 kappa_max=1000.0, reweight_consistency=1, select_path=0, dist_path=0, stream=None):
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda):
            raise ValueError("CudaStages needs the rows as a CUDA tensor")
        self.X, self.h, self.n, self.p = X, int(h), X.shape[0], X.shape[1]
        self.opts = dict(precision=precision, omega=omega, q=q, seed=seed, max_csteps=max_csteps,
                         cutoff_q=cutoff_q, kappa_max=kappa_max, reweight_consistency=reweight_consistency,
                         select_path=select_path, dist_path=dist_path)
        from . import rtdetmcd_workspace_size
        self.ws = torch.empty(rtdetmcd_workspace_size(self.n, self.p, precision, omega, q), dtype=torch.uint8,
                              device=X.device)
        self.stream = stream

    def partition(self):
        return rtdetmcd_partition(self.n, self.p, self.h, **self.opts)

    def _kw(self):
        return dict(stream=self.stream, workspace=self.ws, check=False, **self.opts)

    def standardize(self, lo, hi):
        return rtdetmcd_standardize(self.X, self.h, lo, hi, **self._kw())

    def fit_blocks(self, uni, lo, hi):
        return rtdetmcd_fit_blocks(self.X, self.h, uni, lo, hi, **self._kw())

    def reweight_moments(self, uni, fits, lo, hi):
        return rtdetmcd_reweight_moments(self.X, self.h, uni, fits, lo, hi, **self._kw())

    def reweight_finish(self, uni, fits, moments, lo, hi):
        return rtdetmcd_reweight_finish(self.X, self.h, uni, fits, moments, lo, hi, **self._kw())


class _Comm:
    """Collectives of the group on small float64 / int64 arrays."""

    def __init__(self, group):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        nccl = dist.get_backend(group) == "nccl"
        self.device = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")

    def _t(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).to(self.device)

    def all_gather(self, a, k):
        """Rows of a ((len, w), len <= k) of every process, in rank order."""
        a = np.asarray(a, dtype=np.float64)
        pad = np.zeros((k,) + a.shape[1:], dtype=np.float64)
        pad[:a.shape[0]] = a
        t = self._t(pad)
        parts = [self.torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return [x.cpu().numpy() for x in parts]

    def sum(self, a):
        t = self._t(np.asarray(a, dtype=np.float64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def check(self, status):
        """Largest status over the processes; raises RtdError on every process
        if it is not 0."""
        t = self._t(np.array([int(status)], dtype=np.int64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        code = int(t.cpu().numpy()[0])
        if code:
            raise RtdError(code, rtdetmcd_status_string(code))


def fit_sharded(X, h, *, group=None, stages=None, gather=False, **options):
    """RT-DetMCD fit of X (n x p) with coverage h, sharded over the processes
    of `group` (the default group when None).  Every process passes the same
    X, h and options.  `stages` overrides the stage backend (default
    CudaStages(X, h, **options)).

    Returns a dict with the reweighted and raw fits (X units; the same on
    every process), this process's ranges, the squared distances and flags of
    its rows, n_flagged over all rows, and with gather=True the distances and
    flags of all n rows (host arrays) on every process."""
    comm = _Comm(group)
    st = stages if stages is not None else CudaStages(X, h, **options)
    n, p = st.n, st.p
    q, m = st.partition()
    G = comm.world
    R = shard_ranges(n, p, q, G, comm.rank)
    kc, kb, kr = -(-p // G), -(-q // G), -(-n // G)
    # 1. columns
    code, uni_loc = (0, np.zeros((2, 0))) if R.cols[1] == R.cols[0] else st.standardize(*R.cols)
    comm.check(code)
    parts = comm.all_gather(np.asarray(uni_loc).T, kc)   # (k, 2) per process
    lens = [shard_range(p, G, r) for r in range(G)]
    cols = np.concatenate([parts[r][:hi - lo] for r, (lo, hi) in enumerate(lens)], axis=0)
    uni = np.concatenate([cols[:, 0], cols[:, 1]])
    # 2. blocks
    code, fits_loc = st.fit_blocks(uni, *R.blocks)
    comm.check(code)
    parts = comm.all_gather(np.asarray(fits_loc).reshape(-1, 2 + p + p * p), kb)
    lens = [shard_range(q, G, r) for r in range(G)]
    fits = np.concatenate([parts[r][:hi - lo] for r, (lo, hi) in enumerate(lens)], axis=0)
    # 3. steps 5-7 everywhere, moments of this process's blocks
    code, mom = st.reweight_moments(uni, fits, *R.blocks)
    comm.check(code)
    mom = comm.sum(mom)
    # 4. step 9, step 10 on this process's rows
    code, res = st.reweight_finish(uni, fits, mom, *R.rows)
    comm.check(code)
    out = dict(res)
    out.update(q=q, m=m, world=G, rank=comm.rank, ranges=R, uni=uni, fits=fits, moments=mom,
               n_flagged_local=res["n_flagged"])
    out["n_flagged"] = int(comm.sum(np.array([float(res["n_flagged"])]))[0])
    if gather:
        lens = [shard_range(n, G, r) for r in range(G)]
        for key in ("d2", "flags"):
            loc = res[key]
            loc = loc.cpu().numpy() if hasattr(loc, "cpu") else np.asarray(loc)
            parts = comm.all_gather(loc.astype(np.float64), kr)   # exact for float32 and bytes
            out[key + "_all"] = np.concatenate([parts[r][:hi - lo] for r, (lo, hi) in enumerate(lens)]).astype(
                loc.dtype)
    return out
