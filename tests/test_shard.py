"""The sharded fit's host logic on CPU: the column, block and row ranges of
each process, and the whole orchestration (all-gathers of the column results
and block fits, the sum of the reweighting moments, the status checks) run
by gloo processes with the oracle as the stage backend, against the oracle's
unsharded fit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1910_05615_gb300.shard import shard_range, shard_ranges  # noqa: E402


@pytest.mark.parametrize("total,world", [(12, 1), (12, 2), (12, 5), (4, 3), (3, 8), (1, 2), (1000003, 7)])
def test_shard_ranges_partition_the_range(total, world):
    rs = [shard_range(total, world, r) for r in range(world)]
    k = -(-total // world)
    assert rs[0][0] == 0 and rs[-1][1] == total
    for r, (lo, hi) in enumerate(rs):
        assert 0 <= lo <= hi <= total and hi - lo <= k
        if r:
            assert lo == rs[r - 1][1]          # consecutive, disjoint
        if hi - lo < k:                        # only the trailing shares are short
            assert all(b - a == 0 for a, b in rs[r + 1:])


def test_shard_ranges_fields():
    R = shard_ranges(n=1000, p=5, q=4, world=3, rank=2)
    assert R.cols == (4, 5) and R.blocks == (4, 4) and R.rows == (668, 1000)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import datagen
    fr = datagen.contaminated_gaussian(12_000, 3, eps=0.15, kind="cluster", shift=6.0, seed=5)
    return fr.X, fr.h


def _worker(rank, world, port, q, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle_stages import OracleStages
        from paper_1910_05615_gb300.shard import fit_sharded
        X, h = _case()
        r = fit_sharded(X, h, stages=OracleStages(X, h, q=q), gather=True)
        out.put((rank, {k: r[k] for k in ("mu", "Sigma", "mu_raw", "Sigma_raw", "n_flagged", "d2_all",
                                          "flags_all", "n_reweight", "q", "rows", "d2", "n_flagged_local")}))
    except Exception as e:   # reported to the test
        out.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,q", [(2, 4), (3, 4)])
def test_sharded_fit_equals_oracle_fit(world, q):
    """World 2 (two blocks each) and world 3 (blocks 2 + 2 + 0: a process
    without blocks still takes part in every exchange)."""
    import oracle as O
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q, out)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(out.get(timeout=600) for _ in range(world))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for r in range(world):
        assert isinstance(res[r], dict), res[r]
    X, h = _case()
    f = O.fit(X, h, q=q)
    n = X.shape[0]
    for r in range(world):
        a = res[r]
        assert a["q"] == q
        # the same fit on every process, equal to the unsharded oracle's up to
        # the order of the FP64 moment sums
        for key, ref in (("mu", f.mu), ("Sigma", f.Sigma), ("mu_raw", f.mu_raw), ("Sigma_raw", f.Sigma_raw)):
            np.testing.assert_allclose(a[key], ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
            np.testing.assert_array_equal(a[key], res[0][key])
        assert a["n_reweight"] == int(f.W.sum())
        assert a["n_flagged"] == int(f.flags.sum())
        np.testing.assert_array_equal(a["flags_all"].astype(bool), f.flags)
        np.testing.assert_allclose(a["d2_all"], f.d2, rtol=1e-9)
        lo, hi = a["rows"]
        assert (lo, hi) == shard_range(n, world, r)
        assert a["n_flagged_local"] == int(f.flags[lo:hi].sum())
    assert sum(res[r]["n_flagged_local"] for r in range(world)) == int(f.flags.sum())


class _FailingStages:
    """Oracle stages whose block stage reports a status on one process."""

    def __init__(self, inner, bad_rank, rank):
        self.inner, self.bad = inner, bad_rank == rank
        self.n, self.p = inner.n, inner.p

    def partition(self):
        return self.inner.partition()

    def standardize(self, lo, hi):
        return self.inner.standardize(lo, hi)

    def fit_blocks(self, uni, lo, hi):
        st, r = self.inner.fit_blocks(uni, lo, hi)
        return (4 if self.bad else st), r


def _failing_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle_stages import OracleStages
        from paper_1910_05615_gb300 import RtdError
        from paper_1910_05615_gb300.shard import fit_sharded
        X, h = _case()
        try:
            fit_sharded(X, h, stages=_FailingStages(OracleStages(X, h, q=2), 1, rank))
            out.put((rank, "no error"))
        except RtdError as e:
            out.put((rank, e.code))
    finally:
        dist.destroy_process_group()


def test_a_failed_stage_stops_every_process():
    """A status on one process (here the block stage of process 1) ends the
    fit with the same RtdError on every process, before the next exchange."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(out.get(timeout=600) for _ in range(2))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    assert res == {0: 4, 1: 4}
