"""GPU: the stage entry points of a sharded fit, through the C ABI.

The stages of G processes are run one after another on this GPU, with the
exchanges done in host memory in rank order (no process waits on another);
a last test runs two real processes on this GPU that exchange through gloo.
"""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle as O
from parity import compare_fit, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtd():
    import __graft_entry__ as g
    g.build()
    import paper_1910_05615_gb300 as m
    return m


def _emulate(rtd, X, h, G, **opts):
    from paper_1910_05615_gb300.shard import shard_range
    n, p = X.shape
    q, m = rtd.rtdetmcd_partition(n, p, h, **opts)
    dev = X.device if isinstance(X, torch.Tensor) else torch.device("cuda", 0)
    ws = torch.empty(rtd.rtdetmcd_workspace_size(n, p, opts.get("precision", rtd.RTD_FP32)), dtype=torch.uint8,
                     device=dev)
    kw = dict(workspace=ws, **opts)
    cols = []
    for r in range(G):
        lo, hi = shard_range(p, G, r)
        if hi > lo:
            st, u = rtd.rtdetmcd_standardize(X, h, lo, hi, **kw)
            assert st == 0
            cols.append(u)
    cols = np.concatenate(cols, axis=1)
    uni = np.concatenate([cols[0], cols[1]])
    fits = []
    for r in range(G):
        st, f = rtd.rtdetmcd_fit_blocks(X, h, uni, *shard_range(q, G, r), **kw)
        assert st == 0
        fits.append(f)
    fits = np.concatenate(fits, axis=0)
    assert fits.shape == (q, 2 + p + p * p)
    mom = None
    for r in range(G):
        st, mo = rtd.rtdetmcd_reweight_moments(X, h, uni, fits, *shard_range(q, G, r), **kw)
        assert st == 0
        mom = mo if mom is None else mom + mo
    parts = []
    for r in range(G):
        st, res = rtd.rtdetmcd_reweight_finish(X, h, uni, fits, mom, *shard_range(n, G, r), **kw)
        assert st == 0
        parts.append(res)
    return q, uni, fits, mom, parts


def _case(n, p, seed=3):
    fr = datagen.contaminated_gaussian(n, p, eps=0.2, kind="cluster", shift=5.0, seed=seed)
    return fr.X, fr.h


@pytest.mark.parametrize("form", ["fp32", "fp64"])
@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_stages_compose_to_the_fit(rtd, form, G):
    """Block fits and standardisation equal the whole fit's bit for bit; with
    one process the reweighted fit, distances and flags too; with several,
    the reweighted fit moves only by the order of the FP64 moment sums."""
    prec = {"fp32": rtd.RTD_FP32, "fp64": rtd.RTD_FP64}[form]
    X, h = _case(300_000, 6)
    Xd = torch.from_numpy(X).cuda()
    n, p = X.shape
    f = rtd.rtdetmcd_fit(Xd, h, precision=prec, diag=True)
    q, uni, fits, mom, parts = _emulate(rtd, Xd, h, G, precision=prec)
    assert q == f["q"] == 12
    dg = f["diag"]
    np.testing.assert_array_equal(uni[:p], dg["mu_uni"])
    np.testing.assert_array_equal(uni[p:], dg["sigma_uni"])
    for l in range(q):
        c = dg["blocks"][l]["chosen"]
        assert fits[l, 0] == c
        if c >= 0:
            ch = dg["chains"][2 * l + c]
            np.testing.assert_array_equal(fits[l, 2:2 + p], ch["mu"])
            np.testing.assert_array_equal(fits[l, 2 + p:].reshape(p, p), ch["Sigma"])
            assert fits[l, 1] == ch["logdet"]
    assert int(round(mom[0])) == f["n_reweight"]
    d2 = np.concatenate([to_np(r["d2"]) for r in parts])
    fl = np.concatenate([to_np(r["flags"]) for r in parts])
    assert sum(r["n_flagged"] for r in parts) == f["n_flagged"]
    for r in parts:
        np.testing.assert_array_equal(r["mu_raw"], f["mu_raw"])
        np.testing.assert_array_equal(r["Sigma_raw"], f["Sigma_raw"])
        assert r["n_reweight"] == f["n_reweight"]
        if G == 1:
            np.testing.assert_array_equal(r["mu"], f["mu"])
            np.testing.assert_array_equal(r["Sigma"], f["Sigma"])
        else:
            np.testing.assert_allclose(r["mu"], f["mu"], rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(r["Sigma"], f["Sigma"], rtol=1e-11, atol=1e-13 * np.abs(f["Sigma"]).max())
    if G == 1:
        np.testing.assert_array_equal(d2, to_np(f["d2"]))
    else:
        np.testing.assert_allclose(d2, to_np(f["d2"]), rtol=1e-6)
    np.testing.assert_array_equal(fl, to_np(f["flags"]))


def test_sharded_stages_match_oracle(rtd):
    X, h = _case(60_000, 4, seed=8)
    Xd = torch.from_numpy(X).cuda()
    q, uni, fits, mom, parts = _emulate(rtd, Xd, h, 2)
    ref = O.fit(X, h)
    assert q == ref.q == 3
    got = dict(parts[0])
    got["flags"] = np.concatenate([to_np(r["flags"]) for r in parts])
    ok, rep = compare_fit(got, ref, X, "fp32", check_subsets=False)
    assert ok, rep
    for l, b in enumerate(ref.blocks):
        assert fits[l, 0] == b.chosen


def test_stages_from_host_rows(rtd):
    """Host rows are copied in by every stage call; the results equal those
    of device rows."""
    X, h = _case(50_000, 3, seed=11)
    a = _emulate(rtd, torch.from_numpy(X).cuda(), h, 2)
    b = _emulate(rtd, X, h, 2)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[3], b[3])
    for ra, rb in zip(a[4], b[4]):
        np.testing.assert_array_equal(ra["Sigma"], rb["Sigma"])
        np.testing.assert_array_equal(to_np(ra["flags"]), to_np(rb["flags"]))


def test_stage_data_errors(rtd):
    X, h = _case(40_000, 3, seed=2)
    n, p = X.shape
    q, _ = rtd.rtdetmcd_partition(n, p, h)
    Xd = torch.from_numpy(X).cuda()
    q_, uni, fits, mom, _ = _emulate(rtd, Xd, h, 1)
    Xn = X.copy()
    Xn[123, 1] = np.nan
    Xnd = torch.from_numpy(Xn).cuda()
    assert rtd.rtdetmcd_standardize(Xnd, h, 0, 1, check=False)[0] == 0     # column 0 is finite
    assert rtd.rtdetmcd_standardize(Xnd, h, 1, 2, check=False)[0] == 2     # RTD_ENONFINITE
    assert rtd.rtdetmcd_fit_blocks(Xnd, h, uni, 0, 1, check=False)[0] == 2
    bad = uni.copy()
    bad[p] = 0.0                                                           # zero scale
    assert rtd.rtdetmcd_fit_blocks(Xd, h, bad, 0, 1, check=False)[0] == 1
    f2 = fits.copy()
    f2[1, 0] = 0.5                                                         # no such start
    assert rtd.rtdetmcd_reweight_moments(Xd, h, uni, f2, 0, q, check=False)[0] == 1
    f3 = fits.copy()
    f3[:, 0] = -1.0                                                        # no block has a fit
    assert rtd.rtdetmcd_reweight_moments(Xd, h, uni, f3, 0, q, check=False)[0] == 3
    st, res = rtd.rtdetmcd_reweight_finish(Xd, h, uni, fits, mom * 0.0, 0, n, check=False)
    assert st == 4                                                         # empty reweighting set
    # the context is still usable
    st, res = rtd.rtdetmcd_reweight_finish(Xd, h, uni, fits, mom, 0, n)
    assert st == 0


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1910_05615_gb300.shard import fit_sharded
        torch.cuda.set_device(0)
        X, h = _case(200_000, 5, seed=4)
        r = fit_sharded(torch.from_numpy(X).cuda(), h, gather=True)
        out.put((rank, {k: r[k] for k in ("mu", "Sigma", "n_flagged", "flags_all", "q")}))
    except Exception as e:   # reported to the test
        out.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_processes_through_gloo(rtd):
    """The whole orchestration with the CUDA stages: two processes on this
    GPU (their kernels never wait on each other; the exchanges are gloo
    collectives on host tensors) give the single-process fit."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(out.get(timeout=600) for _ in range(2))
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    X, h = _case(200_000, 5, seed=4)
    f = rtd.rtdetmcd_fit(torch.from_numpy(X).cuda(), h)
    for r in range(2):
        a = res[r]
        assert isinstance(a, dict), a
        assert a["q"] == f["q"]
        np.testing.assert_allclose(a["Sigma"], f["Sigma"], rtol=1e-11, atol=1e-13 * np.abs(f["Sigma"]).max())
        np.testing.assert_allclose(a["mu"], f["mu"], rtol=1e-12, atol=1e-13)
        assert a["n_flagged"] == f["n_flagged"]
        np.testing.assert_array_equal(a["flags_all"], to_np(f["flags"]))
