#!/usr/bin/env python
"""RT-DetMCD fit throughput on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one full RT-DetMCD fit (Section 4 steps 1-10) of the synthetic
workload n = 1,000,000, p = 20, h = floor(0.75 n), 20% cluster outliers
N(5 v_min, 0.1^2 I) around N(0, R), cond(R) = 100 (seeded), with the rows
resident in HBM.  The FP32 form (FP32 row passes, FP64 p x p algebra and FP64
decisions near every threshold) is the headline; the plain FP64 form is
timed beside it.  One JSON line is printed by rank 0.

Timing: CUDA events on the fit's stream around each step, L2 flushed (a
512 MiB write) before every timed step, outside the events.  Several GPUs run
independent replicas (one problem per rank, no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rows/s per full RT-DetMCD fit (n=1e6,p=20) vs plain FP64 GPU; HBM roofline %"
WORKLOAD = ("RT-DetMCD fit, n=1,000,000 x p=20 float32 rows, h=floor(0.75n), q=12 blocks; "
            "N(0,R) cond(R)=100 + 20% cluster outliers N(5 v_min, 0.1^2 I), seed=rank")
# oracle sample: the first 655,360 rows of the workload (q = 8 blocks, so 16
# independent (block, start) units for the host cores)
CPU_SAMPLE_ROWS = 655_360


# dram__bytes_read.sum + dram__bytes_write.sum of one k_dist_win launch at
# n=1e6, p=20 with both chains of every block active (80.22 MB + 3.64 MB)
K_DIST_TRAFFIC = 83.86e6


def selection_stats(pp):
    """Window-path counters of one profiled fit (chain steps summed)."""
    ws = pp.get("win_steps", 0)
    steps = max(1, ws)
    return {"window_chain_steps": ws, "window_misses": pp.get("win_miss", 0),
            "candidates_per_window_step": pp.get("sel_cand", 0) / steps,
            "band_rows_total": pp.get("sel_band", 0)}


SCORE_N, SCORE_P = 2048 * 4096, 4       # one test image of the paper's almond line (Section 6)


def scoring_leg(rtd, torch, datagen, dev, stream, flush, peak, peak_kind, reps=20):
    """Scoring of new rows against an existing fit (Section 6, step 10):
    rtdetmcd_score on device buffers, distances, flags and count in one
    pass.  Algorithmic bytes per call n (4p + 4 + 1): rows read, d2 and
    flags written.  The roofline is taken on the whole call (fit
    preparation, the pass and the status read) and on the pass alone (call
    time minus that of a 1,024-row call)."""
    import numpy as np
    n, p = SCORE_N, SCORE_P
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    R, _ = datagen.random_correlation(p, 100.0, np.random.default_rng(7))
    L = torch.linalg.cholesky(torch.from_numpy(R)).to(dev, torch.float32)
    X = torch.randn(n, p, generator=g, device=dev) @ L.T
    X[: n // 10] += 6.0                      # 10% shifted rows
    mu, Sigma = np.zeros(p), R
    cut = rtd.rtdetmcd_chi2_quantile(p, 0.975)
    ws = torch.empty(rtd.rtdetmcd_score_workspace_size(n, p), dtype=torch.uint8, device=dev)
    d2o = torch.empty(n, dtype=torch.float32, device=dev)
    flo = torch.empty(n, dtype=torch.uint8, device=dev)
    lib = rtd._load()
    import ctypes
    cnt = ctypes.c_int64(0)
    mu_c, S_c = np.ascontiguousarray(mu), np.ascontiguousarray(Sigma)

    def call(Xin):
        k = Xin.shape[0]
        st = lib.rtdetmcd_score(Xin.data_ptr(), k, p, p, mu_c.ctypes.data, S_c.ctypes.data, cut, rtd.RTD_FP32,
                                d2o.data_ptr(), flo.data_ptr(), ctypes.byref(cnt), ws.data_ptr(), ws.numel(),
                                ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        return cnt.value

    def time_calls(Xin, k):
        ts = []
        for i in range(k):
            flush.fill_(i & 255)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nf = call(Xin)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), nf

    for _ in range(3):
        call(X)
        call(X[:1024])
    t_full, nflag = time_calls(X, reps)
    t_small, _ = time_calls(X[:1024], reps)
    bytes_ = n * (4 * p + 4 + 1)
    # the sorting line's form: the fit prepared once, then one launch per
    # image (no factorisation, no host wait inside the call), images
    # submitted back to back.  Four distinct images (4 x 134 MB, larger than
    # L2) are cycled, so no call finds its rows in L2; the time per image is
    # that of a run of calls between two events.
    prep = rtd.rtdetmcd_score_prepare(mu, Sigma, cut, device=dev)
    cnt_d = torch.zeros(1, dtype=torch.int64, device=dev)
    imgs = [X] + [torch.randn(n, p, generator=g, device=dev) @ L.T for _ in range(3)]
    img_ptr = [im.data_ptr() for im in imgs]
    prep_ptr, d2_ptr, fl_ptr, cnt_ptr = prep.data_ptr(), d2o.data_ptr(), flo.data_ptr(), cnt_d.data_ptr()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def call_prepared(k):
        st = lib.rtdetmcd_score_prepared(img_ptr[k % 4], n, p, p, prep_ptr, rtd.RTD_FP32, d2_ptr, fl_ptr, cnt_ptr,
                                         sp)
        assert st == 0

    call_prepared(0)
    torch.cuda.synchronize()
    assert int(cnt_d.item()) == int(nflag)
    for k in range(3):
        call_prepared(k)
    runs = []
    for rep in range(5):
        flush.fill_(rep & 255)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            call_prepared(k)
        e1.record(stream)
        e1.synchronize()
        runs.append(e0.elapsed_time(e1) / reps)
    t_prep = statistics.median(runs)
    del imgs
    a_prep = bytes_ / (t_prep / 1e3) / 1e9
    t_stream = max(t_full - t_small, 1e-6)
    a_call = bytes_ / (t_full / 1e3) / 1e9
    a = bytes_ / (t_stream / 1e3) / 1e9
    return {"workload": f"scoring {n:,} x {p} float32 rows (one {2048}x{4096} image), distances + flags + count",
            "form": "fit prepared once (rtdetmcd_score_prepare), one rtdetmcd_score_prepared launch per image, "
                    f"{reps} images back to back cycling 4 distinct images (537 MB, larger than L2)",
            "rows_per_s": n / (t_prep / 1e3), "ms_per_call": t_prep, "n_flagged": int(nflag),
            "roofline": {"kernel": "k_score (one pass: distances, FP64-band flags, count)",
                         "bound": "hbm", "achieved": a_prep, "peak": peak, "unit": "GB/s", "frac": a_prep / peak,
                         "peak_kind": peak_kind, "bytes_per_call": bytes_},
            "one_shot_call": {"path": "rtdetmcd_score (factorisation, pass, status read per call)",
                              "rows_per_s": n / (t_full / 1e3), "ms_per_call": t_full, "fixed_ms": t_small,
                              "achieved": a_call, "frac": a_call / peak,
                              "pass_only": {"achieved": a, "frac": a / peak, "stream_ms": t_stream}}}


def adjoint_leg(rtd, torch, X, h, dev, stream, flush, peak, peak_kind, reps=20):
    """Value and gradient of log det Sigma + sum_i RD_i in X with the
    reweighting set W of the fit held fixed (steps 8-10): rtdetmcd_grad on
    the bench's own rows.  Algorithmic bytes per call: the rows twice (the
    Gram pass and the gradient pass), the subset bytes twice, the gradient
    written once."""
    fit = rtd.rtdetmcd_fit(X, h, subset=True, d2=False, flags=False, stream=stream.cuda_stream)
    n, p = X.shape
    sub, mu, S, c = fit["subset"], fit["mu"], fit["Sigma"], fit["c_rew"]
    ws = torch.empty(rtd.rtdetmcd_grad_workspace_size(n, p), dtype=torch.uint8, device=dev)

    def call():
        return rtd.rtdetmcd_grad(X, sub, mu, S, c, workspace=ws, stream=stream.cuda_stream)

    for _ in range(3):
        call()
    ts = []
    for i in range(reps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        val, g = call()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    t = statistics.median(ts)
    bytes_ = n * (4 * p * 3 + 2)
    a = bytes_ / (t / 1e3) / 1e9
    return {"workload": f"adjoint of steps 8-10 on the fit of the bench rows ({n:,} x {p}), W fixed",
            "rows_per_s": n / (t / 1e3), "ms_per_call": t, "value": val, "n_reweight": fit["n_reweight"],
            "roofline": {"kernel": "k_grad_gram + k_sum_slots + k_grad_rows (whole call)", "bound": "hbm",
                         "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                         "peak_kind": peak_kind, "bytes_per_call": bytes_}}


BATCH_FRAMES = 4096


def batched_leg(rtd, torch, datagen, dev, stream, nstreams=16, reps=2):
    """Many independent frames (n ~ U[2000, 50000], p ~ U{8, 16, 24, 32, 40},
    0-25% point outliers at 10 v_min, each fitted with q = 1) through
    rtdetmcd_fit_batch.  Frames are drawn on the device: N(0, R) rows with R
    the frame's seeded random correlation matrix (condition 100), outlier
    rows at seeded random positions set to 10 v_min."""
    import numpy as np
    g = torch.Generator(device=dev)
    frames, hs = [], []
    for f in range(BATCH_FRAMES):
        rng = np.random.default_rng(10_000 + f)
        n = int(rng.integers(2000, 50001))
        p = int(rng.choice([8, 16, 24, 32, 40]))
        eps = float(rng.uniform(0.0, 0.25))
        R, v = datagen.random_correlation(p, 100.0, rng)
        C = torch.linalg.cholesky(torch.from_numpy(R)).to(dev, torch.float32)
        g.manual_seed(f)
        X = torch.randn(n, p, generator=g, device=dev) @ C.T
        k = int(np.floor(eps * n))
        if k:
            pos = torch.randperm(n, generator=g, device=dev)[:k]
            X[pos] = (10.0 * torch.from_numpy(v)).to(dev, torch.float32)
        frames.append(X.contiguous())
        hs.append(int(np.floor(0.75 * n)))
    rows = sum(int(X.shape[0]) for X in frames)
    ws = torch.empty(rtd.rtdetmcd_fit_batch_workspace_size(frames, nstreams), dtype=torch.uint8, device=dev)
    def run(graph):
        return rtd.rtdetmcd_fit_batch(frames, hs, nstreams=nstreams, workspace=ws, stream=stream.cuda_stream,
                                      graph=graph, autotune=1)

    res_by = {}
    for graph in (1, 0):
        run(graph)   # warm-up (graph: captures, instantiates and tunes each width class)
        ts = []
        for i in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = run(graph)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        res_by[graph] = (statistics.median(ts), out)
    # the faster launch mode is the leg's figure; the other is reported beside it
    t_graph, t_stream = res_by[1][0], res_by[0][0]
    primary = 1 if t_graph < t_stream else 0
    t, out = res_by[primary]
    tuned = {}
    for pp in (8, 16, 24, 32, 40):
        for nn in (4000, 25000):
            tv = rtd.rtdetmcd_tuned(nn, pp)
            if tv:
                tuned[f"p={pp},n~{nn}"] = {"win_rows": tv["win_rows"], "sel_ctas": tv["sel_ctas"]}
    res = {"workload": f"{BATCH_FRAMES} frames, n ~ U[2000, 50000], p ~ U{{8,16,24,32,40}}, 0-25% point "
                       f"outliers at 10 v_min, FP32 form, q = 1 per frame ({rows:,} rows, inputs larger than L2)",
           "frames_per_s": BATCH_FRAMES / (t / 1e3), "rows_per_s": rows / (t / 1e3), "ms_per_batch": t,
           "nstreams": nstreams, "flagged_total": int(sum(o["n_flagged"] for o in out)),
           "form": ("each frame one captured CUDA graph (device-side C-step loop), updated in place from frame "
                    "to frame" if primary else "stream launches with host loop control per frame") +
                   ", frames concurrent on 16 streams from host worker threads; launch shapes autotuned per "
                   "width class",
           "graph_launches": {"ms_per_batch": t_graph, "frames_per_s": BATCH_FRAMES / (t_graph / 1e3)},
           "stream_launches": {"ms_per_batch": t_stream, "frames_per_s": BATCH_FRAMES / (t_stream / 1e3)},
           "tuned_shapes": tuned}
    del frames, ws
    torch.cuda.empty_cache()
    return res


LARGE_N, LARGE_P = 10_000_000, 40


def large_p_leg(rtd, torch, datagen, dev, stream, flush, peak, peak_kind, reps=3):
    """The large-p workload (n = 10,000,000, p = 40, 15% mixed contamination):
    the split-BF16 form (every Gram on tcgen05) beside the FP32 and FP64
    forms, with the BF16 and FP32 forms' errors against the FP64 form (which
    holds 1e-9 against the FP64 oracle in the parity tests)."""
    import numpy as np
    fr = datagen.large_case(seed=0, n=LARGE_N, p=LARGE_P)
    n, p, h = fr.X.shape[0], fr.X.shape[1], fr.h
    X = torch.from_numpy(fr.X).to(dev)
    del fr
    out = {"workload": f"n={n:,} x p={p} float32 rows, h=floor(0.75n), 7.5% point outliers at 8 v_min "
                       f"+ 7.5% cluster N(5 v_min, 0.1^2 I), cond(R)=100, seed 0"}
    fits = {}
    for name, prec in (("bf16", rtd.RTD_BF16), ("fp32", rtd.RTD_FP32), ("fp64", rtd.RTD_FP64)):
        ws = torch.empty(rtd.rtdetmcd_workspace_size(n, p, precision=prec), dtype=torch.uint8, device=dev)
        r = rtd.rtdetmcd_fit(X, h, precision=prec, workspace=ws, stream=stream.cuda_stream)   # warm-up
        ts = []
        for i in range(reps if name != "fp64" else 1):
            flush.fill_(i & 255)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = rtd.rtdetmcd_fit(X, h, precision=prec, workspace=ws, stream=stream.cuda_stream,
                                 profile=(name == "bf16" and i == 0))
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            if "profile" in r:
                prof = r["profile"]
        t = statistics.median(ts)
        fits[name] = r
        out[name] = {"ms_per_fit": t, "rows_per_s": n / (t / 1e3), "q": r["q"], "csteps": r["csteps_max"]}
        del ws
    ref = fits["fp64"]
    d2ref = ref["d2"].double()
    for name in ("bf16", "fp32"):
        g = fits[name]
        sc = np.sqrt(np.max(np.diag(ref["Sigma"])))
        out[name]["err_vs_fp64"] = {
            "mu": float(np.max(np.abs(g["mu"] - ref["mu"])) / sc),
            "Sigma": float(np.max(np.abs(g["Sigma"] - ref["Sigma"])) / np.max(np.abs(ref["Sigma"]))),
            "Sigma_raw": float(np.max(np.abs(g["Sigma_raw"] - ref["Sigma_raw"])) / np.max(np.abs(ref["Sigma_raw"]))),
            "logdet_abs": abs(g["logdet"] - ref["logdet"]),
            "d2_max_rel": float(((g["d2"].double() - d2ref).abs() / d2ref.clamp_min(1e-3)).max()),
            "flags_differ": int((g["flags"] != ref["flags"]).sum()),
        }
    st = prof["stages"]
    gram_ms = sum(st[k]["ms"] for k in ("starts", "cstep_update", "reweight"))
    gram_by = sum(st[k]["bytes"] for k in ("starts", "cstep_update", "reweight"))
    a = gram_by / (gram_ms / 1e3) / 1e9
    out["bf16"]["gram_stages"] = {
        "stages": "starts + cstep_update + reweight (the kernels holding the tcgen05 Gram)",
        "ms_per_fit": gram_ms, "bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s",
        "frac": a / peak, "peak_kind": peak_kind}
    out["bf16_speedup_vs_fp32"] = out["fp32"]["ms_per_fit"] / out["bf16"]["ms_per_fit"]
    out["bf16_speedup_vs_fp64"] = out["fp64"]["ms_per_fit"] / out["bf16"]["ms_per_fit"]
    del X, fits, ref, d2ref
    torch.cuda.empty_cache()
    return out


# FP64 FMA pipe of this GPU: 152 SMs x 2 FP64 FMA per clock (measured with
# dependent-chain microbenchmarks: about 1 TFLOP/s at the median clock) x 2
# flops x the 2,070 MHz maximum SM clock.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070


def fp64_roofline(pp):
    """The plain FP64 form's C-step distance stage against the FP64 ALU: p (p + 3)
    flops per row and active chain (triangular product and squares), over the
    stage's CUDA-event time."""
    st = pp["stages"]["cstep_dist"]
    a = st["flops"] / (st["ms"] / 1e3) / 1e9
    return {"kernel": "k_dist<FP64> (C-step distances, both starts)", "bound": "alu", "achieved": a,
            "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": a / FP64_PEAK_GFLOPS,
            "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz",
            "stage_ms_per_fit": st["ms"], "share_of_fit": st["ms"] / sum(v["ms"] for v in pp["stages"].values())}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
# The oracle as it stands, in a process of its own (no CUDA): `workers` = 1
# runs it on one thread; more map its independent units (the column
# univariate MCDs and the (block, start) units of steps 1-3, the paper's
# one-thread-per-block topology) over a pool of spawned processes, one
# single-threaded worker per core.
CPU_CODE = r"""
import concurrent.futures as cf, json, multiprocessing as mp, os, sys, time
sys.path.insert(0, os.environ["RTD_ROOT"])
import datagen, oracle
n = int(sys.argv[1]); seed = int(sys.argv[2]); reps = int(sys.argv[3]); workers = int(sys.argv[4])
fr = datagen.main_case(seed=seed)
X = fr.X[:n]
h = int(0.75 * n)
ex = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) if workers > 1 else None
mf = ex.map if ex else map
if ex:
    list(ex.map(abs, range(4 * workers)))       # workers started before the clock
ts = []
for _ in range(reps):
    t = time.perf_counter()
    f = oracle.fit(X, h, map_fn=mf)
    ts.append(time.perf_counter() - t)
if ex:
    ex.shutdown()
print(json.dumps({"n": n, "times": ts, "q": f.q, "workers": workers}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_oracle(n_rows, seed=0, reps=1, workers=1):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["RTD_ROOT"] = ROOT
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", CPU_CODE, str(n_rows), str(seed), str(reps), str(workers)],
                       capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_text(q, workers):
    how = "one host thread" if workers == 1 else (
        f"{workers} single-threaded worker processes over the column MCDs and the 2q (block, start) units")
    return f"first {CPU_SAMPLE_ROWS:,} rows of the seed-0 workload (q={q}), one fit per step, {how}"


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(local_total_ms, rows_per_rank, steps, world, pg=None, device=None):
    """Whole-job rows/s of independent replicas: the rows of every rank over
    the slowest rank's timed total (max over ranks)."""
    tot = float(local_total_ms)
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([tot], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tot = float(t.item())
    return steps * rows_per_rank * world / (tot / 1e3), tot


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    d = run_oracle(CPU_SAMPLE_ROWS, seed=0, reps=args.warmup + args.steps, workers=cores)
    steps = d["times"][args.warmup:]
    t = statistics.mean(steps)
    v = CPU_SAMPLE_ROWS / t
    sample = oracle_sample_text(d["q"], cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": CPU_SAMPLE_ROWS, "p": 20, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--p", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-score", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: each fit as one captured CUDA graph with device-side control flow (cached and "
                         "relaunched); 0: stream launches with host loop control")
    ap.add_argument("--dist-path", type=int, default=0, help="C-step distances: 0 CUDA cores, 1 tensor cores")
    ap.add_argument("--form", default="fp32", choices=["fp32", "bf16"],
                    help="form of the timed fits (the headline is fp32; bf16 needs 25 <= p <= 48)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    import datagen
    import __graft_entry__ as g
    ws_n, rank, local = dist_env()
    g.build()
    import paper_1910_05615_gb300 as rtd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    fr = datagen.main_case(seed=rank, n=args.n, p=args.p)
    n, p, h = fr.X.shape[0], fr.X.shape[1], fr.h
    X = torch.from_numpy(fr.X).to(dev)
    Xh = torch.from_numpy(fr.X).pin_memory()
    stream = torch.cuda.current_stream(dev)
    FORM = rtd.RTD_BF16 if args.form == "bf16" else rtd.RTD_FP32
    ws32 = torch.empty(rtd.rtdetmcd_workspace_size(n, p, precision=FORM), dtype=torch.uint8, device=dev)
    ws64 = (torch.empty(rtd.rtdetmcd_workspace_size(n, p, precision=rtd.RTD_FP64), dtype=torch.uint8,
                        device=dev) if args.fp64_steps > 0 else None)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    d2_buf = torch.empty(n, dtype=torch.float32, device=dev)
    fl_buf = torch.empty(n, dtype=torch.uint8, device=dev)

    def fit(Xin, prec, ws, profile=False):
        if Xin.is_cuda:   # device rows: preallocated outputs, so a captured graph is relaunched
            return rtd.rtdetmcd_fit(Xin, h, precision=prec, workspace=ws, profile=profile,
                                    stream=stream.cuda_stream, graph=bool(args.graph) and not profile,
                                    dist_path=args.dist_path, d2_out=d2_buf, flags_out=fl_buf)
        return rtd.rtdetmcd_fit(Xin, h, precision=prec, workspace=ws, profile=profile, stream=stream.cuda_stream,
                                dist_path=args.dist_path)

    def timed(Xin, prec, ws, k, profile=False):
        out, profs = [], []
        for i in range(k):
            flush.fill_(i & 255)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fit(Xin, prec, ws, profile=profile)
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
            if profile:
                profs.append(r["profile"])
            last = r
        return out, profs, last

    tuning = None
    if args.graph:   # launch shapes of this problem picked by the autotuner (values unchanged)
        tuning = rtd.rtdetmcd_autotune(X, h, precision=FORM, dist_path=args.dist_path, workspace=ws32,
                                       stream=stream.cuda_stream)
    for _ in range(args.warmup):
        fit(X, FORM, ws32)
    barrier()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or str(local)
    clk = Clocks(gpu_index if gpu_index.isdigit() else local)
    time.sleep(0.3)
    t32, _, r32 = timed(X, FORM, ws32, args.steps)
    barrier()
    clocks = clk.stop()
    # the same steps again with per-stage CUDA events on the fit's stream
    tprof, prof32, _ = timed(X, FORM, ws32, args.steps, profile=True)
    # plain FP64 form beside it
    t64, prof64 = [], []
    if args.fp64_steps > 0:
        fit(X, rtd.RTD_FP64, ws64)
        t64, _, r64 = timed(X, rtd.RTD_FP64, ws64, args.fp64_steps)
        _, prof64, _ = timed(X, rtd.RTD_FP64, ws64, 1, profile=True)
    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        fit(Xh, FORM, ws32)
        te = []
        for i in range(max(3, args.steps // 2)):
            flush.fill_(i & 255)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rh = fit(Xh, FORM, ws32)
            e1.record(stream)
            e1.synchronize()
            te.append(e0.elapsed_time(e1))
        e2e_ms = statistics.mean(te)
        e2e = {"value": n / (e2e_ms / 1e3), "unit": "rows/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": n * p * 4, "d2h_bytes_per_step": n * 4 + n + 67_000,
               "path": "rtdetmcd_fit with pinned host X, host d2 and flags outputs"}

    value, tot32 = replica_throughput(sum(t32), n, args.steps, ws_n, pg, dev)
    if rank != 0:
        pg.destroy_process_group()
        return 0

    # stage roofline from the profiles of the timed steps
    peak, peak_kind = peaks()
    stages = {}
    for name in prof32[0]["stages"]:
        ms = sum(pp["stages"][name]["ms"] for pp in prof32)
        by = sum(pp["stages"][name]["bytes"] for pp in prof32)
        la = sum(pp["stages"][name]["launches"] for pp in prof32)
        stages[name] = {"ms_per_fit": ms / len(prof32), "GBps": (by / (ms / 1e3) / 1e9) if ms > 0 else 0.0,
                        "launches_per_fit": la / len(prof32)}
    tot_stage = sum(s["ms_per_fit"] for s in stages.values())
    for s in stages.values():
        s["share"] = s["ms_per_fit"] / tot_stage if tot_stage else 0.0
    def stage_roof(name, kernel):
        ms = sum(pp["stages"][name]["ms"] for pp in prof32)
        by = sum(pp["stages"][name]["bytes"] for pp in prof32)
        la = sum(pp["stages"][name]["launches"] for pp in prof32)
        a = by / (ms / 1e3) / 1e9
        return {"kernel": kernel, "bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s",
                "frac": a / peak, "traffic": None, "peak_kind": peak_kind,
                "bytes_per_launch": by / la, "launch_ms": ms / la}
    dominant = max(stages, key=lambda k: stages[k]["ms_per_fit"])
    roof = stage_roof("sort", "k_sort_hist/scan/scatter (segmented LSD radix sort, 8-bit digits; "
                      "algorithmic bytes per key and pass: 4 B read + 4 B written)")
    roof["dominant_stage"] = dominant
    # ncu DRAM bytes of one launch, taken on the current kernels (null when a
    # kernel changed after its capture); the summaries live under profiles/
    roof["traffic_note"] = ("k_sort_scatter alone: 286.1 MB DRAM per refinement pass of 40 M keys "
                            "(320 MB algorithmic), profiles/k_sort_scatter_refine_n1e6_p20.md")
    roof_c = stage_roof("cstep_dist", "k_dist_win (C-step distances from step 2 on, k_dist at step 1; "
                        "per row 4p B read + 4 B per active chain written)")
    s_ms = sum(pp["stages"][k]["ms"] for pp in prof32 for k in ("cstep_dist", "cstep_select"))
    s_by = sum(pp["stages"][k]["bytes"] for pp in prof32 for k in ("cstep_dist", "cstep_select"))
    roof_c["traffic"] = K_DIST_TRAFFIC
    roof_c["traffic_note"] = "one k_dist_win launch with both chains active: profiles/k_dist_win_cstep_n1e6_p20.md"
    roof_c["dist_plus_select_frac"] = (s_by / (s_ms / 1e3) / 1e9) / peak
    launches = int(sum(sum(st["launches"] for st in pp["stages"].values()) for pp in prof32))
    cpu = None
    if not args.no_cpu:
        try:
            cores = host_cores()
            dm = run_oracle(CPU_SAMPLE_ROWS, seed=0, reps=2, workers=cores)
            d1 = run_oracle(CPU_SAMPLE_ROWS, seed=0, reps=1, workers=1)
            tm = dm["times"][-1]
            cpu = {"value": CPU_SAMPLE_ROWS / tm, "unit": "rows/s", "cores": cores, "kind": "oracle",
                   "sample": oracle_sample_text(dm["q"], cores), "seconds": tm,
                   "single_thread": {"value": CPU_SAMPLE_ROWS / d1["times"][0], "unit": "rows/s", "cores": 1,
                                     "seconds": d1["times"][0], "sample": oracle_sample_text(d1["q"], 1)}}
        except Exception as ex:  # report, do not hide
            cpu = {"error": str(ex)[-300:]}
    scoring = None
    if not args.no_score:
        scoring = scoring_leg(rtd, torch, datagen, dev, stream, flush, peak, peak_kind)
    batched = None
    if not args.no_batch:
        batched = batched_leg(rtd, torch, datagen, dev, stream)
    large = None
    if not args.no_large:
        large = large_p_leg(rtd, torch, datagen, dev, stream, flush, peak, peak_kind)
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_leg(rtd, torch, X, h, dev, stream, flush, peak, peak_kind)
    line = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": ws_n, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.form == "fp32" else "bf16x2 products, f32 rows", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "p": p, "h": h, "q": r32["q"], "form": args.form,
                   "launch": "captured CUDA graph, device-side C-step loop" if args.graph else "stream launches",
                   "cstep_distances": "tensor cores (split TF32)" if args.dist_path else "CUDA cores (FP32)",
                   "l2": "512 MiB write between timed steps (input 80 MB < L2)",
                   "parallelism": f"{ws_n} independent replica(s)"},
        "fp64_form": ({"value": n / (statistics.mean(t64) / 1e3), "unit": "rows/s",
                       "ms_per_step": statistics.mean(t64),
                       "fp32_speedup": statistics.mean(t64) / (tot32 / args.steps),
                       "roofline": fp64_roofline(prof64[0])} if t64 else None),
        "roofline": roof, "roofline_cstep": roof_c, "stages": stages, "csteps": prof32[-1]["csteps"],
        "autotuned_shape": tuning,
        "selection": selection_stats(prof32[-1]),
        "profiled_ms_per_step": statistics.mean(tprof),
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches, "scoring": scoring,
        "adjoint": adjoint, "large_p": large, "batched": batched,
        "n_flagged": r32["n_flagged"], "step_ms": t32,
    }
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
