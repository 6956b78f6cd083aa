#!/usr/bin/env python
"""Benchmark of the residual-periodogram hot path (one JSON line on rank 0).

Workload: the residual periodogram of one series with N = 2000 irregular
times over 3000 d, base model = constant + 3 fixed sinusoids (p = 7 columns),
uniform grid of 1e6 trial frequencies 0 < f <= 2 /d; mixed precision (FP32
trigonometric sums, FP64 phases and solves).  A step is one full pass of the
path: prep (base fit, records) -> periodogram kernel -> FP64 re-evaluation of
ill-conditioned bins -> top-5 peaks.

Metric: freq*obs terms per second (N * nf per step), inputs resident in HBM.
The FP64 path is timed on the same workload for the mixed/FP64 ratio, and a
strided sample of the mixed result is checked against the FP64 CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own series (weak scaling, no collective on
the data path); value = all ranks' terms / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "residual periodogram, N=2000, base = constant + 3 sinusoids (p=7), uniform grid nf=1e6 (0<f<=2 /d)"
L2_FLUSH_BYTES = 256 << 20
METRIC = "freq*obs terms/s, mixed vs FP64 on 1 B300, at stated max rel err vs FP64 oracle"
OPS_PER_TERM = lambda p: 2 * p + 8     # FMA-pipe operations per freq*obs term (rotation 4, sums 2p+4 of sqrt(w)-scaled cos/sin)
GRAD_OPS_PER_TERM = lambda p: 4 * p + 13   # z and dz/df: the 2p+8 above, then 2p+4 t'-weighted sums and t' (s c) 1
VJP_OPS_PER_TERM = 6                   # adjoint: rotation 4, a cos + b sin 2
# Library kernels per mixed step (ncu launch list of this workload): initialisation, prep,
# periodogram (main launch and the tail split of its last part-filled wave), re-evaluation
# of flagged bins, top-k stages 1 and 2.
KERNELS_PER_STEP = 7
# dram__bytes_read.sum + dram__bytes_write.sum of one periodogram launch (the
# main kernel and its tail kernel together) on this workload, keyed by (p,
# frequencies per thread, warps per CTA); measured with ncu on the same command
# (--kernel-only).  z (8 MB) stays in L2 during the launch.
DRAM_BYTES_PER_LAUNCH = {(7, 10, 4): 237824 + 242432}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    return rank, ws


def reduce_max(x, ws):
    """Max over ranks (the timing reduction; the only collective of the run)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_rank_workload(rank):
    """Weak scaling: rank r analyses its own series (seed rep = r) on its own
    frequency band [r, r+1) x (the 1e6-point grid), so no data is exchanged."""
    s = synth.residual_n2000_p7(rep=rank)
    s.grid.f0 += rank * s.grid.nf * s.grid.df
    return s


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.out = ""

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def parity_vs_oracle(z, zr, ratio, chi2, tol, N):
    """Largest relative error (floor 1e-3 of the highest z*) over the bins whose
    2x2 system has a condition number below 1e12 (oracle column ratio >= 1e-6),
    the largest |z - z*| / bound with the bound tol max(z*, floor) +
    8 eps64 sqrt(N) chi2_base / ratio^2 (the rounding of an FP64 normal-equation
    method grows as 1/ratio^2), and the number of bins left out."""
    keep = ratio >= 1e-6
    den = np.maximum(np.abs(zr), 1e-3 * np.max(np.abs(zr)))
    bound = tol * den + 8.0 * 2.0 ** -52 * np.sqrt(N) * chi2 / np.maximum(ratio, 1e-6) ** 2
    d = np.abs(z - zr)
    return float(np.max(d[keep] / den[keep])), float(np.max(d[keep] / bound[keep])), int((~keep).sum())


def cpu_baseline(s, nsample):
    """The oracle as it stands, single-threaded, on a strided sample of the grid."""
    import oracle
    f = s.grid.array()
    idx = np.linspace(0, f.size - 1, nsample).astype(np.int64)
    t0 = time.perf_counter()
    oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[idx])
    dt = time.perf_counter() - t0
    return {"value": s.N * nsample / dt, "unit": "terms/s", "cores": 1, "kind": "oracle",
            "sample": f"same series, {nsample} of the {f.size} trial frequencies (evenly strided), "
                      f"one thread, {dt:.1f} s"}


def _oracle_shard(args):
    """One worker of the parallel CPU baseline: the oracle on a shard of the
    sampled frequencies (runs in a spawned process)."""
    import oracle
    t, y, sigma, base, f = args
    oracle.periodogram(t, y, sigma, base, f)
    return f.size


def cpu_baseline_parallel(s, nsample):
    """The same oracle as independent processes over shards of the same
    strided sample, one per available host core (spawned: no GPU context
    is forked)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    f = s.grid.array()
    idx = np.linspace(0, f.size - 1, nsample).astype(np.int64)
    shards = [(s.t, s.y, s.sigma, s.base_freqs, f[idx[r::cores]]) for r in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_shard, [(s.t[:8], s.y[:8], s.sigma[:8], s.base_freqs[:1], f[:2])] * cores)   # start-up
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_shard, shards))
        dt = time.perf_counter() - t0
    return {"value": s.N * done / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"same series, the same {nsample} strided trial frequencies split over {cores} processes "
                      f"(one per host core), {dt:.1f} s"}


def _timed(stream, fn, reps, flush):
    """CUDA-event time (ms) of each of reps calls of fn on stream, L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    out = []
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def bench_batch(F, peak_ops, flush):
    """The 4096-series batch (uneven N, base sizes and grids): one replay of
    the plan's captured graph (prep, persistent periodogram kernel,
    re-evaluation of flagged bins, top-5) per step; parity on sampled series."""
    import torch
    import oracle
    w = synth.batch_4096()
    plan = F.BatchPlan(w.series, precision="mixed", topk=5)
    stream = torch.cuda.Stream()
    for _ in range(2):
        plan.run(stream)
    torch.cuda.synchronize()
    ms = _timed(stream, lambda: plan.run(stream), 4, flush)
    ops = sum(OPS_PER_TERM(2 * len(s.base_freqs) + 1) * s.N * s.grid.nf for s in w.series)
    z, top = plan.download()
    rng = np.random.default_rng(3)
    errs, worst, excl = [], [], 0
    for k in rng.choice(len(w.series), 6, replace=False):
        s = w.series[k]
        zk = z[plan.z_offsets[k]:plan.z_offsets[k] + s.grid.nf]
        idx = np.unique(np.concatenate([np.linspace(0, s.grid.nf - 1, 20).astype(int), top[k][top[k] >= 0]]))
        zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx], want_ratio=True)
        e, wst, n = parity_vs_oracle(zk[idx], zr, ratio, c2, 1e-5, s.N)
        errs.append(e)
        worst.append(wst)
        excl += n
    plan.close()
    t_ms = statistics.median(ms)
    return {"value": plan.terms / (t_ms * 1e-3), "unit": "terms/s", "ms_per_replay": t_ms, "replays": len(ms),
            "series": len(w.series), "terms": plan.terms,
            "roofline_frac": ops / (t_ms * 1e-3) / peak_ops,
            "roofline_note": "2p+8 FP32 ops per term of every series over the whole replay (prep, top-k and "
                             "re-evaluation included) against the unit-count FP32 peak",
            "max_rel_err_vs_oracle": max(errs), "worst_over_bound": max(worst), "excluded_cond_above_1e12": excl,
            "sample": "6 random series x (20 strided bins + their top-5 peaks)"}


def bench_nightly(F, peak_ops, flush):
    """The N = 1e5, 1e7-frequency survey-like series (p = 11), mixed: the
    whole single-series step per call, its periodogram kernel timed by the
    library's events; then the adjoint dL/dy for all points."""
    import torch
    import oracle
    s = synth.nightly_n1e5_p11()
    dev = torch.device("cuda", torch.cuda.current_device())
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    t, y, sg, b = tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs)
    nf = s.grid.nf
    z = torch.empty(nf, dtype=torch.float64, device=dev)
    coef = torch.empty((nf, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    res = {}

    def step():
        res.update(F.periodogram_dev(t, y, sg, b, s.grid.f0, s.grid.df, nf, precision="mixed", topk=5, out=z,
                                     want_coef=True, stream=stream))

    with torch.cuda.stream(stream):
        step()
    torch.cuda.synchronize()
    kev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    kev[0].record(stream)
    kev[1].record(stream)
    kms = []

    def kstep():
        F.profile_events(*kev)
        step()
        F.profile_events(None, None)

    ms = []
    for _ in range(3):
        ms += _timed(stream, kstep, 1, flush)
        kms.append(kev[0].elapsed_time(kev[1]))
    top = res["topk"].cpu().numpy()
    zh = z.cpu().numpy()
    idx = np.unique(np.concatenate([np.linspace(0, nf - 1, 12).astype(int)] + [np.arange(j - 1, j + 2) for j in top[:2]]))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx], want_ratio=True)
    err, worst, excl = parity_vs_oracle(zh[idx], zr, ratio, c2, 1e-5, s.N)
    v = tt(np.random.default_rng(1).standard_normal(nf))
    vjp_ms = _timed(stream, lambda: F.periodogram_vjp_dev(t, y, sg, b, s.grid.f0, s.grid.df, nf, res["coef"],
                                                          res["info"], v, precision="mixed", stream=stream), 2, flush)
    t_ms, k_ms = statistics.median(ms), statistics.median(kms)
    p = 2 * len(s.base_freqs) + 1
    return {"value": s.N * nf / (t_ms * 1e-3), "unit": "terms/s", "ms_per_step": t_ms, "steps": len(ms),
            "kernel_ms": k_ms, "roofline_frac": OPS_PER_TERM(p) * s.N * nf / (k_ms * 1e-3) / peak_ops,
            "max_rel_err_vs_oracle": err, "worst_over_bound": worst, "excluded_cond_above_1e12": excl,
            "sample": "12 strided bins and the neighbourhoods of the two highest peaks",
            "vjp": {"value": s.N * nf / (statistics.median(vjp_ms) * 1e-3), "unit": "terms/s",
                    "ms_per_call": statistics.median(vjp_ms),
                    "roofline_frac": VJP_OPS_PER_TERM * s.N * nf / (statistics.median(vjp_ms) * 1e-3) / peak_ops,
                    "ops_per_term": VJP_OPS_PER_TERM,
                    "what": "dL/dy for all 1e5 points, v ~ N(0,1) on all 1e7 bins (whole call against the "
                            "unit-count FP32 peak)"}}


def bench_grad(F, peak_ops, flush):
    """The benchmark series' z and dz/df on the whole 1e6-frequency grid in one
    pass (two-set records), mixed; the two-set kernel timed by the library's
    events; dz/df sampled against the oracle's gradient."""
    import torch
    import oracle
    s = synth.residual_n2000_p7()
    dev = torch.device("cuda", torch.cuda.current_device())
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    t, y, sg, b = tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs)
    nf = s.grid.nf
    z = torch.empty(nf, dtype=torch.float64, device=dev)
    g = torch.empty(nf, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    call = lambda: F.periodogram_grad_dev(t, y, sg, b, s.grid.f0, s.grid.df, nf, precision="mixed", out=z,
                                          out_grad=g, stream=stream)
    with torch.cuda.stream(stream):
        call()
    torch.cuda.synchronize()
    kev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    kev[0].record(stream)
    kev[1].record(stream)
    ms, kms = [], []
    for _ in range(5):
        def kstep():
            F.profile_events(*kev)
            call()
            F.profile_events(None, None)
        ms += _timed(stream, kstep, 1, flush)
        kms.append(kev[0].elapsed_time(kev[1]))
    gh = g.cpu().numpy()
    idx = np.arange(0, nf, nf // 60)
    gr = oracle.periodogram_grad(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx])
    _, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx], want_ratio=True)
    p = 2 * len(s.base_freqs) + 1
    t_ms, k_ms = statistics.median(ms), statistics.median(kms)
    # the z reading carried over to dz/df (|dz/df| <= about 2 pi T chi2): bins
    # with a 2x2 condition above 1e12 left out, the rounding bound scaled by
    # 1/ratio^2; the mixed path's flagged bins are float-float (eps 2e-15)
    T = s.t.max() - s.t.min()
    keep = ratio >= 1e-6
    den = np.maximum(np.abs(gr), 1e-3 * np.max(np.abs(gr)))
    bound = 1e-4 * den + 8.0 * 2e-15 * np.sqrt(s.N) * 2 * np.pi * T * c2 / np.maximum(ratio, 1e-6) ** 2
    d = np.abs(gh[idx] - gr)
    return {"value": s.N * nf / (t_ms * 1e-3), "unit": "terms/s", "ms_per_step": t_ms, "kernel_ms": k_ms,
            "roofline_frac": GRAD_OPS_PER_TERM(p) * s.N * nf / (k_ms * 1e-3) / peak_ops,
            "ops_per_term": GRAD_OPS_PER_TERM(p),
            "max_rel_err_dzdf_vs_oracle": float(np.max((d / den)[keep & (ratio > 0.45)])),
            "worst_over_bound": float(np.max((d / bound)[keep])), "excluded_cond_above_1e12": int((~keep).sum()),
            "sample": "60 strided bins, floor 1e-3 of the largest sampled |dz/df|; the relative error over the "
                      "bins the kernel does not re-evaluate (ratio > 0.45), the bound over all"}


def bench_pool16(peak_ops):
    """All 65535 non-empty subtuples of the 16-frequency pool (N = 1000)
    refined by Gauss-Newton (at most 20 steps, mixed; the host API call,
    transfers and the float-float redo of ill-conditioned tuples included).
    Roofline: the FP32 work of one pass over the points for a tuple of m
    frequencies is the Gram of its 4m + 2 columns ((4m+2)(4m+3)/2 FMAs a
    point) plus their generation (8 operations a frequency: rotation and
    weighting of cos, sin, t' cos, t' sin), counted for the passes of the
    accepted steps (plus the first) of every tuple, against the unit-count
    FP32 peak; rejected half steps and the float-float redo are not counted
    as work."""
    import paper_1309_0100_b300 as F
    import oracle
    s = synth.pool16_n1000()
    masks = np.arange(1, 1 << 16, dtype=np.uint32)
    F.pool_refine(s.t, s.y, s.sigma, s.pool, masks[:64], max_iter=20, precision="mixed")   # warm-up
    times, it = [], None
    for _ in range(2):
        t0 = time.perf_counter()
        mk, f, l, it = F.pool_refine(s.t, s.y, s.sigma, s.pool, masks, max_iter=20, precision="mixed")
        times.append(time.perf_counter() - t0)
    m = np.array([bin(int(x)).count("1") for x in masks])
    work = int(np.sum((it.astype(np.int64) + 1) * m)) * s.N
    ops = float(np.sum((it.astype(np.float64) + 1) * ((4 * m + 2) * (4 * m + 3) / 2 + 8 * m))) * s.N
    dt = min(times)
    rng = np.random.default_rng(4)
    lerr = 0.0
    l0 = oracle.l0(s.t, s.y, s.sigma)
    for q in rng.choice(masks.size, 6, replace=False):
        sel = [k for k in range(16) if int(masks[q]) >> k & 1]
        lerr = max(lerr, abs(oracle.tuple_l(s.t, s.y, s.sigma, f[q, sel]) - l[q]) / l0)
    return {"seconds": dt, "tuples": int(masks.size), "value": work / dt, "unit": "terms/s",
            "terms": work, "terms_note": "sum over tuples of (accepted Gauss-Newton steps + 1) x m x N "
                                         "(rejected half steps not counted)",
            "roofline_frac": ops / dt / peak_ops,
            "roofline_note": "FP32 Gram and column operations of the counted passes against the unit-count FP32 peak",
            "max_err_l_vs_oracle_at_gpu_freqs": lerr, "err_unit": "of l_0 (FP32 sums resolve l to about 3e-7 of "
                                                                   "l_0)", "sample": "6 random subtuples"}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    s = synth.residual_n2000_p7()
    nsample = 400
    times = []
    import oracle
    f = s.grid.array()
    for k in range(args.warmup + args.steps):
        idx = np.arange(k % 7, f.size, f.size // nsample)[:nsample]
        t0 = time.perf_counter()
        oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, f[idx])
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    T = sum(times)
    value = s.N * nsample * args.steps / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": s.N, "nf": s.grid.nf, "n_base": 3},
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {nsample} evenly strided trial frequencies of the 1e6 grid"},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the batch, survey-series and pool-refinement lines")
    ap.add_argument("--cpu-sample", type=int, default=30000)
    ap.add_argument("--kernel-only", action="store_true",
                    help="profiling runs: fixed launch shape, mixed steps only (no tuning, FP64, e2e or CPU legs)")
    ap.add_argument("--fpt", type=int, default=4)
    ap.add_argument("--warps", type=int, default=4)
    args = ap.parse_args()
    rank, ws = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import paper_1309_0100_b300 as F

    dev = torch.device("cuda", torch.cuda.current_device())
    s = make_rank_workload(rank)
    N, nf, nb = s.N, s.grid.nf, len(s.base_freqs)
    p = 2 * nb + 1
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    t, y, sg, base = tt(s.t), tt(s.y), tt(s.sigma), tt(s.base_freqs)
    z = torch.empty(nf, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    best = {}
    if args.kernel_only:
        best["mixed"] = (args.fpt, args.warps)
    else:
        for prec in ("mixed", "fp64"):
            best[prec] = F.tune(prec, nb, N, nf)

    def timed_steps(prec, steps, warmup):
        shape = best[prec]
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in kev:          # torch creates the CUDA events on first record; the library re-records them
            a.record(stream)
            b.record(stream)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                F.periodogram_dev(t, y, sg, base, s.grid.f0, s.grid.df, nf, precision=prec, topk=5, out=z,
                                  fpt=shape[0], warps=shape[1])
            torch.cuda.synchronize()
            barrier(ws)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for k in range(steps):
                flush.fill_(float(k))                              # L2 flush between steps (untimed)
                sev[k][0].record(stream)
                F.profile_events(*kev[k])
                F.periodogram_dev(t, y, sg, base, s.grid.f0, s.grid.df, nf, precision=prec, topk=5, out=z,
                                  fpt=shape[0], warps=shape[1])
                F.profile_events(None, None)
                sev[k][1].record(stream)
            torch.cuda.synchronize()
            barrier(ws)
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
        step_ms = [a.elapsed_time(b) for a, b in sev]
        kern_ms = [a.elapsed_time(b) for a, b in kev]
        return step_ms, kern_ms, wall

    with Clocks(torch.cuda.current_device()) as clk:
        step_ms, kern_ms, wall = timed_steps("mixed", args.steps, args.warmup)
    clocks = clk.summary()
    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"kernel_only": True, "step_ms": step_ms, "kernel_ms": kern_ms, "clocks": clocks}))
        return
    T = reduce_max(sum(step_ms), ws)
    ms_per_step = T / args.steps
    value = ws * N * nf / (ms_per_step * 1e-3)
    z_mixed = z.cpu().numpy().copy()
    k64 = max(2, args.steps // 5)
    step64, kern64, _ = timed_steps("fp64", k64, 3)
    value64 = ws * N * nf / (reduce_max(sum(step64), ws) / k64 * 1e-3)
    z64 = z.cpu().numpy().copy()

    # end to end through the host-pointer API: pinned inputs in, z out, per step
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
    th, yh, sh, bh, fh = pin(s.t), pin(s.y), pin(s.sigma), pin(s.base_freqs), pin(s.grid.array())
    zh = pin(np.zeros(nf))
    e2e_t, e2e_k = [], []
    eev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    eev[0].record(stream)
    eev[1].record(stream)
    torch.cuda.synchronize()
    for k in range(args.warmup + max(10, args.steps // 2)):
        F.profile_events(*eev)        # the periodogram kernel's device time inside the call
        t0 = time.perf_counter()
        zz, top = F.periodogram(th, yh, sh, bh, fh, precision="mixed", topk=5, out=zh)
        dt = time.perf_counter() - t0
        F.profile_events(None, None)
        if k >= args.warmup:
            e2e_t.append(dt)
            e2e_k.append(eev[0].elapsed_time(eev[1]))
    e2e_value = ws * N * nf / reduce_max(statistics.median(e2e_t), ws)   # median call: host-side jitter

    if rank != 0:
        return
    peaks = measured_peaks()
    pipe = F.pipe_peaks()
    # roofline: FP32 FMA-pipe operations of the periodogram kernel against the
    # pipe's unit count x maximum SM clock (148 SMs x 128 lanes x 2032 MHz)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    peak_ops = 148 * 128 * sm_max * 1e6
    k_ms = statistics.mean(kern_ms)
    achieved = OPS_PER_TERM(p) * N * nf / (k_ms * 1e-3)
    # DRAM bytes (read + write) of one launch of this kernel at this launch
    # shape, from an ncu capture of the same command; None for shapes that
    # were not captured
    traffic = DRAM_BYTES_PER_LAUNCH.get((p, best["mixed"][0], best["mixed"][1]))
    # parity on a strided sample against the FP64 CPU oracle
    import oracle
    idx = np.unique(np.concatenate([np.arange(0, nf, nf // 200), np.asarray(top, dtype=np.int64)]))
    zr, c2, ratio = oracle.periodogram(s.t, s.y, s.sigma, s.base_freqs, s.grid.array()[idx], want_ratio=True)
    err_mixed, worst_mixed, n_excl = parity_vs_oracle(z_mixed[idx], zr, ratio, c2, 1e-5, N)
    err_64, worst_64, _ = parity_vs_oracle(z64[idx], zr, ratio, c2, 1e-10, N)
    cpu = None if args.no_cpu_baseline else cpu_baseline(s, args.cpu_sample)
    cpu_par = None if args.no_cpu_baseline else cpu_baseline_parallel(s, args.cpu_sample)
    others = {}
    if not args.no_other_workloads:
        others["batch_4096"] = bench_batch(F, peak_ops, flush)
        others["nightly_n1e5_p11"] = bench_nightly(F, peak_ops, flush)
        others["pool16_refine"] = bench_pool16(peak_ops)
        others["residual_n2000_p7_dzdf"] = bench_grad(F, peak_ops, flush)
    line = {
        "metric": METRIC,
        "value": value, "unit": "terms/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "nf": nf, "n_base": nb, "precision": "mixed",
                   "launch_shape": {"fpt": best["mixed"][0], "warps": best["mixed"][1]},
                   "l2": "flushed between steps (256 MiB write, outside the step events)"},
        "fp64": {"value": value64, "unit": "terms/s", "steps": k64,
                 "launch_shape": {"fpt": best["fp64"][0], "warps": best["fp64"][1]}},
        "mixed_over_fp64": value / value64,
        "max_rel_err_vs_oracle": {"mixed": err_mixed, "fp64": err_64, "sampled_bins": int(idx.size),
                                  "excluded_cond_above_1e12": n_excl,
                                  "worst_over_bound": {"mixed": worst_mixed, "fp64": worst_64},
                                  "floor": "1e-3 of the highest sampled z",
                                  "bound": "tol max(z*, floor) + 8 eps64 sqrt(N) chi2_base / ratio^2"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "T FP32-FMA-pipe ops/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "pgram_kernel + pgram_tail_kernel<mixed, P=7> (whole waves, then the tail split)",
                     "kernel_ms": k_ms,
                     "ops_per_term": OPS_PER_TERM(p),
                     "peak_source": f"148 SMs x 128 FP32 lanes x {sm_max:.0f} MHz (unit counts x max clock)",
                     "measured_pipe_rates": {k: v / 1e12 for k, v in pipe.items()}},
        "cpu_baseline": cpu,
        "cpu_baseline_parallel": cpu_par,
        "other_workloads": others,
        "e2e": {"value": e2e_value, "unit": "terms/s", "h2d_bytes_per_step": int(8 * (3 * N + nb)),
                "d2h_bytes_per_step": int(8 * nf + 8 * 5)},
        "e2e_detail": {"ms_per_call_median": statistics.median(e2e_t) * 1e3, "ms_per_call_min": min(e2e_t) * 1e3,
                       "kernel_ms_median": statistics.median(e2e_k), "calls": len(e2e_t),
                       "what": "host-pointer calls: wall time per call, and the periodogram kernel's device "
                               "time inside it (page-locked inputs and z_out)"},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
