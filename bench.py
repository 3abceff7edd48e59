"""Benchmark of the PLUGIN hot path: psi6 + psi4 pair evaluations per second.

A step is one whole PLUGIN run (Algorithm 1, Steps I-VII) through the C ABI on
each of the three large samples: n = 2^20 values of Student-t3 (seed 3),
lognormal(0,1) (seed 4) and U[0,1] (seed 5), seeded and synthetic.  Per sample:
moments, psi6(g1) over n(n-1)/2 unique pairs, g2, psi4(g2) over n(n-1)/2 pairs,
h.  Pairs in far tile pairs (every term below 1e-31 of the diagonal) are skipped
by the kernels and are not counted as evaluated.

  value     FP32 pair path, inputs resident in HBM, device time per step (CUDA
            events on the launching stream); L2 flushed between steps.
  e2e       same metric through the same call with pinned HOST input and a host
            result struct per sample: H2D copy, all kernels, D2H copy, synchronize.
  roofline  the r = 6 pair kernel (Step IV), timed live by events recorded around it
            inside the captured graphs, against the ALU bound of its algorithmic
            per-pair sequence: FADD, FMUL, 3 FFMA (He_6 Horner), MUFU ex2, FFMA =
            7 issue slots (6 for He_4), i.e. SMs x clock x min(128/7, MUFU rate).
  accuracy  psi6, psi4 and h of every sample against the oracle's stored values
            (tests/golden/plugin_large_n1048576.txt), FP32 and FP64 paths.
  fp64      the all-binary64 GPU path on the same three samples.
  batch     512 samples, n log-uniform in [256, 262144], one batched call (FP32 and
            FP64), errors against the stored oracle values for the samples that
            have them.
  serving   requests of the seeded served stream (n log-uniform in [1000,
            4194304]), Poisson arrivals at given fractions of the measured FP32
            capacity, replayed through the continuous-batching server: p50/p99.
  bimodal   the n = 65536 bimodal sample offset by 1e4: FP32, FP64, Q32.32.
  kde_eval  the density estimate of Eq. 1 for n = 2^20 values at 2^14 points.
  cpu_baseline  the CPU oracle on this host's cores on a bounded sample.

`--impl reference` times the CPU oracle instead (the reference arm).
Under torchrun (N > 1) every rank runs the workload on its own GPU (replicas);
value is the sum over ranks and the time the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "psi4+psi6 pair-evals/s"
UNIT = "pair-evals/s"
FAMILIES = ("t3", "lognormal", "uniform")
N_LARGE = 1 << 20
WORKLOAD = "plugin-n1048576-t3+lognormal+uniform"
REF_N = 65536          # reference arm: oracle on the first REF_N values of each sample
CPU_N = 98304          # cpu_baseline: oracle on the first CPU_N values of each sample
RESULT_FIELDS = ("psi6", "psi4", "h")

# Issue slots per pair of the binary32 kernel's factorised sequence (segments
# whose rows and columns are narrow, >99.8% of the evaluated pairs here): FADD u,
# He_r straight from u in t = u^2 - (r - 1) (r/2 FFMA), 2 FFMA for the 3-term
# coupling factor (1 for the 2-term one, one slot less), FFMA accumulate, 4/16 for
# one Kahan step per 16 terms, and one LDS.128 of column factors per column shared
# by 4 rows.
OWN_SLOTS = {6: 7.0 + 0.25 + 0.25, 4: 6.0 + 0.25 + 0.25}
# The algorithmic per-pair sequence the roofline counts (one MUFU ex2 per pair).
ALGO_SLOTS = {6: 7.0, 4: 6.0}
KERNEL_SOURCE = os.path.join(ROOT, "paper_1505_02100_gb300", "csrc", "kde_kernels.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pairs_kernel_r6_t3_n1048576.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-n", type=int, default=REF_N,
                    help="reference arm: values of each sample the oracle takes per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-sample batch leg")
    ap.add_argument("--no-eval", action="store_true", help="skip the density-estimate leg")
    ap.add_argument("--no-bimodal", action="store_true", help="skip the n = 65536 bimodal leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the tile autotuner (built-in rule or KDE_FP32_TILE_CONFIG)")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="requests of the served stream to replay (0: skip the serving leg)")
    ap.add_argument("--serve-loads", type=str, default="0.8",
                    help="comma-separated arrival rates as fractions of the measured FP32 capacity")
    ap.add_argument("--serve-fp64", choices=["no", "also", "only"], default="no",
                    help="the FP64 subset (requests with n <= 65536 plus 20 random ones): "
                         "also, or only (without the FP32 replays)")
    ap.add_argument("--serve-fp64-random", type=int, default=20,
                    help="random requests with n > 65536 added to the FP64 subset")
    ap.add_argument("--out-json", type=str, default=None, help="also write the JSON line here")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def dist_max(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def large_samples():
    import synthdata
    return {fam: synthdata.large_sample(fam) for fam in FAMILIES}


def golden(kind: str) -> dict:
    """Oracle values stored by tests/golden/make_golden.py (written by the oracle only)."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_golden
    try:
        return make_golden.load(kind)
    except OSError:
        return {}


def rel_errors(res, ref):
    return {f: abs(res[f] - ref[f]) / abs(ref[f]) for f in RESULT_FIELDS}


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join(os.environ.get("KDE_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"kde_bench_clocks_gpu{gpu}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            c = [v.strip() for v in line.split(",")]
            if len(c) >= 9 and c[1].isdigit():
                rows.append(c)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        mx = max(int(r[2]) for r in rows)
        loaded = [v for v in sm if v > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def measured_traffic(tile_config: int):
    """DRAM bytes per launch of the r = 6 pair kernel on the t3 sample from the
    committed ncu summary, or None when the kernel source or its tile configuration
    differ from the ones those counters were taken with."""
    import hashlib
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    fields = dict(re.findall(r"^- (kernel_source_sha256|dram_bytes_per_launch_cfg\d+): `([^`]+)`",
                             text, re.M))
    digest = hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest()
    key = f"dram_bytes_per_launch_cfg{tile_config}"
    if fields.get("kernel_source_sha256") != digest or key not in fields:
        return None
    return float(fields[key])


def run_plugin_steps(kde, torch, xs, outs, prec, stream, flush, steps, warmup, ws):
    """`steps` timed steps (after `warmup`), each one kde_plugin_h per sample with the
    profiling events on; returns per-step ms and per-run kernel ms / skip counts."""
    kde.kde_profile_enable(True)
    for _ in range(warmup):
        for x, o in zip(xs, outs):
            kde.kde_plugin_h(x, prec, out=o, stream=stream)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    prof = []
    barrier(ws)
    torch.cuda.synchronize()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        runs = []
        for x, o in zip(xs, outs):
            kde.kde_plugin_h(x, prec, out=o, stream=stream)
            runs.append(kde.kde_profile_last(stream))
        ev[i][1].record(stream)
        prof.append(runs)
    torch.cuda.synchronize()
    barrier(ws)
    kde.kde_profile_enable(False)
    return [a.elapsed_time(b) for a, b in ev], prof


def result_from(kde, out):
    import numpy as np
    v = out.cpu().numpy()
    d = {f: float(v[i]) for i, f in enumerate(kde.RESULT_FIELDS)}
    d["status"] = int(v[len(kde.RESULT_FIELDS):].view(np.int32)[0])
    return d


def batch_leg(kde, torch, dev, stream, flush, with_fp64: bool, steps: int = 2, warmup: int = 1):
    """512 samples, n log-uniform in [256, 262144] (normal, mixture or t3 each), one
    kde_plugin_h_batch call per step, input resident on the device; FP32 timed by
    events, FP64 by the in-graph kernel events of one run; errors against the stored
    oracle values (samples with n <= 65536, and larger ones where stored)."""
    import numpy as np

    import synthdata
    specs = synthdata.batch_specs()
    xs = [synthdata.sample_from_spec(s) for s in specs]
    ns = np.array([x.size for x in xs], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(ns)])
    xd = torch.tensor(np.concatenate(xs), dtype=torch.float64, device=dev)
    m = len(xs)
    pairs = int((ns * (ns - 1)).sum())          # psi6 + psi4: 2 x n(n-1)/2 per sample
    out = torch.empty(m * kde.RESULT_BYTES // 8, dtype=torch.float64, device=dev)
    gold = golden("batch")

    def results():
        res = out.cpu().numpy().reshape(m, kde.RESULT_BYTES // 8)
        st = res.view(np.int32)[:, 16]
        return res, st

    def errors(res):
        errs = {f: [] for f in RESULT_FIELDS}
        for k, spec in enumerate(specs):
            ref = gold.get(str(spec.index))
            if ref is None:
                continue
            for i, f in enumerate(kde.RESULT_FIELDS):
                if f in RESULT_FIELDS:
                    errs[f].append(abs(res[k, i] - ref[f]) / abs(ref[f]))
        return {f: {"max": float(np.max(v)), "median": float(np.median(v)), "samples": len(v)}
                for f, v in errs.items() if v}

    kde.kde_profile_enable(True)
    for _ in range(warmup):
        kde.kde_plugin_h_batch(xd, off, kde.KDE_FP32, out=out, stream=stream)
    prof = kde.kde_profile_last(stream)
    kde.kde_profile_enable(False)
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kde.kde_plugin_h_batch(xd, off, kde.KDE_FP32, out=out, stream=stream)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
    res, st = results()
    t = statistics.mean(ms) / 1e3
    skipped = prof["skipped6"] + prof["skipped4"]   # far tile pairs, not evaluated
    leg = {"samples": m, "n_total": int(ns.sum()), "pair_evals": pairs - skipped,
           "pairs_skipped": skipped, "ms": 1e3 * t,
           "pair_evals_per_s": (pairs - skipped) / t, "bandwidths_per_s": m / t,
           "status_ok": int((st == 0).sum()), "steps": steps,
           "input": "device-resident binary64, L2 flushed before each step",
           "rel_err_vs_oracle": errors(res)}
    if with_fp64:
        kde.kde_profile_enable(True)
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kde.kde_plugin_h_batch(xd, off, kde.KDE_FP64, out=out, stream=stream)
        e1.record(stream)
        p64 = kde.kde_profile_last(stream)
        stream.synchronize()
        kde.kde_profile_enable(False)
        # device time of the kernels (the first call on a plan also captures its graph)
        dev_ms = p64["setup"] + p64["pairs6"] + p64["prescale4"] + p64["pairs4"]
        sk64 = p64["skipped6"] + p64["skipped4"]
        res64, st64 = results()
        leg["fp64"] = {"ms": dev_ms, "pair_evals_per_s": (pairs - sk64) / (dev_ms / 1e3),
                       "pairs_skipped": sk64, "status_ok": int((st64 == 0).sum()),
                       "rel_err_vs_oracle": errors(res64),
                       "timing": "sum of the in-graph kernel events of one run (setup, pairs6, "
                                 "prescale, pairs4)"}
        leg["fp32_over_fp64"] = leg["pair_evals_per_s"] / leg["fp64"]["pair_evals_per_s"]
    return leg


def eval_leg(kde, torch, dev, stream, flush, steps: int = 3, warmup: int = 1):
    """Density estimate (Eq. 1) of n = 2^20 normal values at m = 2^14 grid points with
    the sample's own plug-in bandwidth, inputs resident on the device, FP32 path."""
    import numpy as np

    import synthdata
    n, m = 1 << 20, 1 << 14
    x = synthdata.normal(31, n) * 1.7 + 4.0
    h = kde.kde_plugin_h(x, kde.KDE_FP32)["h"]
    t = np.linspace(x.min(), x.max(), m)
    xd = torch.tensor(x, dtype=torch.float64, device=dev)
    td = torch.tensor(t, dtype=torch.float64, device=dev)
    out = torch.empty(m, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        kde.kde_eval(xd, h, td, kde.KDE_FP32, out=out, stream=stream)
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kde.kde_eval(xd, h, td, kde.KDE_FP32, out=out, stream=stream)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
    t_s = statistics.mean(ms) / 1e3
    return {"n": n, "m": m, "h": h, "ms": 1e3 * t_s, "pair_evals_per_s": n * m / t_s,
            "values": out.cpu().numpy(), "x": x, "t": t,
            "includes": "copy of x and t into the workspace, sort of x, prescale, pairs, reduce"}


def serve_replay(kde, specs, xs, arrivals, prec):
    """Replay requests in real time through one server; per-request latency, queueing
    and evaluated pairs."""
    with kde.Server(hbm_budget_bytes=24 << 30, max_inflight=256) as srv:
        t0 = time.perf_counter()
        tickets = []
        for k, x in enumerate(xs):
            wait = t0 + arrivals[k] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit(x, prec))
        return [srv.poll(t, timeout_ms=3600000) for t in tickets]


def serve_summary(got, xs, gold=None, keys=None):
    import numpy as np
    lat, queue, ok, pairs, skipped = [], [], 0, 0, 0
    errs = {f: [] for f in RESULT_FIELDS}
    for k, ((res, tm), x) in enumerate(zip(got, xs)):
        ok += int(res["status"] == 0)
        lat.append((tm["t_done_ns"] - tm["t_submit_ns"]) / 1e6)
        queue.append((tm["t_admit_ns"] - tm["t_submit_ns"]) / 1e6)
        pairs += x.size * (x.size - 1)
        skipped += tm["skipped6"] + tm["skipped4"]
        if gold is not None and keys[k] in gold and res["status"] == 0:
            for f in RESULT_FIELDS:
                errs[f].append(abs(res[f] - gold[keys[k]][f]) / abs(gold[keys[k]][f]))
    span = (max(tm["t_done_ns"] for _, tm in got) - min(tm["t_submit_ns"] for _, tm in got)) / 1e9
    out = {"requests": len(got), "status_ok": ok,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(max(lat))},
           "admit_wait_ms_p50": float(np.percentile(queue, 50)),
           "pair_evals": pairs - skipped, "pairs_skipped": skipped,
           "pair_evals_per_s": (pairs - skipped) / span, "span_s": span}
    if gold is not None:
        out["rel_err_vs_oracle"] = {f: {"max": float(np.max(v)), "median": float(np.median(v)),
                                        "requests": len(v)} for f, v in errs.items() if v}
    return out


def serve_leg(kde, capacity: float, count: int, loads, fp64_mode: str, out_prefix=None,
              fp64_random: int = 20):
    """The first `count` requests of the served stream (n log-uniform in [1000, 4194304],
    FP32 samples, Poisson arrivals at `load` x the measured FP32 capacity), replayed in
    real time through the continuous-batching server, once per load (FP32 path).
    fp64_mode "also" / "only": the FP64 subset as well / alone -- the requests with
    n <= 65536 plus `fp64_random` random ones, arriving at the first load's arrival times, served
    in FP64; its FP32 figures are those requests' figures from the FP32 replay at that
    load.  With `out_prefix`, every replay's summary and per-request records are written
    as soon as it ends."""
    import numpy as np

    import synthdata
    specs = synthdata.server_specs()[:count]
    xs = [synthdata.sample_from_spec(s, np.float32) for s in specs]
    keys = [str(s.index) for s in specs]
    lo, hi = 1000.0, 4194304.0
    e_pairs = (hi * hi - lo * lo) / (2.0 * math.log(hi / lo))     # E[n^2] ~ E[n(n-1)], log-uniform n
    gold = golden("serve")
    out = {"sample": f"first {count} of the seeded 10000-request stream", "fp32": {}}

    def dump(tag, summary, got, idx):
        if not out_prefix:
            return
        with open(f"{out_prefix}.{tag}.json", "w") as f:
            json.dump({"summary": summary,
                       "requests": [{"index": int(specs[k].index), "n": int(specs[k].n),
                                     "latency_ms": (tm["t_done_ns"] - tm["t_submit_ns"]) / 1e6,
                                     "status": int(res["status"]), "h": res["h"], "psi6": res["psi6"],
                                     "psi4": res["psi4"], "skipped": int(tm["skipped6"] + tm["skipped4"])}
                                    for k, (res, tm) in zip(idx, got)]}, f)

    first = {}
    for load in loads:
        rate = load * capacity / e_pairs
        arrivals = synthdata.poisson_arrivals(count, rate)
        if fp64_mode == "only":
            if load == loads[0]:
                first = {"got": None, "arrivals": arrivals, "rate": rate}
            continue
        got = serve_replay(kde, specs, xs, arrivals, kde.KDE_FP32)
        s = serve_summary(got, xs, gold, keys)
        s.update({"load": load, "arrival_rate_per_s": rate})
        out["fp32"][f"load_{load:g}"] = s
        dump(f"fp32_load{load:g}", s, got, range(count))
        if load == loads[0]:
            first = {"got": got, "arrivals": arrivals, "rate": rate}
    if fp64_mode in ("also", "only"):
        small = [k for k, s in enumerate(specs) if s.n <= 65536]
        rng = np.random.default_rng(7)
        others = [k for k in range(len(specs)) if specs[k].n > 65536]
        extra = list(rng.choice(others, size=min(fp64_random, len(others)), replace=False)) if fp64_random > 0 else []
        pick = sorted(small + extra)
        sub_xs = [xs[k] for k in pick]
        sub_keys = [keys[k] for k in pick]
        arrivals = first["arrivals"][pick]
        arrivals = arrivals - arrivals[0]
        got64 = serve_replay(kde, [specs[k] for k in pick], sub_xs, arrivals, kde.KDE_FP64)
        s64 = serve_summary(got64, sub_xs, gold, sub_keys)
        s64.update({"load_of_arrivals": loads[0], "arrival_rate_per_s": first["rate"]})
        dump(f"fp64_subset_load{loads[0]:g}", s64, got64, pick)
        sub = {"requests": len(pick), "selection": f"n <= 65536 plus {len(extra)} random requests "
               "(numpy default_rng(7)) of the replayed stream, at their arrival times", "fp64": s64}
        if first.get("got") is not None:
            s32 = serve_summary([first["got"][k] for k in pick], sub_xs, gold, sub_keys)
            sub["fp32_same_requests_in_the_fp32_replay"] = s32
            sub["fp32_over_fp64_pair_evals_per_s"] = s32["pair_evals_per_s"] / s64["pair_evals_per_s"]
        out["fp64_subset"] = sub
    return out


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle (the paper publishes no code) on the same
    three samples, each step one PLUGIN run on the first `ref_n` values of each."""
    if rank != 0:
        return
    import oracle
    ref_n = getattr(args, "ref_n", REF_N)
    xs = [x[:ref_n].copy() for x in large_samples().values()]
    cores = oracle.default_threads()
    for _ in range(args.warmup):
        for x in xs:
            oracle.plugin(x, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for x in xs:
            oracle.plugin(x, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    per_step = sum(x.size * (x.size - 1) for x in xs)
    value = args.steps * per_step / total
    sample = (f"one full PLUGIN run per step on the first {ref_n} values of each of the three "
              f"n = 2^20 samples ({per_step} pair-evals per step, symmetric form)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_LARGE, "ref_n": ref_n,
                                        "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def bimodal_leg(kde, torch, dev, stream, flush, steps=10, warmup=3, with_fp64=True):
    """The n = 65536 bimodal sample offset by 1e4 (tests centring): FP32, FP64 and the
    paper's Q32.32 arithmetic, errors against the oracle run live on the same sample."""
    import synthdata
    n = 65536
    x = synthdata.bimodal_offset()
    xd = [torch.tensor(x, dtype=torch.float64, device=dev)]
    out = [torch.empty(kde.RESULT_BYTES // 8, dtype=torch.float64, device=dev)]
    ms, prof = run_plugin_steps(kde, torch, xd, out, kde.KDE_FP32, stream, flush, steps, warmup, 1)
    sk = sum(p[0]["skipped6"] + p[0]["skipped4"] for p in prof) / steps
    pairs = n * (n - 1)
    leg = {"n": n, "distribution": "0.5N(-1,0.5^2)+0.5N(1,0.5^2)+1e4",
           "fp32": {"pair_evals_per_s": steps * (pairs - sk) / (sum(ms) / 1e3),
                    "ms_per_step": statistics.mean(ms),
                    "pairs6_ms": statistics.mean(p[0]["pairs6"] for p in prof),
                    "pairs4_ms": statistics.mean(p[0]["pairs4"] for p in prof),
                    "setup_ms": statistics.mean(p[0]["setup"] for p in prof)}}
    res = {"fp32": kde.kde_plugin_h(xd[0], kde.KDE_FP32)}
    if with_fp64:
        ms64, prof64 = run_plugin_steps(kde, torch, xd, out, kde.KDE_FP64, stream, flush, 2, 1, 1)
        sk64 = prof64[0][0]["skipped6"] + prof64[0][0]["skipped4"]
        leg["fp64"] = {"pair_evals_per_s": 2 * (pairs - sk64) / (sum(ms64) / 1e3),
                       "ms_per_step": statistics.mean(ms64)}
        res["fp64"] = kde.kde_plugin_h(xd[0], kde.KDE_FP64)
        leg["fp32_over_fp64"] = leg["fp32"]["pair_evals_per_s"] / leg["fp64"]["pair_evals_per_s"]
        kde.kde_profile_enable(True)
        kde.kde_plugin_h(xd[0], kde.KDE_Q32, out=out[0], stream=stream)
        pq = kde.kde_profile_last(stream)
        kde.kde_profile_enable(False)
        qe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for a, b in qe:
            with torch.cuda.stream(stream):
                flush.zero_()
            a.record(stream)
            kde.kde_plugin_h(xd[0], kde.KDE_Q32, out=out[0], stream=stream)
            b.record(stream)
        stream.synchronize()
        tq = statistics.mean(a.elapsed_time(b) for a, b in qe) / 1e3
        skq = pq["skipped6"] + pq["skipped4"]
        leg["q32"] = {"pair_evals_per_s": (pairs - skq) / tq, "ms_per_step": 1e3 * tq,
                      "pairs_skipped_per_step": skq,
                      "note": "pair terms in Q32.32 fixed point on z-scored data; far tile pairs "
                              "(every term exactly 0) are skipped and not counted"}
        res["q32"] = kde.kde_plugin_h(xd[0], kde.KDE_Q32)
    return leg, res, x


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1505_02100_gb300 as kde
    from paper_1505_02100_gb300 import build as kbuild

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 and not kbuild.up_to_date():
        kbuild.build()
    barrier(ws)
    kde.load()
    tuned = None if args.no_tune else kde.kde_autotune(kde.KDE_FP32)   # per size class, this device
    samples = large_samples()
    xs_host = list(samples.values())
    xd = [torch.tensor(x, dtype=torch.float64, device=dev) for x in xs_host]
    outs = [torch.empty(kde.RESULT_BYTES // 8, dtype=torch.float64, device=dev) for _ in xs_host]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    n = N_LARGE
    pairs_one = n * (n - 1) // 2

    # FP32 pair path: the headline
    with ClockSampler(local) as clk:
        step_ms, prof = run_plugin_steps(kde, torch, xd, outs, kde.KDE_FP32, stream, flush,
                                         args.steps, args.warmup, ws)
    clocks = clk.summary()
    total_s = dist_max(sum(step_ms) / 1e3, ws)
    res32 = {fam: result_from(kde, o) for fam, o in zip(FAMILIES, outs)}
    skipped6 = [p["skipped6"] for p in prof[0]]
    skipped4 = [p["skipped4"] for p in prof[0]]
    evaluated_per_step = 2 * pairs_one * len(FAMILIES) - sum(skipped6) - sum(skipped4)
    value = ws * args.steps * evaluated_per_step / total_s
    launches = sum(p["launches"] for runs in prof for p in runs)

    # end to end through the C ABI: pinned host input, host result, synchronous
    xh = [torch.tensor(x, dtype=torch.float64).pin_memory() for x in xs_host]
    for _ in range(args.warmup):
        for x in xh:
            kde.kde_plugin_h(x, kde.KDE_FP32, stream=stream)
    e2e_t = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        for x in xh:
            r = kde.kde_plugin_h(x, kde.KDE_FP32, stream=stream)
            assert r["status"] == 0
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = dist_max(sum(e2e_t), ws)
    e2e_value = ws * args.steps * evaluated_per_step / e2e_total

    # FP64 path on the same samples: one step (kernel time from the in-graph events)
    fp64 = res64 = None
    if not args.no_fp64:
        ms64, prof64 = run_plugin_steps(kde, torch, xd, outs, kde.KDE_FP64, stream, flush, 1, 0, ws)
        res64 = {fam: result_from(kde, o) for fam, o in zip(FAMILIES, outs)}
        runs = prof64[0]
        dev_ms = sum(p["setup"] + p["pairs6"] + p["prescale4"] + p["pairs4"] for p in runs)
        ev64 = 2 * pairs_one * len(FAMILIES) - sum(p["skipped6"] + p["skipped4"] for p in runs)
        fp64 = {"value": ws * ev64 / (dist_max(dev_ms, ws) / 1e3), "unit": UNIT,
                "ms_per_step": dev_ms, "steps": 1,
                "pairs6_ms": [p["pairs6"] for p in runs], "pairs4_ms": [p["pairs4"] for p in runs],
                "timing": "sum of the in-graph kernel events of each run (one step, no warm-up: "
                          "the first replay's graph capture is host time outside them)"}

    batch = serve = evl = bim = None
    if ws == 1 and not args.no_eval:
        evl = eval_leg(kde, torch, dev, stream, flush)
    if ws == 1 and not args.no_batch:
        batch = batch_leg(kde, torch, dev, stream, flush, not args.no_fp64)
    if ws == 1 and not args.no_bimodal:
        bim = bimodal_leg(kde, torch, dev, stream, flush, with_fp64=not args.no_fp64)
    if ws == 1 and args.serve_requests > 0:
        loads = [float(v) for v in args.serve_loads.split(",") if v]
        serve = serve_leg(kde, value, args.serve_requests, loads, args.serve_fp64,
                          args.out_json[:-5] if args.out_json and args.out_json.endswith(".json") else args.out_json,
                          args.serve_fp64_random)

    if rank != 0:
        return
    with ClockSampler(local) as pclk:
        rates = kde.kde_probe_pipe_rates()
    probe_mhz = pclk.summary()["sm_mhz"] or 2070.0
    sms = int(rates["sms"])
    mufu_clk = rates["mufu_ex2_per_s_sm"] / (probe_mhz * 1e6)
    rates_clk = {"fp32_fma_lanes_per_clk_sm": rates["fp32_fma_lanes_per_s_sm"] / (probe_mhz * 1e6),
                 "mufu_ex2_per_clk_sm": mufu_clk,
                 "fp64_fma_lanes_per_clk_sm": rates["fp64_fma_lanes_per_s_sm"] / (probe_mhz * 1e6),
                 "probe_sm_mhz": probe_mhz}

    def peak(r, mhz=2070.0):
        return sms * mhz * 1e6 * min(128.0 / ALGO_SLOTS[r], mufu_clk)

    k6_ms = sum(p["pairs6"] for runs in prof for p in runs)
    k4_ms = sum(p["pairs4"] for runs in prof for p in runs)
    ev6 = args.steps * (pairs_one * len(FAMILIES) - sum(skipped6))
    ev4 = args.steps * (pairs_one * len(FAMILIES) - sum(skipped4))
    achieved6 = ev6 / (k6_ms / 1e3)
    achieved4 = ev4 / (k4_ms / 1e3)
    cfg_n = list(kde.kde_tile_config(n, kde.KDE_FP32))
    gold = golden("large")
    accuracy = {"fp32": {fam: rel_errors(res32[fam], gold[fam]) for fam in FAMILIES if fam in gold},
                "fp32_status": [res32[f]["status"] for f in FAMILIES],
                "reference": "oracle values stored by tests/golden/make_golden.py"}
    if res64:
        accuracy["fp64"] = {fam: rel_errors(res64[fam], gold[fam]) for fam in FAMILIES if fam in gold}
        accuracy["fp64_status"] = [res64[f]["status"] for f in FAMILIES]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "samples": {"t3": "seed 3", "lognormal": "seed 4",
                                                             "uniform": "seed 5"},
                   "precision": "fp32 pair terms, fp64 moments/reductions/scalars",
                   "l2": "flushed between steps (512 MiB write outside the timed events)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "tile_configs": {"tuned_per_class": tuned, "this_n": cfg_n}},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n * len(FAMILIES),
                "d2h_bytes_per_step": kde.RESULT_BYTES * len(FAMILIES)},
        "roofline": {"bound": "alu", "kernel": "pairs_kernel r=6 (Step IV)",
                     "achieved": achieved6 / 1e9, "peak": peak(6) / 1e9, "unit": "Gpair/s",
                     "frac": achieved6 / peak(6),
                     "traffic": measured_traffic(cfg_n[0]),
                     "peak_basis": (f"{sms} SMs x 2070 MHz x min(128 / {ALGO_SLOTS[6]:g} issue slots per pair, "
                                    f"measured MUFU ex2 {mufu_clk:.1f}/clk/SM): FADD, FMUL, 3 FFMA, ex2, FFMA"),
                     "pairs4_kernel": {"ms": k4_ms / args.steps, "achieved": achieved4 / 1e9,
                                       "peak": peak(4) / 1e9, "frac": achieved4 / peak(4),
                                       "peak_basis": f"min(128 / {ALGO_SLOTS[4]:g}, MUFU): FADD, FMUL, 2 FFMA, ex2, FFMA"},
                     "pairs6_ms_per_step": k6_ms / args.steps,
                     "pairs_skipped_per_step": {"r6": sum(skipped6), "r4": sum(skipped4)},
                     "frac_at_measured_clock": achieved6 / peak(6, clocks["sm_mhz"] or 2070.0),
                     "frac_vs_own_sequence": {str(r): a / (sms * 2070e6 * 128.0 / OWN_SLOTS[r])
                                              for r, a in ((6, achieved6), (4, achieved4))},
                     "own_slots_per_pair": OWN_SLOTS,
                     "probe": rates_clk},
        "clocks": clocks,
        "accuracy": accuracy,
        "per_sample": {fam: {"h": res32[fam]["h"], "pairs6_ms": statistics.mean(runs[i]["pairs6"] for runs in prof),
                             "pairs4_ms": statistics.mean(runs[i]["pairs4"] for runs in prof),
                             "setup_ms": statistics.mean(runs[i]["setup"] for runs in prof),
                             "skipped6": skipped6[i], "skipped4": skipped4[i]}
                       for i, fam in enumerate(FAMILIES)},
    }
    if fp64:
        line["fp64"] = fp64
        line["fp32_over_fp64"] = value / fp64["value"]
        # binary64 pair sequence on the factorised path: DADD u, DMUL w, 3 DFMA (He_6
        # Horner), 4 DFMA (coupling to p^4/24), 1 DFMA (accumulate); bound by the FP64 pipe
        fp64_ops = 10.0
        fp64_peak = ws * sms * 2070e6 * rates_clk["fp64_fma_lanes_per_clk_sm"] / fp64_ops   # all ranks
        line["fp64"]["roofline"] = {
            "bound": "fp64", "unit": "Gpair-evals/s", "achieved": fp64["value"] / 1e9,
            "peak": fp64_peak / 1e9, "frac": fp64["value"] / fp64_peak,
            "peak_basis": (f"{sms} SMs x 2070 MHz x measured FP64 FMA "
                           f"{rates_clk['fp64_fma_lanes_per_clk_sm']:.2f} lanes/clk/SM / {fp64_ops:g} "
                           "binary64 operations per pair (psi6 sequence; psi4 has one fewer)")}
    if batch:
        line["batch"] = batch
    if serve:
        line["serving"] = serve
    if evl:
        # issue slots per pair: 3 FADD (double-float difference), FMUL, MUFU ex2,
        # 0.75 FADD tree + 1 Kahan step per 4 terms; MUFU itself allows 32 per clock
        slots = 6.75
        eval_peak = sms * 2070e6 * min(128.0 / slots, mufu_clk)
        line["kde_eval"] = {k: v for k, v in evl.items() if k not in ("values", "x", "t")}
        line["kde_eval"]["roofline"] = {"bound": "alu", "achieved": evl["pair_evals_per_s"] / 1e9,
                                        "peak": eval_peak / 1e9, "unit": "Gpair/s",
                                        "frac": evl["pair_evals_per_s"] / eval_peak,
                                        "peak_basis": f"{sms} SMs x 2070 MHz x 128 / {slots} slots per pair"}
    if bim:
        line["bimodal_n65536"] = bim[0]
    if not args.no_cpu_baseline:
        import oracle
        cores = oracle.default_threads()
        sub = [x[:CPU_N].copy() for x in xs_host]
        t0 = time.perf_counter()
        for x in sub:
            oracle.plugin(x, threads=cores)
        dt = time.perf_counter() - t0
        per = sum(x.size * (x.size - 1) for x in sub)
        line["cpu_baseline"] = {"value": per / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one full PLUGIN run on the first {CPU_N} values of each of the "
                                          f"three n = 2^20 samples ({per} pair-evals, {dt:.1f} s)"}
        n1 = 16384
        t0 = time.perf_counter()
        oracle.plugin(sub[0][:n1], threads=1)
        dt1 = time.perf_counter() - t0
        line["cpu_baseline"]["value_1_core"] = n1 * (n1 - 1) / dt1
        line["cpu_baseline"]["sample_1_core"] = (f"one PLUGIN run on the first {n1} values of the t3 "
                                                 f"sample, one thread ({n1 * (n1 - 1)} pair-evals, {dt1:.2f} s)")
        if evl:
            pick = np.linspace(0, evl["m"] - 1, 32).astype(int)
            ref_e = oracle.kde_eval(evl["x"], evl["h"], evl["t"][pick], threads=cores)
            line["kde_eval"]["max_rel_err_vs_oracle_32_points"] = float(
                np.max(np.abs(evl["values"][pick] - ref_e) / ref_e))
        if bim:
            ref = oracle.plugin(bim[2], threads=cores)
            line["bimodal_n65536"]["rel_err_vs_oracle"] = {k: rel_errors(v, ref) for k, v in bim[1].items()}
    text = json.dumps(line)
    if args.out_json:
        with open(args.out_json, "w") as f:
            f.write(text + "\n")
    print(text)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
