#!/usr/bin/env python
"""Benchmark: Viola-Jones AdaBoost training throughput (boosting rounds/s) on GB300.

One step = one whole training job on the 24x24 / 15,000-window workload
(5,000 faces, 10,000 non-faces, synthetic): load the windows, integral images,
all 162,336 Haar features evaluated and sorted, then 200 boosting rounds, each
a search over every feature, polarity and threshold plus the reweighting.
value = rounds of all jobs / time, with the windows already in HBM when the
timed region starts.  e2e = the same through the C ABI from host buffers
(windows copied in, stumps copied out, inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank trains its own job on its own GPU
(replicas: the method has no exchange step on one GPU); the slowest rank's
time is used.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "boosting rounds/s at 24x24, 15k samples"
STUMP_BYTES = 40
PROFILE_DIR = os.path.join(ROOT, "profiles")
SEARCH_SRC = os.path.join(ROOT, "paper_1306_1467_gb300", "csrc", "k_search.cu")
FALLBACK_HBM_GBS = 6800.0


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="paper_24x24_15k")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batch", action="store_true",
                   help="leave the batched-vs-plain comparison out of the default line")
    p.add_argument("--precision", action="store_true",
                   help="precision form: 300 rounds from log-uniform weights, search vs FP64")
    p.add_argument("--oracle-rounds", type=int, default=6,
                   help="precision form: rounds whose weight range is reported")
    p.add_argument("--batch", action="store_true",
                   help="batching form only: 64 uneven 24x24 jobs batched against the plain path")
    p.add_argument("--batch-jobs", type=int, default=64)
    p.add_argument("--batch-rounds", type=int, default=100)
    p.add_argument("--batch-n", type=int, nargs=2, default=(2000, 20000), metavar=("LO", "HI"),
                   help="batching form: range of the jobs' sample counts")
    p.add_argument("--serve", action="store_true",
                   help="serving form only: Poisson stream of training requests, continuous batching")
    p.add_argument("--serve-rate", type=float, default=4.0, help="serving form: mean arrivals per second")
    p.add_argument("--serve-seconds", type=float, default=30.0, help="serving form: arrival window")
    p.add_argument("--serve-budget-gb", type=float, default=48.0, help="serving form: HBM for sorted tables")
    p.add_argument("--serve-pool", type=int, default=16, help="serving form: distinct jobs the requests cycle over")
    p.add_argument("--serve-rounds", type=int, default=50)
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def search_source_digest() -> str:
    """SHA-256 of the plain search kernel's source: k_screen, the device pieces
    it shares with the batched kernels, and the device header."""
    csrc = os.path.dirname(SEARCH_SRC)
    src = open(SEARCH_SRC).read()
    a = src.index("template <int U>\n__global__ void __launch_bounds__")
    b = src.index("cudaError_t launch_screen(")
    shared = open(os.path.join(csrc, "k_search.cuh")).read()
    dev = open(os.path.join(csrc, "vjb_device.cuh")).read()
    return hashlib.sha256((shared + src[a:b] + dev).encode()).hexdigest()


def _traffic(workload: str = "paper_24x24_15k"):
    """DRAM bytes per search launch from the committed ncu summary of this
    workload (profiles/k_screen_<workload>.txt), if it was taken on the
    current kernel source."""
    try:
        sha = search_source_digest()
        kv = {}
        for line in open(os.path.join(PROFILE_DIR, f"k_screen_{workload}.txt")):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != sha:
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, flag in zip(names, parts[4:8]):
                    if flag.lower() in ("active", "1", "0x1"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_model() -> str:
    """The host CPU's model name (x86 `model name`, else the Arm implementer
    and part numbers), for the CPU baseline's record."""
    import platform
    info = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if info.get("model name"):
        return info["model name"]
    if "CPU implementer" in info:
        return (f"{platform.machine()} implementer {info['CPU implementer']} "
                f"part {info.get('CPU part', '?')}")
    return platform.machine() or "unknown"


def cpu_baseline(px, y, rounds: int, every: int = 1, sample_rounds: int = 2, threads: int = 0):
    """The CPU oracle as it stands, on a bounded sample of the workload: every
    `every`-th feature, its values, value orders and `sample_rounds` rounds;
    the job time is scaled to all features and `rounds` rounds.  `threads` > 0
    runs the oracle's loops on that many host threads (0: all of them)."""
    import numpy as np

    import oracle as O
    n, H, W = px.shape
    all_threads = O.num_threads()
    O.set_num_threads(threads if threads > 0 else all_threads)
    desc, _ = O.haar_enumerate(W, H)
    sub = desc[::every]
    t0 = time.perf_counter()
    ii = O.integral(px)
    vals = O.feature_values(px, sub, ii)
    order = O.sort_rows(vals)
    t1 = time.perf_counter()
    w = O.initial_weights(y)
    for _ in range(sample_rounds):
        st, s, w = O.round_step(vals, order, y, w)
    t2 = time.perf_counter()
    scale = desc.shape[0] / sub.shape[0]
    prep_s = (t1 - t0) * scale
    round_s = (t2 - t1) / sample_rounds * scale
    job_s = prep_s + rounds * round_s
    cores = O.num_threads()
    O.set_num_threads(all_threads)
    del np
    return {"value": rounds / job_s, "unit": "rounds/s", "cores": cores, "cpu": cpu_model(),
            "kind": "oracle",
            "sample": (f"{sub.shape[0]} of {desc.shape[0]} features (every {every}), all {n} windows: "
                       f"values + stable sort + {sample_rounds} FP64 rounds, scaled to all features "
                       f"and {rounds} rounds"),
            "job_s": job_s, "prep_s": prep_s, "round_s": round_s, "measured_s": t2 - t0}


def run_reference(a, ws, rank):
    if rank != 0:
        return
    from paper_1306_1467_gb300 import synth
    px, y, rounds = synth.workload(a.workload)
    for _ in range(a.warmup):
        cpu_baseline(px, y, rounds, every=32, sample_rounds=1)
    vals = [cpu_baseline(px, y, rounds, every=32, sample_rounds=1) for _ in range(a.steps)]
    v = statistics.median([x["value"] for x in vals])
    job_ms = 1000.0 * rounds / v
    measured_ms = 1000.0 * statistics.median([x["measured_s"] for x in vals])
    # a step is the bounded sample (what the run's clock sees); the metric is
    # the whole job's rate, scaled from the sample
    line = {"metric": METRIC, "value": v, "unit": "rounds/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": measured_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": a.workload, "rounds_per_job": rounds},
            "cpu_baseline": {"value": v, "unit": "rounds/s", "kind": "oracle", "cores": vals[0]["cores"],
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "rounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "job_ms_extrapolated": job_ms,
            "note": ("a step is the sample named in cpu_baseline.sample (ms_per_step is its measured "
                     "time); value scales it to the whole job, whose time is job_ms_extrapolated")}
    print(json.dumps(line), flush=True)


def replica_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s job: replicas train independent jobs."""
    return seed + 1000 * rank


def slowest_rank_ms(times_ms, dist, device):
    """Element-wise max over ranks of a list of timed-region durations (ms)."""
    if dist is None:
        return [float(t) for t in times_ms]
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world: int, steps: int, rounds: int, ms: float) -> float:
    """Rounds of every rank's jobs per second of the slowest rank's timed region."""
    return world * steps * rounds / (ms / 1000.0)


def run_ours(a, ws, rank, local):
    import numpy as np
    import torch

    from paper_1306_1467_gb300 import synth, vjb

    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(synth.WORKLOADS[a.workload])
    rounds = cfg.pop("rounds")
    cfg["seed"] = replica_seed(cfg["seed"], rank)
    px, y = synth.make_windows(**cfg)
    n, H, W = px.shape
    stream = torch.cuda.Stream(device=dev)
    d_px = torch.from_numpy(px).to(dev)
    d_y = torch.from_numpy(y).to(dev)
    torch.cuda.synchronize()
    tr = vjb.Trainer(local, stream=stream.cuda_stream)

    def job(host: bool):
        if host:
            tr.load_windows(px, y)
        else:
            tr.load_windows(d_px, d_y)
        tr.build_integral()
        nf = tr.feature_count()
        st, stumps = tr.train_strong(rounds)
        assert st == vjb.OK and len(stumps) == rounds, (st, len(stumps))
        return nf, stumps

    for _ in range(max(a.warmup, 1)):
        nf, _ = job(False)
    info0 = tr.info()
    tr.set_timing(False)  # value: no per-round timing events in the timed region
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        pass
    clocks = Clocks(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        job(False)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    info1 = tr.info()
    launches = info1["launches"] - info0["launches"]

    # roofline: a second pass of the same jobs with CUDA events around every
    # search launch (a round then replays as two graphs with the events between)
    tr.set_timing(True)
    for _ in range(a.steps):
        job(False)
    tm = tr.timing()
    tr.set_timing(False)

    # setup vs rounds split of one job (extra run, untimed for `value`)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s2 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    tr.load_windows(d_px, d_y)
    tr.build_integral()
    tr.feature_count()
    s1.record(stream)
    tr.train_strong(rounds)
    s2.record(stream)
    s2.synchronize()
    setup_ms, rounds_ms = s0.elapsed_time(s1), s1.elapsed_time(s2)

    e2e = None
    if not a.no_e2e:
        job(True)  # warm the host path
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        h0.record(stream)
        t_host = time.perf_counter()
        for _ in range(a.steps):
            job(True)
        h1.record(stream)
        h1.synchronize()
        host_s = time.perf_counter() - t_host
        e2e_ms = max(h0.elapsed_time(h1), 1000.0 * host_s)
        e2e = {"value": None, "unit": "rounds/s", "h2d_bytes_per_step": int(px.nbytes + y.nbytes),
               "d2h_bytes_per_step": int(rounds * STUMP_BYTES), "ms_per_step": e2e_ms / a.steps,
               "_ms": e2e_ms}

    ms, e2e_ms = slowest_rank_ms([ms, e2e["_ms"] if e2e else 0.0], dist, dev)
    value = whole_job_rate(ws, a.steps, rounds, ms)
    if e2e:
        e2e.pop("_ms")
        e2e["value"] = whole_job_rate(ws, a.steps, rounds, e2e_ms)

    search_bytes = 2.0 * nf * n
    avg_search_ms = tm["search_ms_total"] / max(tm["rounds"], 1)
    achieved = search_bytes / (avg_search_ms / 1000.0) / 1e9
    peak, peak_src = _peak()
    traffic = _traffic(a.workload)
    line = {
        "metric": METRIC, "value": value, "unit": "rounds/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": a.workload, "window": f"{W}x{H}", "samples": n,
                   "positives": int(y.sum()), "negatives": int(n - y.sum()), "features": nf,
                   "rounds_per_step": rounds,
                   "step": "load windows + integral images + feature values + sort + rounds",
                   "l2": f"inputs larger than L2: the {search_bytes / 1e9:.2f} GB sorted table is read every round",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "search_shape": {"warps": info1["kernel_warps"], "stages": info1["kernel_stages"],
                                    "ctas": info1["kernel_ctas"]}},
        "roofline": {"kernel": "k_screen", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_source": f"{peak_src} hbm_gbs", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": search_bytes,
                     "avg_launch_ms": avg_search_ms, "min_launch_ms": tm["search_ms_min"],
                     "max_launch_ms": tm["search_ms_max"], "launches_timed": tm["rounds"],
                     "timed": "a second pass of the same jobs with per-launch events"},
        "gpu_launches": int(launches),
        "rounds_only_per_s": 1000.0 * rounds / rounds_ms,
        "setup_ms": setup_ms,
        # a round's share of the timed step (no per-round events), and as the
        # second pass's events saw it
        "round_ms": (ms / a.steps - setup_ms) / rounds,
        "round_ms_with_events": tm["round_ms_total"] / max(tm["rounds"], 1),
    }
    if e2e:
        line["e2e"] = e2e
    if ck:
        line["clocks"] = ck
    if ws == 1 and rank == 0 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(px, y, rounds)
        one = cpu_baseline(px, y, rounds, every=16, sample_rounds=2, threads=1)
        line["cpu_baseline"]["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample", "job_s",
                                                                      "prep_s", "round_s", "measured_s")}
    tr.close()
    del d_px, d_y
    if ws == 1 and rank == 0 and not a.no_batch:
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        line["batched"] = batch_comparison(a, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    del np


def run_precision_report(a):
    """Precision form on the 24x24 / 15k shape: weights drawn log-uniformly in
    [1e-12, 1], then 300 rounds.  Per round (the library's own diagnostics):
    the compensated-FP32 search error of the chosen stump and its FP32
    screened error against the FP64 error of that stump, the shortlist size;
    on a few rounds the weights' dynamic range.  The chosen stumps against
    the full FP64 oracle on the same weights are checked by
    tests/precision_form.py, outside the benchmark."""
    import numpy as np

    from paper_1306_1467_gb300 import synth, vjb

    px, y, rounds = synth.workload("precision_24x24_15k")
    n = px.shape[0]
    tr = vjb.Trainer(0)
    tr.prepare(px, y)
    tr.set_weights(synth.log_uniform_weights(n, seed=1308))
    check_at = sorted(set(np.linspace(0, rounds - 1, max(a.oracle_rounds, 1)).astype(int).tolist()))
    stumps, ranges = [], []
    status = vjb.OK
    while len(stumps) < rounds and status == vjb.OK:
        r = len(stumps)
        if r in check_at:
            w = tr.get_weights().astype(np.float64)
            ranges.append({"round": r, "max_over_min": float(w.max() / w[w > 0].min())})
        nxt = min([c for c in check_at if c > r] + [rounds])
        status, st = tr.train_strong(nxt - r)
        stumps.extend(st)
    diag = tr.round_diag(0, len(stumps))
    e64 = np.array([s["error"] for s in stumps])
    es = np.array([d["search_error"] for d in diag])
    ef = np.array([d["screen_error"] for d in diag], np.float64)
    cand = np.array([d["candidates"] for d in diag])
    dev_s = np.abs(es - e64) / e64
    dev_f = np.abs(ef - e64) / e64
    q = lambda x: {"max": float(x.max()), "median": float(np.median(x)), "p99": float(np.quantile(x, 0.99))}  # noqa: E731
    line = {"metric": "precision form: per-round weighted-error deviation against FP64",
            "workload": "precision_24x24_15k (24x24, 15,000 windows, weights log-uniform in [1e-12, 1])",
            "rounds": len(stumps), "status": int(status),
            "compensated_fp32_search_vs_fp64": q(dev_s),
            "fp32_screen_vs_fp64": q(dev_f),
            "shortlist_size": {"max": int(cand.max()), "median": float(np.median(cand))},
            "eps_range": [float(e64.min()), float(e64.max())],
            "weight_dynamic_range": ranges,
            "oracle_checks": "python tests/precision_form.py"}
    tr.close()
    print(json.dumps(line), flush=True)


def _make_job(shape):
    """Windows and labels of one batching job (runs in a worker process)."""
    from paper_1306_1467_gb300 import synth
    p, q, h, w, sd = shape
    return synth.make_windows(p, q, h, w, seed=sd)


def batch_comparison(a, device: int = 0) -> dict:
    """Batching form: `--batch-jobs` independent 24x24 jobs (N uniform in
    2,000..20,000, positive fraction 0.2..0.5), `--batch-rounds` rounds each,
    trained (1) one after another through the plain path and (2) together in
    one batch (one launch of each round kernel per round for all jobs, CUDA
    graph, launch shape from the batch autotuner).  Both arms are timed on
    the device over their rounds only (the one-time sort of each job is the
    same work in both), with no per-round timing events; the batched search's
    roofline comes from a few extra-timed rounds.  Reports both throughputs,
    the speedup and whether every job's stumps are identical in the two."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import torch

    from paper_1306_1467_gb300 import synth, vjb

    shapes = synth.batch_jobs(a.batch_jobs, seed=1309, n_lo=a.batch_n[0], n_hi=a.batch_n[1])
    t_gen = time.perf_counter()
    # the host generator costs about 0.4 s per job: draw the jobs in worker
    # processes started with spawn (this process already holds a CUDA context)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_make_job, shapes))
    gen_s = time.perf_counter() - t_gen
    R = a.batch_rounds
    nf = None
    byts = []
    stream = torch.cuda.Stream(device=device)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # (1) plain: one context, the jobs one after another; each job's rounds
    # timed on the device
    plain_ms, plain_stumps = 0.0, []
    with vjb.Trainer(device, stream=stream.cuda_stream) as tr:
        for px, y in data:
            nf = tr.prepare(px, y).shape[0]
            byts.append(2.0 * nf * px.shape[0])
            e0, e1 = ev(), ev()
            e0.record(stream)
            st, stumps = tr.train_strong(R)
            e1.record(stream)
            e1.synchronize()
            plain_ms += e0.elapsed_time(e1)
            plain_stumps.append(stumps)
    torch.cuda.synchronize(device)
    # (2) batched
    budget = sum(vjb.Batch.table_bytes(px.shape[0], px.shape[1], px.shape[2]) for px, _ in data)
    t0 = time.perf_counter()
    b = vjb.Batch(budget, device=device, stream=stream.cuda_stream)
    ids = [b.add_job(px, y, R) for px, y in data]
    setup_s = time.perf_counter() - t0
    tuned = b.autotune(trial_rounds=2)
    b_trials = b.trials
    info = b.info()
    # a few rounds with events around every batched search (the roofline)
    b.set_timing(True)
    roof_rounds = b.train(min(4, max(R - tuned - 1, 0)))
    tm = b.timing()
    b.set_timing(False)
    # the rest, no per-round events: job-rounds per second of device time
    done0 = sum(b.job_state(j)[0] for j in ids)
    e0, e1 = ev(), ev()
    e0.record(stream)
    rest = b.train()
    e1.record(stream)
    e1.synchronize()
    batch_ms = e0.elapsed_time(e1)
    job_rounds = sum(b.job_state(j)[0] for j in ids) - done0
    equal = sum(b.stumps(j) == ps for j, ps in zip(ids, plain_stumps))
    b.close()
    peak, peak_src = _peak()
    round_bytes = sum(byts)
    plain_rps = len(data) * R / (plain_ms / 1000.0)
    batch_rps = job_rounds / (batch_ms / 1000.0) if rest else 0.0
    search_ms = tm["search_ms_total"] / max(tm["rounds"], 1)
    search_gbs = round_bytes / (search_ms / 1000.0) / 1e9 if tm["rounds"] else 0.0
    return {"workload": f"{len(data)} jobs, 24x24, N uniform {a.batch_n[0]}-{a.batch_n[1]} "
                        f"(sum {sum(p + q for p, q, *_ in shapes)}), "
                        f"positive fraction 0.2-0.5, {R} rounds each, seed 1309",
            "features_per_job": nf, "table_bytes": budget, "host_generation_s": gen_s,
            "timed": "rounds only, CUDA events on the device, no per-round events",
            "plain": {"job_rounds_per_s": plain_rps, "ms_rounds_total": plain_ms,
                      "gbs": round_bytes * R / (plain_ms / 1000.0) / 1e9},
            "batched": {"job_rounds_per_s": batch_rps, "batch_round_ms": batch_ms / max(rest, 1),
                        "gbs": round_bytes * rest / (batch_ms / 1000.0) / 1e9, "rounds_timed": rest,
                        "job_rounds_timed": job_rounds, "autotune_rounds": tuned, "roofline_rounds": roof_rounds,
                        "shape": {**{k: info[k] for k in ("warps", "stages", "unroll", "box_lines")},
                                  "schedule": {-1: "partitioned", -2: "interleaved"}.get(
                                      info["rows_per_warp"], f"work queue, {info['rows_per_warp']} rows per warp and item")},
                        "setup_s": setup_s, "launches_per_round": 6},
            "roofline": {"kernel": "k_bscreen", "bound": "hbm", "achieved": search_gbs, "peak": peak,
                         "peak_source": f"{peak_src} hbm_gbs", "unit": "GB/s", "frac": search_gbs / peak,
                         "algorithmic_bytes_per_launch": round_bytes, "avg_launch_ms": search_ms,
                         "min_launch_ms": tm["search_ms_min"], "max_launch_ms": tm["search_ms_max"],
                         "launches_timed": tm["rounds"],
                         "round_ms_with_events": tm["round_ms_total"] / max(tm["rounds"], 1)},
            "autotune_trials": b_trials,
            "speedup": batch_rps / plain_rps,
            "identical_jobs": f"{equal}/{len(data)}"}


def serve_report(a, device: int = 0) -> dict:
    """Serving form: training requests arrive as a Poisson stream (`--serve-rate`
    per second for `--serve-seconds`); each is a job of N uniform in
    2,000..20,000 windows (positive fraction 0.2..0.5) at 24x24, or 20x20 for
    1 in 4 and 32x32 for 1 in 8 of them, trained to `--serve-rounds` rounds.
    The library's server admits requests against a fixed HBM budget for the
    sorted tables and trains the admitted ones together (continuous
    batching).  Requests cycle over a pool of distinct jobs whose results alone
    (plain path) are computed first; every served result is compared with its
    job's result alone."""
    import numpy as np

    from paper_1306_1467_gb300 import synth, vjb

    rng = np.random.Generator(np.random.PCG64(1310))
    pool = []
    for k in range(a.serve_pool):
        u = rng.uniform()
        hw = 32 if u < 0.125 else (20 if u < 0.375 else 24)
        n = int(rng.integers(2000, 20001))
        n_pos = max(1, min(n - 1, int(round(rng.uniform(0.2, 0.5) * n))))
        pool.append(synth.make_windows(n_pos, n - n_pos, hw, hw, seed=1310 * 1000 + k))
    R = a.serve_rounds
    alone = []
    with vjb.Trainer(device) as tr:
        for px, y in pool:
            tr.prepare(px, y)
            st, stumps = tr.train_strong(R)
            alone.append((st, stumps, tr.get_weights()))
    # arrival times
    t, arrivals = 0.0, []
    while True:
        t += rng.exponential(1.0 / a.serve_rate)
        if t > a.serve_seconds:
            break
        arrivals.append(t)
    budget = int(a.serve_budget_gb * 1e9)
    ids = []
    with vjb.Server(budget, max_jobs=64, device=device) as srv:
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                px, y = pool[k % len(pool)]
                ids.append((srv.submit(px, y, R), k % len(pool)))
                k += 1
            st = srv.stats()
            busy = st["queued"] + st["preparing"] + st["training"]
            if k == len(arrivals) and busy == 0:
                break
            if busy == 0:
                time.sleep(max(0.0, min(arrivals[k] - (time.perf_counter() - t0), 0.05)))
                continue
            srv.step(1)
        wall_s = time.perf_counter() - t0
        infos = [srv.request(rid) for rid, _ in ids]
        same = 0
        for (rid, j), info in zip(ids, infos):
            st, stumps, w = srv.result(rid)
            st_a, stumps_a, w_a = alone[j]
            same += int(st == st_a and stumps == stumps_a and np.array_equal(w, w_a))
        ms, jobs = srv.round_times()
        summary = srv.stats()
    lat = np.array([i["t_done_ms"] - i["t_submit_ms"] for i in infos])
    wait = np.array([i["t_admit_ms"] - i["t_submit_ms"] for i in infos])
    prep = np.array([i["t_ready_ms"] - i["t_admit_ms"] for i in infos])
    per_job_round = np.array([i["round_ms_sum"] / max(i["rounds_timed"], 1) for i in infos])
    job_round_ms = np.repeat(ms, jobs)  # the latency each job saw for each of its rounds
    q = lambda x: {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)),  # noqa: E731
                   "mean": float(np.mean(x)), "max": float(np.max(x))}
    span_s = (max(i["t_done_ms"] for i in infos) - min(i["t_submit_ms"] for i in infos)) / 1000.0
    return {"workload": (f"Poisson arrivals, mean {a.serve_rate}/s over {a.serve_seconds} s ({len(ids)} requests); "
                         f"jobs of N uniform 2,000-20,000, positive fraction 0.2-0.5, 24x24 (20x20 for 1 in 4, "
                         f"32x32 for 1 in 8), {R} rounds; requests cycle over {len(pool)} distinct jobs, seed 1310"),
            "table_budget_bytes": budget, "max_jobs": 64,
            "requests": len(ids), "identical_to_alone": f"{same}/{len(ids)}",
            "job_rounds": int(summary["job_rounds"]), "batched_rounds": int(summary["rounds"]),
            "job_rounds_per_s": summary["job_rounds"] / span_s, "span_s": span_s, "wall_s": wall_s,
            "gpu_round_busy_frac": float(ms.sum()) / 1000.0 / span_s,
            "latency_ms": {"per_job": q(lat), "admission_wait": q(wait), "preparation": q(prep),
                           "per_round": q(job_round_ms), "batched_round": q(ms),
                           "per_job_mean_round": q(per_job_round)},
            "jobs_per_round": {"mean": float(jobs.mean()), "max": int(jobs.max())}}


def main():
    a = _args()
    ws, rank, local = _dist()
    if a.precision:
        run_precision_report(a)
        return
    if a.batch:
        print(json.dumps({"metric": "batching form: batched vs plain on one GPU", **batch_comparison(a, local)}),
              flush=True)
        return
    if a.serve:
        print(json.dumps({"metric": "serving form: continuous batching of training requests", **serve_report(a, local)}),
              flush=True)
        return
    if a.impl == "reference":
        run_reference(a, ws, rank)
    else:
        run_ours(a, ws, rank, local)


if __name__ == "__main__":
    main()
