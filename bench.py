#!/usr/bin/env python3
"""Throughput benchmark of OLS variable-bandwidth filtering on GB300.

Default workload (one step): 64 complex64 channels x 2^22 samples, N = 1024, overlap 256
(M = 768), L_V = 12 shared transition samples, k1 redrawn from U{32..480} every 16 blocks per
channel; the whole batch is one prepared vbw batch (one fused-kernel launch). Inputs are resident
in HBM when the timed region starts and exceed L2 (2.1 GB read + 2.1 GB written per step).

Other workloads (--workload): single (1 x 2^16, N=256; L2 flushed between steps), mixed (4096
streams of mixed length and N in one batch, replayed as a CUDA graph), precision (16384 x 2^16,
N = 256 or 512, FP32 path), serving (2000 live streams, N in {512, 1024, 2048}, open-loop
Poisson chunk arrivals through the continuous-batching server; p50/p99 latency), real (64 real
float32 channels x 2^23 samples, N = 1024, two real blocks per complex transform).

Printed JSON line:
  value        device-resident throughput (output Gsamples/s, whole job, max over ranks)
  e2e          the same through vbw_batch_run_host with pinned HOST buffers (copies timed)
  roofline     HBM roofline of the fused kernel: 16 algorithmic bytes per output sample
  cpu_baseline the FP64 oracle on a bounded sample of the same workload, on the host cores
  clocks       nvidia-smi SM clocks and throttle reasons sampled during the timed region

--impl reference times the FP64 oracle (the method's plain definition) on the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes
import gc
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered Gsamples/s at stated error vs FP64, % of HBM peak; p99 stream latency"
UNIT = "Gsamples/s"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_SAMPLE = 16          # 8 B complex64 read + 8 B complex64 written per output sample
FP32_RMS_TOL = 2e-6
L2_BYTES = 126 * 1024 * 1024

CHANNELS = dict(seed=2, nch=64, nsamples=1 << 22, N=1024, overlap=256, LV=12, every=16, lo=32, hi=480)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=["channels", "single", "mixed", "precision", "serving", "real",
                                           "ptvir", "ola"],
                    default="channels")
    ap.add_argument("--duration", type=float, default=10.0,
                    help="serving: seconds of Poisson arrivals")
    ap.add_argument("--rate", type=float, default=50_000.0, help="serving: chunks/s offered")
    ap.add_argument("--pool-mb", type=int, default=4096, help="serving: device pool (MiB)")
    ap.add_argument("--slots", type=int, default=4, help="serving: batch slots")
    ap.add_argument("--channels", type=int, default=None, help="channels / streams per GPU")
    ap.add_argument("--samples", type=int, default=None, help="samples per channel")
    ap.add_argument("--N", type=int, default=256, help="transform size of the precision workload")
    ap.add_argument("--prec", choices=["fp32", "bf16", "fp16", "bf16x6"], default="fp32",
                    help="DFT arithmetic: FP32 CUDA-core FFT, or tensor-core GEMMs with BF16 "
                         "hi+lo, scaled FP16 hi+lo, or BF16 hi+mid+lo pieces")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-mode", choices=["tuned", "per_plan", "mixed"], default="tuned",
                    help="mixed-N batches: the autotuner's launch mode, or one forced")
    ap.add_argument("--no-configs", action="store_true",
                    help="channels workload: skip the record of the other four workloads")
    return ap.parse_args()


KERNEL_SOURCES = ("ols_fp32.cuh", "fft_reg.cuh", "vbw_common.cuh")   # the fused FP32 kernel
TC_SOURCES = ("ols_tc.cuh", "tc_common.cuh") + KERNEL_SOURCES             # the tensor-core kernel
SPLIT_SOURCES = ("ols_split2048.cu", "tc_common.cuh") + KERNEL_SOURCES   # N = 2048, overlap N/4
OLA_SOURCES = KERNEL_SOURCES + ("vbw_ola.cu",)                        # the overlap-add kernel


# ---- cross-rank reductions (replicas: each rank runs its own streams; no data-path collective)

def _group_size() -> int:
    import torch.distributed as dist
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def rank_reduce(value: float, op: str, device) -> float:
    """MAX or SUM of a per-rank scalar over the process group (the value itself on one rank)."""
    if _group_size() == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_gsamples(samples_per_rank: int, steps: int, seconds_per_rank: float, device) -> float:
    """Whole-job throughput: every rank's samples over the slowest rank's time (weak scaling)."""
    slowest = rank_reduce(seconds_per_rank, "max", device)
    return samples_per_rank * _group_size() * steps / slowest / 1e9


def source_hash(files=None) -> str:
    """Hash of the sources that define a kernel (default: the fused FP32 OLS kernel); profiles
    record it."""
    h = hashlib.sha256()
    for f in (files or KERNEL_SOURCES):
        h.update(open(os.path.join(ROOT, "paper_2406_14116_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profile_traffic(kernel_tag: str, files=None, key: str = "dram_bytes_per_full_launch"):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_h = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    if not m_h or not m_t or m_h.group(1) != source_hash(files):
        return None
    return float(m_t.group(1))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# ---- clocks -----------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and self.uuid not in parts[1]:
                    continue
                rows.append(parts)
            os.remove(self.path)
        return self.summarize(rows)

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[2]) for r in rows])
        smax = np.array([num(r[3]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names, r[6:10]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        loaded = sm[sm >= 0.5 * np.nanmax(sm)] if np.isfinite(sm).any() else sm
        return {"sm_mhz": float(np.nanmedian(loaded)), "sm_max_mhz": float(np.nanmax(smax)),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": float(np.nanmax([num(r[4]) for r in rows]))}


def device_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---- workloads --------------------------------------------------------------------------------

class Stream:
    """One signal of a workload: plan geometry, per-block bands, its generator id."""

    def __init__(self, N, overlap, nsamples, band, gen):
        self.N, self.overlap, self.nsamples, self.band, self.gen = N, overlap, nsamples, band, gen


def make_streams(name, args, rank):
    """(streams, V, config, seed) of a workload; streams carry how to regenerate their samples."""
    from paper_2406_14116_gb300 import workloads as wl
    if name == "channels":
        c = CHANNELS
        nch = args.channels or c["nch"]
        T = args.samples or c["nsamples"]
        ids = [rank * nch + i for i in range(nch)]
        V = wl.transition_table(c["seed"], c["LV"])
        streams = [Stream(c["N"], c["overlap"], T,
                          wl.channels_band(c["seed"], ch, T, c["N"], c["overlap"], c["every"],
                                           c["lo"], c["hi"]), ("gauss", c["seed"], ch))
                   for ch in ids]
        cfg = {"workload": f"channels: {nch} x {T} complex64 per GPU, N={c['N']}, overlap "
                           f"{c['overlap']}, L_V={c['LV']}, k1~U{{{c['lo']}..{c['hi']}}} every "
                           f"{c['every']} blocks",
               "channels_per_gpu": nch, "samples_per_channel": T, "N": c["N"],
               "overlap": c["overlap"], "L_V": c["LV"], "seed": c["seed"]}
        return streams, V, cfg
    if name == "single":
        T = args.samples or (1 << 16)
        V = wl.transition_table(1, 6)
        nb = wl.nblocks_for(T, 256, 64)
        streams = [Stream(256, 64, T, np.full(nb, 60, np.int32), ("gauss", 1, 0))]
        cfg = {"workload": f"single: 1 x {T} complex64, N=256, overlap 64, k1=60, L_V=6",
               "N": 256, "overlap": 64, "L_V": 6, "seed": 1}
        return streams, V, cfg
    if name == "mixed":
        n = args.channels or 4096
        lengths, Nsel, ovl, k1 = wl.mixed_stream_params(3, n)
        if args.samples:
            lengths = np.minimum(lengths, args.samples)
        V = wl.transition_table(3, 12)
        streams = [Stream(int(Nsel[i]), int(ovl[i]), int(lengths[i]),
                          np.full(wl.nblocks_for(int(lengths[i]), int(Nsel[i]), int(ovl[i])),
                                  int(k1[i]), np.int32), ("tones", 3, rank * n + i))
                   for i in range(n)]
        cfg = {"workload": f"mixed: {n} streams, length floor(2^U(12,20)), N~U{{128..2048}}, "
                           f"overlap N/4, k1~U{{1..N/2-13}}, L_V=12, noise + 1-8 tones",
               "streams": n, "total_samples": int(sum(s.nsamples for s in streams)), "seed": 3}
        return streams, V, cfg
    if name == "precision":
        n = args.channels or 16384
        T = args.samples or (1 << 16)
        N = args.N
        V = wl.transition_table(4, 12)
        k1 = wl.precision_bands(4, n, N, 12)
        nb = wl.nblocks_for(T, N, N // 4)
        streams = [Stream(N, N // 4, T, np.full(nb, int(k1[i]), np.int32), ("gauss", 4, i))
                   for i in range(n)]
        cfg = {"workload": f"precision: {n} x {T} complex64, N={N}, overlap {N // 4}, "
                           f"k1~U{{1..N/2-13}}, L_V=12, DFT stages {PREC_NAME[args.prec]}",
               "channels": n, "samples_per_channel": T, "N": N, "seed": 4,
               "precision": PREC_NAME[args.prec]}
        return streams, V, cfg
    raise ValueError(name)


PREC_CODE = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x6": 3}
PREC_NAME = {"fp32": "FP32 register FFT (CUDA cores)",
             "bf16": "tensor-core GEMMs, BF16 hi+lo (3 products), FP32 accumulation",
             "fp16": "tensor-core GEMMs, row-scaled FP16 hi+lo (3 products), FP32 accumulation",
             "bf16x6": "tensor-core GEMMs, BF16 hi+mid+lo (6 products), FP32 accumulation"}


def gen_samples(gen, n):
    from paper_2406_14116_gb300 import workloads as wl
    kind, seed, sid = gen
    if kind == "gauss":
        return wl.complex_gaussian(seed, sid, n)
    return wl.tones_signal(seed, sid, n)


def fill_inputs(streams, views, threads=None):
    """Draws every stream's samples into its (pinned) host view, in parallel threads."""
    def one(i):
        views[i][:] = gen_samples(streams[i].gen, streams[i].nsamples)
    with cf.ThreadPoolExecutor(max_workers=threads or min(32, os.cpu_count() or 8)) as ex:
        list(ex.map(one, range(len(streams))))


# ---- oracle timing (the cpu_baseline leg and the reference arm) ------------------------------

def oracle_blocks(oracle, V, s, x, b0, nb):
    """Oracle output of blocks [b0, b0 + nb) of one stream: the segment from b0*M with the O
    preceding samples as its prefix (the OLS definition makes this the same blocks)."""
    M = s.N - s.overlap
    O = s.overlap
    lo = b0 * M
    hi = min(len(x), (b0 + nb) * M)
    tail = x[lo - O: lo] if lo >= O else np.concatenate([np.zeros(O - lo, np.complex64), x[:lo]])
    return oracle.filter(s.N, O, V, s.band[b0: b0 + nb], x[lo:hi], tail=tail)


def pick_runs(streams, g, run_len, count):
    """(stream index, first block) of runs of consecutive blocks: the first stream's start, the
    last stream's ragged end, then seeded positions. A workload with fewer than count x run_len
    blocks is covered whole, by non-overlapping runs."""
    nbs = [(s.nsamples + s.N - s.overlap - 1) // (s.N - s.overlap) for s in streams]
    if sum(nbs) <= count * run_len:
        return [(i, b0) for i, nb in enumerate(nbs) for b0 in range(0, nb, run_len)]
    runs = [(0, 0)]
    last = len(streams) - 1
    runs.append((last, max(0, nbs[last] - run_len)))
    while len(runs) < count:
        i = int(g.integers(0, len(streams)))
        runs.append((i, int(g.integers(0, max(1, nbs[i] - run_len)))))
    return runs


def cpu_baseline(streams, V, host_views, out_fetch, seconds):
    """FP64 oracle on runs of consecutive blocks for about `seconds`; the same blocks of the GPU
    output are compared with it (RMS relative error)."""
    import oracle
    g = np.random.default_rng(12345)
    run_len = 64
    runs = pick_runs(streams, g, run_len, 4096)
    num = den = 0.0
    t_used = 0.0
    samples = 0
    done = 0
    for i, b0 in runs:
        if t_used >= seconds and done >= 2:
            break
        s = streams[i]
        x = host_views[i]
        t0 = time.perf_counter()
        ref = oracle_blocks(oracle, V, s, x, b0, run_len)
        t_used += time.perf_counter() - t0
        lo = b0 * (s.N - s.overlap)
        y = out_fetch(i, lo, lo + len(ref)).astype(np.complex128)
        num += float(np.sum(np.abs(y - ref) ** 2))
        den += float(np.sum(np.abs(ref) ** 2))
        samples += len(ref)
        done += 1
    return {
        "value": samples / t_used / 1e9, "unit": UNIT, "cores": oracle.max_threads(),
        "kind": "oracle",
        "sample": f"{done} runs of up to {run_len} consecutive blocks ({samples} output samples) at "
                  f"seeded stream/block positions incl. the first stream's start and the last "
                  f"stream's end; FP64 direct-DFT OLS",
        "seconds": t_used, "samples": samples,
    }, (float(np.sqrt(num / den)) if den > 0 else None)


def reference_arm(args):
    """The FP64 oracle as the reference implementation, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    streams, V, cfg = make_streams(args.workload, args, 0)
    pool = [0, len(streams) - 1] + list(range(1, min(4, len(streams) - 1)))
    xs = {i: gen_samples(streams[i].gen, streams[i].nsamples) for i in pool}
    s0 = streams[pool[0]]
    t0 = time.perf_counter()
    oracle_blocks(oracle, V, s0, xs[pool[0]], 0, 8)
    t_blk = (time.perf_counter() - t0) / 8
    budget = 150.0
    nb_step = int(max(1, min(512, budget / max(1, args.steps + args.warmup) / t_blk)))
    g = np.random.default_rng(7)

    def step(k):
        i = pool[k % len(pool)]
        s = streams[i]
        M = s.N - s.overlap
        nbi = (s.nsamples + M - 1) // M
        b0 = int(g.integers(0, max(1, nbi - nb_step)))
        return len(oracle_blocks(oracle, V, s, xs[i], b0, nb_step))

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    samples = 0
    for k in range(args.steps):
        samples += step(k)
    dt = time.perf_counter() - t0
    value = samples / dt / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"each step: {nb_step} consecutive blocks of one stream "
                                   f"(FP64 direct-DFT OLS, the method's definition)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- native arm --------------------------------------------------------------------------------

# Pinned host input and its device copy, reused by runs over the same signals (the precision
# sweep filters one input with every (N, precision) pair).
_INPUT_CACHE = {}


def native_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    line = native_run(args)
    if line is None:
        return
    if args.workload == "channels" and world == 1 and not args.no_configs:
        line["configs"] = config_records(args)
    print(json.dumps(line), flush=True)


def native_run(args):
    """One workload through the batch API; returns rank 0's JSON record (None on other ranks)."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2406_14116_gb300 import build as vbw_build
    from paper_2406_14116_gb300 import tune
    from paper_2406_14116_gb300 import vbw
    vbw_build.build()

    streams, V, cfg = make_streams(args.workload, args, rank)
    cfg["parallelism"] = f"replicas x{world} (independent streams per GPU, no collective)"
    Ns = sorted({s.N for s in streams})
    if not args.no_tune:
        tune.load_or_tune(torch, Ns)
        cfg["tuned_shapes"] = {str(N): vbw_tune_shape(tune, torch, N) for N in Ns}

    # pinned host inputs (one buffer), seeded per stream
    offs = np.concatenate([[0], np.cumsum([s.nsamples for s in streams])]).astype(np.int64)
    total = int(offs[-1])
    key = (tuple(s.gen for s in streams), tuple(int(s.nsamples) for s in streams))
    if key in _INPUT_CACHE:
        host_in, d_in = _INPUT_CACHE[key]
        hnp = host_in.numpy()
        views = [hnp[offs[i]:offs[i + 1]] for i in range(len(streams))]
    else:
        _INPUT_CACHE.clear()
        host_in = torch.empty(total, dtype=torch.complex64, pin_memory=True)
        hnp = host_in.numpy()
        views = [hnp[offs[i]:offs[i + 1]] for i in range(len(streams))]
        fill_inputs(streams, views)
        d_in = host_in.cuda()
        if getattr(args, "keep_input", False):
            _INPUT_CACHE[key] = (host_in, d_in)
    d_out = torch.empty_like(d_in)
    plans = {}
    for s in streams:
        key = (s.N, s.overlap)
        if key not in plans:
            plans[key] = vbw.Plan(s.N, s.overlap, V, precision=PREC_CODE[args.prec])
    batch = vbw.Batch([(plans[(s.N, s.overlap)], d_in[offs[i]:offs[i + 1]],
                        d_out[offs[i]:offs[i + 1]], s.band) for i, s in enumerate(streams)])
    side = torch.cuda.Stream()          # graphs cannot be captured on the default stream
    torch.cuda.set_stream(side)
    stream = side
    forced = getattr(args, "batch_mode", "tuned")
    if len(plans) > 1 and forced != "tuned":
        batch.set_mode(vbw.VBW_BATCH_PER_PLAN if forced == "per_plan" else vbw.VBW_BATCH_MIXED)
        cfg["batch_mode"] = {"mode": forced, "forced": True}
    elif len(plans) > 1 and not args.no_tune:
        tm = tune.tune_mixed(torch, batch)
        names = {vbw.VBW_BATCH_PER_PLAN: "per_plan", vbw.VBW_BATCH_MIXED: "mixed"}
        cfg["batch_mode"] = {"mode": names.get(tm["mode"], tm["mode"]), "share": tm["share"],
                             "ms_by_mode": {f"{names.get(r['mode'], r['mode'])}"
                                            f"{'@' + str(r['share']) if r['mode'] == vbw.VBW_BATCH_MIXED else ''}":
                                            round(r["ms"], 4) for r in tm["table"]}}

    # a CUDA graph of one step (one batch launch, or the mixed launch and its forked branch)
    graph = None
    if args.workload == "mixed":
        batch.run(stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            batch.run(stream)
        cfg["cuda_graph"] = True

    def step():
        if graph is not None:
            graph.replay()
        else:
            batch.run(stream)

    flush = None
    if total * 16 < 2 * L2_BYTES:
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        cfg["l2"] = "L2 flushed between timed steps (a 252 MB write); only the step is timed"
    else:
        cfg["l2"] = "inputs larger than L2 (no flush needed)"

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    launches_per_step = batch.launches
    barrier()
    sampler = ClockSampler(device_uuid(torch, local))

    def timed():
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        sampler.start()
        barrier()
        for k in range(args.steps):
            if flush is not None:
                flush.fill_(float(k))
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
        barrier()
        clocks = sampler.stop()
        per = np.array([ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)])
        total_ms = float(per.sum()) if flush is not None else float(ev0[0].elapsed_time(ev1[-1]))
        return total_ms, per, clocks

    total_ms, per_ms, clocks = timed()
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    remeasured = False
    if bad & set(clocks.get("reasons", [])):
        total_ms, per_ms, clocks = timed()
        remeasured = True
    value = job_gsamples(total, args.steps, total_ms / 1e3, "cuda")
    total_ms = rank_reduce(total_ms, "max", "cuda")
    step_ms = float(np.mean(per_ms))
    peak, peak_src = measured_peaks()
    achieved = BYTES_PER_SAMPLE * total / (step_ms / 1e3) / 1e9
    tag = {"channels": "ols_fp32_n1024_channels"}.get(args.workload, f"ols_fp32_{args.workload}")
    traffic = profile_traffic(tag)
    if args.workload == "precision" and args.prec == "bf16" and not args.channels and not args.samples:
        traffic = profile_traffic("ols_tc_n256-512_bf16_precision", TC_SOURCES,
                                  key=f"dram_bytes_per_full_launch_n{args.N}")
    split2048 = (args.workload == "precision" and args.prec == "fp32" and args.N == 2048 and
                 os.environ.get("VBW_SPLIT2048", "1") != "0")
    if split2048 and not args.channels and not args.samples:
        traffic = profile_traffic("ols_split2048_n2048_precision", SPLIT_SOURCES)

    e2e = None
    if not args.no_e2e:
        host_out = torch.empty_like(host_in, pin_memory=True)
        onp = host_out.numpy()
        oviews = [onp[offs[i]:offs[i + 1]] for i in range(len(streams))]
        # the buffers' addresses, made once (a caller that repeats a batch keeps them)
        pin_in, pin_out = vbw.host_pointers(views), vbw.host_pointers(oviews)
        batch.run_host(pin_in, pin_out, stream)
        k_e2e = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            batch.run_host(pin_in, pin_out, stream)
        barrier()
        dt = time.perf_counter() - t0
        e2e = {"value": job_gsamples(total, k_e2e, dt, "cuda"), "unit": UNIT,
               "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total,
               "steps": k_e2e,
               "api": "vbw_batch_run_host, pinned host buffers (zero copy: the kernels read and "
                      "write host memory over NVLink-C2C)"}
        step()
        torch.cuda.synchronize()
        n_chk = min(total, 1 << 20)
        if not np.array_equal(onp[:n_chk], d_out[:n_chk].cpu().numpy()):
            e2e["mismatch_vs_device_path"] = True

    latency = None
    if args.workload == "single":
        # per-call latency of the stream API on this signal: vbw_filter + vbw_flush, synchronized,
        # host wall time (launch and completion included)
        s0 = streams[0]
        M0 = s0.N - s0.overlap
        plan0 = plans[(s0.N, s0.overlap)]
        xs, ys = d_in[:s0.nsamples], d_out[:s0.nsamples]
        nfull = s0.nsamples // M0
        st_api = vbw.Stream(plan0, int(s0.band[0]), stream)
        lat = []
        for k in range(210):
            st_api.reset(int(s0.band[0]))
            t0 = time.perf_counter()
            st_api.filter(xs[:nfull * M0], ys[:nfull * M0], nfull)
            st_api.flush(xs[nfull * M0:], ys[nfull * M0:], s0.nsamples - nfull * M0)
            stream.synchronize()
            if k >= 10:
                lat.append(time.perf_counter() - t0)
        lat = np.array(lat) * 1e6
        latency = {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                   "calls": len(lat), "api": "vbw_filter + vbw_flush on one stream, synchronized"}
        st_api.close()

    cpu = None
    rms = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, rms = cpu_baseline(streams, V, views,
                                lambda i, lo, hi: d_out[offs[i] + lo: offs[i] + hi].cpu().numpy(),
                                args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16x2 split, f32 acc", "fp16": "f16x2 scaled, f32 acc",
                      "bf16x6": "bf16x3 split, f32 acc"}[args.prec],
            "data": "synthetic",
            "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS hbm_gbs)" if peak_src == "measured"
                         else "fallback 6.8 TB/s",
                         "kernel": ("ols_tc_kernel (tcgen05)" if args.prec != "fp32" else
                                    "ols_split2048_kernel" if split2048 else
                                    "ols_fp32_kernel" if launches_per_step == 1 else "ols_fp32/ols_mixed kernels"),
                         "launch_ms": step_ms / launches_per_step,
                         "step_ms": step_ms,
                         "algorithmic_bytes_per_step": BYTES_PER_SAMPLE * total},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
            "rms_rel_err_sampled": rms,
            "rms_tol": FP32_RMS_TOL if args.prec == "fp32" else 1e-5,
        }
        if latency is not None:
            line["latency_us"] = latency
        if remeasured:
            line["remeasured_after_throttle"] = True
    for p in plans.values():
        p.close()
    batch.close()
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


# ---- serving workload --------------------------------------------------------------------------

SERVING = dict(seed=5, nstreams=2000, LV=12, Ns=(512, 1024, 2048), lo=1024, hi=65536,
               change_frac=0.01)


def serving_arm(args):
    line = serving_run(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def serving_run(args):
    """Open-loop serving: chunks arrive at Poisson times (aggregate --rate chunks/s, stream
    uniform, length U{1024..65536}, 1% carry a band change) and go through vbw_server_submit /
    vbw_server_poll as they arrive. Latency = completion time - scheduled arrival. Then a
    saturation pass submits the same chunks as fast as the queue accepts them (the engine's
    sustainable throughput). Inputs are pinned host buffers; every sample crosses the host link
    both ways."""
    import torch
    import torch.distributed as dist

    from paper_2406_14116_gb300 import build as vbw_build
    from paper_2406_14116_gb300 import vbw
    from paper_2406_14116_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vbw_build.build()
    c = SERVING
    V = wl.transition_table(c["seed"], c["LV"])
    Nsel, Osel, k1 = wl.serving_streams(c["seed"] + rank, c["nstreams"], c["LV"], c["Ns"])
    t_arr, sid, lens, nbands = wl.serving_arrivals(c["seed"] + rank, c["nstreams"], args.rate,
                                                   args.duration, c["lo"], c["hi"],
                                                   c["change_frac"], Nsel, c["LV"])
    nreq = len(t_arr)
    plans = [vbw.Plan(N, N // 4, V) for N in c["Ns"]]
    pidx = {N: i for i, N in enumerate(c["Ns"])}
    M_of = (Nsel - Nsel // 4).astype(np.int64)

    # pinned host memory: one seeded base signal that every stream reads cyclically from its own
    # offset, and an output ring that completions free in order
    base_len = 1 << 22
    base_t = torch.empty(base_len + c["hi"], dtype=torch.complex64, pin_memory=True)
    base = base_t.numpy()
    base[:base_len] = wl.complex_gaussian(c["seed"], 10_000 + rank, base_len)
    base[base_len:] = base[:c["hi"]]
    ring_len = 1 << 28
    ring_t = torch.empty(ring_len, dtype=torch.complex64, pin_memory=True)
    ring = ring_t.numpy()
    base_addr, ring_addr = int(base.ctypes.data), int(ring.ctypes.data)
    soff = (np.arange(c["nstreams"], dtype=np.int64) * 7919 * 97) % base_len

    # per chunk: input address, output count (blocks the chunk completes)
    pos = np.zeros(c["nstreams"], dtype=np.int64)
    in_addr = np.empty(nreq, dtype=np.int64)
    outn = np.empty(nreq, dtype=np.int64)
    for k in range(nreq):
        s = sid[k]
        S = pos[s]
        in_addr[k] = base_addr + 8 * ((soff[s] + S) % base_len)
        outn[k] = (S + lens[k]) // M_of[s] * M_of[s] - S // M_of[s] * M_of[s]
        pos[s] = S + lens[k]
    L = vbw.lib()

    def ring_place(head, n, tail, outstanding):
        """Start of n free ring samples at or after head (wrapping to 0), or None if the ring is
        full. Outputs in flight occupy [tail, head) cyclically."""
        if not outstanding:
            return head if head + n <= ring_len else 0
        if head >= tail:
            if head + n <= ring_len:
                return head
            return 0 if n < tail else None
        return head if head + n < tail else None

    def run(open_loop: bool, limit: int = nreq):
        sv = vbw.Server(plans, max_streams=c["nstreams"], pool_bytes=args.pool_mb << 20,
                        slots=args.slots)
        for i in range(c["nstreams"]):
            sv.open_stream(i, pidx[int(Nsel[i])], int(k1[i]))
        done_t = np.full(nreq, np.nan)
        out_end = np.zeros(nreq, dtype=np.int64)
        buf = sv._buf
        h = sv.handle
        nd = ctypes.c_int(0)
        ndp = ctypes.byref(nd)
        bufp = buf.ctypes.data
        state = {"tail": 0, "ndone": 0}

        def harvest(block=False):
            rc = (L.vbw_server_wait if block else L.vbw_server_poll)(h, bufp, len(buf), ndp)
            if rc != 0:
                raise vbw.VbwError(rc, vbw.vbw_last_error())
            n = nd.value
            if n:
                tags = buf["tag"][:n]
                done_t[tags] = buf["t_done"][:n]
                state["tail"] = int(out_end[tags[-1]])
                state["ndone"] += n
            return n

        head = 0
        clock = L.vbw_server_clock
        t0 = clock()
        sched = t0 + t_arr
        if not open_loop:
            # saturation: groups of chunks per vbw_server_submit_many call, outputs contiguous
            G = 512
            k = 0
            while k < limit:
                g1 = min(limit, k + G)
                outs = outn[k:g1]
                total = int(outs.sum())
                while True:
                    at = ring_place(head, max(total, 1), state["tail"], state["ndone"] < k)
                    if at is not None:
                        head = at
                        break
                    harvest(block=True)
                offs = head + np.concatenate([[0], np.cumsum(outs)[:-1]]).astype(np.int64)
                req = np.zeros(g1 - k, dtype=vbw.REQUEST_DTYPE)
                req["stream"] = sid[k:g1]
                req["new_band"] = nbands[k:g1]
                req["host_in"] = in_addr[k:g1]
                req["n"] = lens[k:g1]
                req["host_out"] = np.where(outs > 0, ring_addr + 8 * offs, 0)
                req["out_capacity"] = outs
                req["tag"] = np.arange(k, g1)
                sv.submit_many(req)
                out_end[k:g1] = offs + outs
                head += total
                harvest()
                k = g1
            while state["ndone"] < limit:
                harvest(block=True)
            t_end = clock()
            info = sv.info()
            sv.close()
            return sched, done_t, t0, t_end, info
        for k in range(limit):
            if open_loop:
                while clock() < sched[k]:
                    harvest()
            n_out = int(outn[k])
            # output ring: contiguous space for the chunk's output, freed in completion order
            if n_out:
                while True:
                    at = ring_place(head, n_out, state["tail"], state["ndone"] < k)
                    if at is not None:
                        head = at
                        break
                    harvest(block=True)
            rc = L.vbw_server_submit(h, int(sid[k]), int(in_addr[k]), int(lens[k]), int(nbands[k]),
                                     ring_addr + 8 * head if n_out else 0, n_out, k)
            if rc != 0:
                raise vbw.VbwError(rc, vbw.vbw_last_error())
            out_end[k] = head + n_out
            head += n_out
            if not open_loop and (k & 15) == 0:
                harvest()
        while state["ndone"] < limit:
            harvest(block=True)
        t_end = clock()
        info = sv.info()
        sv.close()
        return sched, done_t, t0, t_end, info

    run(open_loop=False, limit=min(nreq, 4000))     # warm-up: first launches, page-in
    sampler = ClockSampler(device_uuid(torch, local))
    sampler.start()
    # no garbage-collector pauses inside the arrival loop (a serving process keeps its heap
    # frozen while it serves)
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        sched, done_t, t0, t_end, info = run(open_loop=True)
    finally:
        gc.enable()
        gc.unfreeze()
    clocks = sampler.stop()
    lat = (done_t - sched) * 1e3
    samples = int(lens.sum())
    span = t_end - t0
    _, _, s0, s1, info_sat = run(open_loop=False)
    value = rank_reduce(samples / span / 1e9, "sum", "cuda")
    sat = rank_reduce(samples / (s1 - s0) / 1e9, "sum", "cuda")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": nreq,
            "warmup": min(nreq, 4000), "ms_per_step": 1e3 * span / nreq, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: {c['nstreams']} streams, N in {list(c['Ns'])}, O = N/4, "
                                   f"L_V {c['LV']}, Poisson {args.rate:.0f} chunks/s for "
                                   f"{args.duration:g} s, chunk U{{{c['lo']}..{c['hi']}}}, "
                                   f"{c['change_frac']:.0%} band changes",
                       "pool_mib": args.pool_mb, "slots": args.slots,
                       "parallelism": f"replicas x{world}",
                       "l2": "host-resident chunks, every sample crosses the host link both ways"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(np.max(lat)),
                           "from": "scheduled arrival", "to": "outputs on the host (seen by poll)"},
            "offered_gsamples_s": samples / args.duration / 1e9 * world,
            "saturation_gsamples_s": sat,
            "saturation_api": "vbw_server_submit_many, 512 chunks per call",
            "batches": info["batches"], "chunks_per_batch": nreq / max(1, info["batches"]),
            "saturation_batches": info_sat["batches"],
            "gpu_launches": info["launches"],
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(8 * lens.mean()),
                    "d2h_bytes_per_step": int(8 * outn.mean()),
                    "api": "vbw_server_submit / vbw_server_poll, pinned host buffers; a step is one chunk"},
            "roofline": None, "cpu_baseline": None, "clocks": clocks,
        }
    for p in plans:
        p.close()
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


# ---- the other four workloads, recorded beside the headline ------------------------------------

CONFIG_CPU_SECONDS = 4.0      # oracle seconds per recorded workload (sampled parity)


def _brief(line):
    """The compact record of one workload's JSON line."""
    cpu = line.get("cpu_baseline") or {}
    roof = line.get("roofline") or {}
    return {
        "workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
        "ms_per_step": line["ms_per_step"], "steps": line["steps"], "dtype": line["dtype"],
        "roofline_frac": roof.get("frac"), "roofline_kernel": roof.get("kernel"),
        "launch_ms": roof.get("launch_ms"), "gpu_launches": line.get("gpu_launches"),
        "clocks": line.get("clocks"), "l2": line["config"].get("l2"),
        "rms_rel_err_sampled": line.get("rms_rel_err_sampled"), "rms_tol": line.get("rms_tol"),
        "rms_samples": cpu.get("samples"), "rms_sample": cpu.get("sample"),
        "cpu_baseline_gsamples_s": cpu.get("value"), "cpu_cores": cpu.get("cores"),
    }


def config_records(args):
    """Runs the single-stream, mixed, precision and serving workloads at full size after the
    headline (rank 0 of a one-GPU run) and returns one compact record per workload: throughput,
    HBM fraction, clocks, and the oracle's RMS error on sampled blocks with the sample size."""
    import copy

    import torch

    def sub(**kw):
        a = copy.copy(args)
        a.channels = None
        a.samples = None
        a.no_e2e = True
        a.no_cpu = args.no_cpu
        a.cpu_seconds = CONFIG_CPU_SECONDS
        a.steps = max(3, min(args.steps, 20))
        a.warmup = 3
        a.prec = "fp32"
        a.keep_input = False
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    out = {}
    t0 = time.perf_counter()
    try:
        # single stream (2^16 samples, N = 256): throughput with L2 flushed, and per-call latency
        line = native_run(sub(workload="single", steps=200))
        r = _brief(line)
        r["latency_us"] = line.get("latency_us")
        out["single"] = r
        torch.cuda.empty_cache()

        # mixed batch (4096 streams, N = 128..2048) as one CUDA graph
        line = native_run(sub(workload="mixed"))
        r = _brief(line)
        r["batch_mode"] = line["config"].get("batch_mode")
        out["mixed"] = r
        torch.cuda.empty_cache()

        # precision (16384 x 2^16): the FP32 path and every tensor-core split at N = 256 and 512,
        # one input for all of them
        prec = {}
        for N in (256, 512):
            rows = {}
            for pr in ("fp32", "bf16", "fp16", "bf16x6"):
                line = native_run(sub(workload="precision", N=N, prec=pr, keep_input=True,
                                      cpu_seconds=3.0))
                rows[pr] = _brief(line)
            for pr in ("bf16", "fp16", "bf16x6"):
                rows[pr]["speedup_vs_fp32"] = rows[pr]["value"] / rows["fp32"]["value"]
            ok = [pr for pr in ("bf16", "fp16", "bf16x6")
                  if rows[pr]["rms_rel_err_sampled"] is not None
                  and rows[pr]["rms_rel_err_sampled"] <= rows[pr]["rms_tol"]]
            best = max(ok, key=lambda pr: rows[pr]["value"]) if ok else None
            prec[str(N)] = {"runs": rows, "best_split": best,
                            "best_split_speedup_vs_fp32": rows[best]["speedup_vs_fp32"] if best else None}
        out["precision"] = prec
        _INPUT_CACHE.clear()
        torch.cuda.empty_cache()

        # serving: 2000 streams, Poisson arrivals at 50k chunks/s for a few seconds, then saturation;
        # in a process of its own, so that the other workloads' host threads and memory do not
        # stall its arrival loop
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serving", "--duration", "5",
               "--rate", str(args.rate), "--pool-mb", str(args.pool_mb), "--slots", str(args.slots)]
        proc = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
        lines = [x for x in proc.stdout.splitlines() if x.startswith("{")]
        if proc.returncode != 0 or not lines:
            raise RuntimeError(f"serving run failed (rc {proc.returncode}): {proc.stderr[-300:]}")
        line = json.loads(lines[-1])
        out["serving"] = {
            "workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
            "latency_ms": line["latency_ms"], "offered_gsamples_s": line["offered_gsamples_s"],
            "saturation_gsamples_s": line["saturation_gsamples_s"], "chunks": line["steps"],
            "batches": line["batches"], "gpu_launches": line["gpu_launches"],
            "clocks": line["clocks"], "process": "separate (python bench.py --workload serving)",
            "parity": "tests/test_serving_gpu.py (per-stream oracle parity, alone vs mixed bit-equal)",
        }
    except Exception as e:   # the headline stands; the record says what failed
        out["error"] = f"{type(e).__name__}: {e}"
    out["seconds"] = time.perf_counter() - t0
    return out


# ---- real-valued signals ------------------------------------------------------------------------

REAL = dict(seed=6, nch=64, nsamples=1 << 23, N=1024, overlap=256, LV=12, every=16, lo=32, hi=480)


def real_arm(args):
    """Real float32 channels through vbw_batch_create_real: two real blocks per complex transform.
    8 algorithmic bytes per real output sample (4 read + 4 written)."""
    import torch
    import torch.distributed as dist

    from paper_2406_14116_gb300 import build as vbw_build
    from paper_2406_14116_gb300 import tune
    from paper_2406_14116_gb300 import vbw
    from paper_2406_14116_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vbw_build.build()
    c = dict(REAL)
    if args.channels:
        c["nch"] = args.channels
    if args.samples:
        c["nsamples"] = args.samples
    N, O, nch, T = c["N"], c["overlap"], c["nch"], c["nsamples"]
    M = N - O
    V = wl.transition_table(c["seed"], c["LV"])
    if not args.no_tune:
        tune.load_or_tune(torch, [N])
    # seeded real Gaussian input, generated on the device (host pinned copy for the e2e leg)
    g = torch.Generator(device="cuda").manual_seed(c["seed"] * 1000 + rank)
    x = torch.randn((nch, T), dtype=torch.float32, device="cuda", generator=g)
    y = torch.empty_like(x)
    nb = (T + M - 1) // M
    bands = [wl.band_schedule(c["seed"], i, nb, c["every"], c["lo"], c["hi"]) for i in range(nch)]
    plan = vbw.Plan(N, O, V)
    batch = vbw.Batch([(plan, x[i], y[i], bands[i]) for i in range(nch)], real=True)
    side = torch.cuda.Stream()
    torch.cuda.set_stream(side)
    total = nch * T
    for _ in range(max(3, args.warmup)):
        batch.run(side)
    torch.cuda.synchronize()
    sampler = ClockSampler(device_uuid(torch, local))
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler.start()
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev0[k].record(side)
        batch.run(side)
        ev1[k].record(side)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per = np.array([ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)])
    total_ms = float(ev0[0].elapsed_time(ev1[-1]))
    value = job_gsamples(total, args.steps, total_ms / 1e3, "cuda")
    step_ms = float(per.mean())
    peak, peak_src = measured_peaks()
    achieved = 8 * total / (step_ms / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        hx = x.cpu().pin_memory()
        hy = torch.empty_like(hx, pin_memory=True)
        k_e2e = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            x.copy_(hx, non_blocking=True)
            batch.run(side)
            hy.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": job_gsamples(total, k_e2e, dt, "cuda"), "unit": UNIT,
               "h2d_bytes_per_step": 4 * total, "d2h_bytes_per_step": 4 * total, "steps": k_e2e,
               "api": "pinned host -> device copy, vbw_batch_run (real batch), device -> host copy"}

    cpu = None
    rms = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        rng = np.random.default_rng(7)
        t0 = time.perf_counter()
        num = den = 0.0
        done = 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            i = int(rng.integers(0, nch))
            b0 = int(rng.integers(0, max(1, nb - 64)))
            lo, hi = b0 * M, min(T, (b0 + 64) * M)
            xs = x[i, max(0, lo - O):hi].cpu().numpy().astype(np.complex64)
            tail = None
            if lo >= O:
                tail, xs = xs[:O], xs[O:]
            ref = oracle.filter(N, O, V, bands[i][b0:b0 + 64], xs, tail=tail).real
            got = y[i, lo:hi].cpu().numpy().astype(np.float64)
            num += float(np.sum((got - ref) ** 2))
            den += float(np.sum(ref ** 2))
            done += hi - lo
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{done} real samples in runs of 64 blocks at seeded positions (FP64 oracle on x + 0j)",
               "seconds": dt}
        rms = math.sqrt(num / den) if den > 0 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"real: {nch} x {T} float32 real samples, N={N}, overlap {O}, "
                                   f"L_V={c['LV']}, k1~U{{{c['lo']}..{c['hi']}}} every {c['every']} blocks; "
                                   "two real blocks per complex transform",
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (no flush needed)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profile_traffic("ols_fp32_n1024_real"),
                         "peak_source": f"{peak_src} (MEASURED_PEAKS hbm_gbs)",
                         "kernel": "ols_fp32_kernel (real pairs)", "step_ms": step_ms,
                         "algorithmic_bytes_per_step": 8 * total},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": batch.launches * args.steps, "rms_rel_err_sampled": rms,
            "rms_tol": FP32_RMS_TOL,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# PTVIR error analysis on the channel workload's geometry: every band of its range, the design
# grid of each band (passband [0, w_c], stopband [w_s, pi])
PTVIR = dict(seed=2, N=1024, overlap=256, LV=12, lo=32, hi=480, K=4096)
FP32_LANES_PER_SM = 128        # FP32 FMA lanes per SM (4 SM sub-partitions x 32)


def ptvir_grid(N, LV, bands, K):
    """K points per band over [0, w_c] and [w_s, pi], w_c = 2 pi (k1 - 1)/N the last passband bin,
    w_s = 2 pi (k1 + L_V)/N the first stopband bin, in proportion to their widths."""
    W = np.empty((len(bands), K))
    Dd = np.empty((len(bands), K), dtype=np.float32)
    for j, k1 in enumerate(bands):
        wc = 2 * np.pi * (k1 - 1) / N
        ws = 2 * np.pi * (k1 + LV) / N
        Kp = int(np.clip(round(K * wc / (wc + np.pi - ws)), 1, K - 1))
        W[j] = np.concatenate([np.linspace(0.0, wc, Kp), np.linspace(ws, np.pi, K - Kp)])
        Dd[j] = np.concatenate([np.ones(Kp), np.zeros(K - Kp)])
    return W, Dd


def ptvir_arm(args):
    """vbw_ptvir_error over the channel geometry's design grid: max over the M output phases of
    |E_n(w, b)| (eq. (OLS_Hn), eq. (err_min)) at every band and grid point. The unit of work is
    one (band, frequency) point, i.e. M error evaluations; the kernel is bound by FP32 arithmetic:
    10 N + 11 M algorithmic flops per point (a complex phasor and a real x complex accumulation
    per tap, a complex multiply-add and a squared modulus per phase)."""
    import torch

    from paper_2406_14116_gb300 import build as vbw_build
    from paper_2406_14116_gb300 import vbw
    from paper_2406_14116_gb300 import workloads as wl

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    c = dict(PTVIR)
    N, O, LV = c["N"], c["overlap"], c["LV"]
    M = N - O
    V = wl.transition_table(c["seed"], LV)
    bands = np.arange(c["lo"], c["hi"] + 1, dtype=np.int32)
    W, Dd = ptvir_grid(N, LV, bands, c["K"])
    points = W.size
    flops_per_point = 10 * N + 11 * M
    cfg = {"workload": f"ptvir: N={N}, overlap {O}, L_V={LV}, k1 in {c['lo']}..{c['hi']} "
                       f"({len(bands)} bands) x {c['K']} grid points, max over {M} output phases",
           "N": N, "overlap": O, "L_V": LV, "bands": len(bands), "K": c["K"], "phases": M,
           "parallelism": f"replicas x{world}",
           "l2": "arithmetic-bound; the 22 MB of inputs stay in L2 (no flush needed)"}
    metric = "PTVIR error evaluations |E_n(w, b)| per second (max over output phases)"
    unit = "Gevals/s"

    def oracle_leg(seconds):
        import oracle
        g = np.random.default_rng(3)
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < seconds:
            j = int(g.integers(0, len(bands)))
            cols = g.choice(W.shape[1], 4, replace=False)
            oracle.ptvir_errors(N, O, V, int(bands[j]), W[j, cols], Dd[j, cols])
            done += 4 * M
        dt = time.perf_counter() - t0
        return {"value": done / dt / 1e9, "unit": unit, "cores": oracle.max_threads(), "kind": "oracle",
                "sample": f"{done // M} (band, frequency) points x {M} phases at seeded positions "
                          "(FP64 direct sums over the taps, one phase at a time)", "seconds": dt}

    if args.impl == "reference":
        if rank != 0:
            return
        for _ in range(args.warmup):
            oracle_leg(0.5)
        cpu = oracle_leg(max(5.0, 2.0 * args.steps))
        print(json.dumps({"metric": metric, "value": cpu["value"], "unit": unit, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "impl": "reference", "config": cfg, "cpu_baseline": cpu,
                          "e2e": {"value": cpu["value"], "unit": unit, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    vbw_build.build()
    plan = vbw.Plan(N, O, V)
    t_b = torch.tensor(bands, device="cuda")
    t_w = torch.tensor(W, dtype=torch.float64, device="cuda")
    t_d = torch.tensor(Dd, device="cuda")
    t_e = torch.empty(W.shape, dtype=torch.float32, device="cuda")
    t_p = torch.empty(W.shape, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    for _ in range(max(3, args.warmup)):
        vbw.vbw_ptvir_error(plan.handle, t_b, t_w, t_d, t_e, t_p, side)
    torch.cuda.synchronize()
    steps = args.steps
    sampler = ClockSampler(device_uuid(torch, local))
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler.start()
    torch.cuda.synchronize()
    for k in range(steps):
        ev0[k].record(side)
        vbw.vbw_ptvir_error(plan.handle, t_b, t_w, t_d, t_e, t_p, side)
        ev1[k].record(side)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per = np.array([ev0[k].elapsed_time(ev1[k]) for k in range(steps)])
    total_ms = float(ev0[0].elapsed_time(ev1[-1]))
    evals = points * M
    value = rank_reduce(evals * steps / (total_ms / 1e3), "sum", "cuda") / 1e9
    step_ms = float(per.mean())
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = 2070.0
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        try:
            mhz = float(json.load(open(pk)).get("sm_max_mhz", mhz))
        except Exception:
            pass
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flops_per_point * points / (step_ms / 1e3) / 1e12

    # end to end through the same call with host buffers: grid in, errors and phases out
    e2e = None
    if not args.no_e2e:
        hw = torch.from_numpy(W).pin_memory()
        hd = torch.from_numpy(Dd).pin_memory()
        he = torch.empty(W.shape, dtype=torch.float32).pin_memory()
        hp = torch.empty(W.shape, dtype=torch.int32).pin_memory()
        k_e2e = max(3, min(steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(side):
            for _ in range(k_e2e):
                t_w.copy_(hw, non_blocking=True)
                t_d.copy_(hd, non_blocking=True)
                vbw.vbw_ptvir_error(plan.handle, t_b, t_w, t_d, t_e, t_p, side)
                he.copy_(t_e, non_blocking=True)
                hp.copy_(t_p, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": evals * k_e2e / dt / 1e9, "unit": unit,
               "h2d_bytes_per_step": int(W.nbytes + Dd.nbytes), "d2h_bytes_per_step": int(2 * 4 * points),
               "steps": k_e2e, "api": "pinned host grid -> device, vbw_ptvir_error, errors and phases -> host"}

    cpu = None
    worst = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        cpu = oracle_leg(args.cpu_seconds)
        # sampled parity: the kernel's maxima against the oracle's at seeded points
        err = t_e.cpu().numpy()
        g = np.random.default_rng(9)
        worst = 0.0
        for j in g.choice(len(bands), 3, replace=False):
            cols = g.choice(W.shape[1], 8, replace=False)
            E = oracle.ptvir_errors(N, O, V, int(bands[j]), W[j, cols], Dd[j, cols])
            h = oracle.impulse_response(N, O, V, int(bands[j]))
            tol = 1e-6 * max(1.0, float(np.abs(h).sum()))
            worst = max(worst, float(np.abs(err[j, cols] - E.max(axis=0)).max() / tol))

    if rank == 0:
        print(json.dumps({
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x "
                                        f"{mhz:.0f} MHz (maximum SM clock)",
                         "kernel": "ptvir_error_kernel", "step_ms": step_ms,
                         "algorithmic_flops_per_point": flops_per_point, "points_per_step": points},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": steps,
            "max_err_over_tol_sampled": worst, "tol": "1e-6 x max(1, sum_q |h(q)|)",
        }), flush=True)


def ola_reference(args):
    """The FP64 OLA oracle on the OLA workload's geometry, timed on the host cores: each step one
    run of consecutive blocks of a seeded signal (the reference arm of --workload ola)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    from paper_2406_14116_gb300 import workloads as wl
    c = CHANNELS
    N, O = c["N"], c["overlap"]
    M = N - O
    V = wl.transition_table(c["seed"], c["LV"])
    nblk = 24
    x = wl.complex_gaussian(c["seed"], 0, nblk * M)
    bands = wl.band_schedule(c["seed"], 0, nblk, c["every"], c["lo"], c["hi"])
    for _ in range(args.warmup):
        oracle.filter_ola(N, O, V, bands, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.filter_ola(N, O, V, bands, x)
    dt = time.perf_counter() - t0
    value = len(x) * args.steps / dt / 1e9
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": f"ola: N={N}, overlap {O}, L_V={c['LV']}, one signal of {nblk} blocks per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: {nblk} consecutive blocks of one signal (FP64 direct-DFT OLA)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def ola_arm(args):
    """The channel workload (64 x 2^22 complex64, N=1024, overlap 256, bands redrawn every 16
    blocks) through vbw_filter_ola: overlap-add with the same coefficients, one launch per step.
    16 algorithmic bytes per output sample, as for OLS."""
    import torch
    import torch.distributed as dist

    from paper_2406_14116_gb300 import build as vbw_build
    from paper_2406_14116_gb300 import vbw
    from paper_2406_14116_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vbw_build.build()
    c = dict(CHANNELS)
    if args.channels:
        c["nch"] = args.channels
    if args.samples:
        c["nsamples"] = args.samples
    N, O, nch, T = c["N"], c["overlap"], c["nch"], c["nsamples"]
    M = N - O
    V = wl.transition_table(c["seed"], c["LV"])
    nb = (T + M - 1) // M
    g = torch.Generator(device="cuda").manual_seed(c["seed"] * 1000 + 17 + rank)
    x = torch.randn((nch, T), dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    bands_np = np.stack([wl.band_schedule(c["seed"], i, nb, c["every"], c["lo"], c["hi"]) for i in range(nch)])
    bands = torch.from_numpy(bands_np.astype(np.int32)).cuda()
    plan = vbw.Plan(N, O, V)
    side = torch.cuda.Stream()

    def step():
        vbw.vbw_filter_ola(plan.handle, x, y, T, nch, 0, bands, side)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(device_uuid(torch, local))
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler.start()
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev0[k].record(side)
        step()
        ev1[k].record(side)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per = np.array([ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)])
    total_ms = float(ev0[0].elapsed_time(ev1[-1]))
    total = nch * T
    value = job_gsamples(total, args.steps, total_ms / 1e3, "cuda")
    step_ms = float(per.mean())
    peak, peak_src = measured_peaks()
    achieved = BYTES_PER_SAMPLE * total / (step_ms / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        hx = x.cpu().pin_memory()
        hy = torch.empty_like(hx, pin_memory=True)
        k_e2e = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(side):
            for _ in range(k_e2e):
                x.copy_(hx, non_blocking=True)
                step()
                hy.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": job_gsamples(total, k_e2e, dt, "cuda"), "unit": UNIT,
               "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total, "steps": k_e2e,
               "api": "pinned host -> device copy, vbw_filter_ola, device -> host copy"}

    cpu = None
    rms = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        rng = np.random.default_rng(7)
        t0 = time.perf_counter()
        num = den = 0.0
        done = 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            i = int(rng.integers(0, nch))
            b0 = int(rng.integers(1, max(2, nb - 16)))
            lo, hi = (b0 - 1) * M, min(T, (b0 + 16) * M)
            xs = x[i, lo:hi].cpu().numpy()
            ref = oracle.filter_ola(N, O, V, bands_np[i][b0 - 1:], xs)[M:]
            got = y[i, b0 * M:hi].cpu().numpy().astype(np.complex128)
            num += float(np.sum(np.abs(got - ref) ** 2))
            den += float(np.sum(np.abs(ref) ** 2))
            done += hi - b0 * M
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} output samples in runs of 16 blocks at seeded positions (FP64 direct-DFT "
                         "OLA, sequential)", "seconds": dt}
        rms = math.sqrt(num / den) if den > 0 else None

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ola: {nch} x {T} complex64, N={N}, overlap {O}, L_V={c['LV']}, "
                                   f"k1~U{{{c['lo']}..{c['hi']}}} every {c['every']} blocks; overlap-add",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush needed)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": profile_traffic("ola_fp32_n1024_channels", OLA_SOURCES),
                         "peak_source": f"{peak_src} (MEASURED_PEAKS hbm_gbs)", "kernel": "ola_fp32_kernel",
                         "step_ms": step_ms, "algorithmic_bytes_per_step": BYTES_PER_SAMPLE * total},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": args.steps,
            "rms_rel_err_sampled": rms, "rms_tol": FP32_RMS_TOL,
        }), flush=True)
    if world > 1:
        dist.destroy_process_group()


def vbw_tune_shape(tune, torch, N):
    c = tune.load(torch) or {}
    d = c.get("shapes", {}).get(str(N))
    return None if d is None else {"warps": d["warps"], "ctas_per_sm": d["ctas_per_sm"]}


def main():
    args = parse_args()
    if args.workload == "ptvir":
        ptvir_arm(args)
    elif args.workload == "ola":
        ola_reference(args) if args.impl == "reference" else ola_arm(args)
    elif args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serving":
        serving_arm(args)
    elif args.workload == "real":
        real_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
