"""Autotuner for libvbw's launch shapes on the current GPU.

For every transform size N it times the single-plan kernel on a synthetic channel batch
(overlap N/4, bands redrawn every 16 blocks) for each (warps per CTA, resident CTAs per SM) pair
and keeps the fastest. For a mixed-N batch it times the per-plan and mixed launch modes, the
latter with a few SM shares. The choices are kept in a JSON cache keyed by the GPU name and
applied through ``vbw_tune_set`` / ``vbw_batch_set_mode``; the numbers are timings only, the
arithmetic does not depend on them (tests check that every shape gives bit-identical output).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import vbw

PKG = os.path.dirname(os.path.abspath(__file__))
ALL_N = (128, 256, 512, 1024, 2048)
WARPS = (4, 8)
CTAS = (0, 1, 2, 3, 4)


def cache_path(torch) -> str:
    env = os.environ.get("VBW_TUNE_CACHE")
    if env:
        return env
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(PKG, "_tune", f"{name}.json")


def _time_ms(torch, fn, reps: int, stream) -> float:
    """Median over reps of the device time of fn() on stream (CUDA events)."""
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times))


def _channel_batch(torch, N: int, nch: int, nsamples: int):
    from . import workloads as wl
    O = N // 4
    V = wl.transition_table(101, 12)
    plan = vbw.Plan(N, O, V)
    g = torch.Generator(device="cuda").manual_seed(N)
    x = torch.randn((nch, nsamples), dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    nb = wl.nblocks_for(nsamples, N, O)
    rows = [(plan, x[c], y[c], wl.band_schedule(101, c, nb, 16, 1, wl.max_band(N, 12)))
            for c in range(nch)]
    return plan, x, y, vbw.Batch(rows)


def _probe_shapes(torch, N: int, nch: int, nsamples: int, reps: int, stream) -> dict:
    plan, x, y, batch = _channel_batch(torch, N, nch, nsamples)
    table = []
    best = None
    for w in WARPS:
        for c in CTAS:
            vbw.vbw_tune_set(N, w, c)
            ms = _time_ms(torch, lambda: batch.run(stream), reps, stream)
            gsps = nch * nsamples / (ms * 1e-3) / 1e9
            table.append({"warps": w, "ctas_per_sm": c, "ms": ms, "gsps": gsps})
            if best is None or ms < best["ms"]:
                best = table[-1]
    vbw.vbw_tune_set(N, 0, 0)
    batch.close()
    plan.close()
    return {"warps": best["warps"], "ctas_per_sm": best["ctas_per_sm"], "gsps": best["gsps"], "table": table}


def tune_shapes(torch, Ns=ALL_N, nch: int = 16, nsamples: int = 1 << 21, reps: int = 15) -> dict:
    """{N: {"warps", "ctas_per_sm", "gsps", "table"}} for the single-plan kernel. For N = 2048 that
    is the 64 x 32 four-step kernel (launches that take the split kernel use its own 12-warp
    shape), so its probe runs with the split kernel switched off."""
    stream = torch.cuda.current_stream()
    out = {}
    for N in Ns:
        prev = os.environ.get("VBW_SPLIT2048")
        if N == 2048:
            os.environ["VBW_SPLIT2048"] = "0"
        try:
            out[str(N)] = _probe_shapes(torch, N, nch, nsamples, reps, stream)
        finally:
            if N == 2048:
                if prev is None:
                    os.environ.pop("VBW_SPLIT2048", None)
                else:
                    os.environ["VBW_SPLIT2048"] = prev
    return out


def tune_mixed(torch, batch, reps: int = 10, shares=(0.0, 0.6, 0.7, 0.8, 0.9)) -> dict:
    """Fastest launch mode (and SM share) for one prepared mixed batch."""
    stream = torch.cuda.current_stream()
    table = []
    batch.set_mode(vbw.VBW_BATCH_PER_PLAN)
    table.append({"mode": vbw.VBW_BATCH_PER_PLAN, "share": 0.0,
                  "ms": _time_ms(torch, lambda: batch.run(stream), reps, stream)})
    for sh in shares:
        batch.set_mode(vbw.VBW_BATCH_MIXED, sh)
        table.append({"mode": vbw.VBW_BATCH_MIXED, "share": sh,
                      "ms": _time_ms(torch, lambda: batch.run(stream), reps, stream)})
    best = min(table, key=lambda r: r["ms"])
    batch.set_mode(best["mode"], best["share"])
    return {"mode": best["mode"], "share": best["share"], "table": table}


def apply(cache: dict):
    for N, d in cache.get("shapes", {}).items():
        vbw.vbw_tune_set(int(N), int(d["warps"]), int(d["ctas_per_sm"]))


def load(torch) -> dict | None:
    path = cache_path(torch)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def save(torch, cache: dict) -> str:
    path = cache_path(torch)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return path


def load_or_tune(torch, Ns=ALL_N, force: bool = False) -> dict:
    """Applies the cached shapes for Ns, measuring the ones the cache lacks."""
    cache = None if force else load(torch)
    cache = cache or {"gpu": torch.cuda.get_device_name(), "shapes": {}}
    missing = [N for N in Ns if str(N) not in cache["shapes"]]
    if missing:
        cache["shapes"].update(tune_shapes(torch, missing))
        save(torch, cache)
    apply(cache)
    return cache


if __name__ == "__main__":
    import torch
    from . import build
    build.build()
    c = load_or_tune(torch, force=True)
    print(json.dumps({N: {k: v for k, v in d.items() if k != "table"} for N, d in c["shapes"].items()}))
