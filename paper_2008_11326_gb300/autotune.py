"""Tile-shape autotuner for the batched GPP launch.

For a batch of instances it times each candidate (threads per CTA, G-vectors per thread
per tile) on a proxy of the batch -- the same instances restricted to a fraction of their
igp columns (at least one), which keeps every tile's work (all bands x the tile's
G-vectors) and shortens the batch -- and keeps the fastest. Results are cached in a JSON
file (``$GPP_TUNE_CACHE``, default ``~/.cache/gpp/tune.json``) keyed by device, precision,
nw and the batch's shapes.
"""

from __future__ import annotations

import hashlib
import json
import math
import os

import torch

from . import gpp

CANDIDATES = tuple((bt, k) for bt in (64, 128, 256) for k in (1, 2, 4, 8))


def cache_path() -> str:
    return os.environ.get("GPP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gpp", "tune.json"))


def batch_key(dps, precision: str, occ_mode: str) -> str:
    shapes = sorted((d.number_bands, d.ngpown, d.ncouls) for d in dps)
    sig = hashlib.sha1(json.dumps(shapes).encode()).hexdigest()[:16]
    dev = torch.cuda.get_device_name(dps[0].device)
    return f"{dev}|{precision}|{occ_mode}|nw{dps[0].nw}|n{len(dps)}|{sig}"


def _proxy(d: gpp.DeviceProblem, fraction: float) -> gpp.DeviceProblem:
    """The first ceil(fraction * ngpown) columns of ``d`` (views)."""
    p = min(d.ngpown, max(1, math.ceil(d.ngpown * fraction)))
    return gpp.DeviceProblem(d.number_bands, d.nvband, d.ncouls, p, d.nw, d.aqsmtemp,
                             d.aqsntemp, d.I_eps_array[:p], d.wtilde_array[:p], d.vcoul,
                             d.inv_igp_index[:p], d.indinv, d.wx_array, d.aqsntemp_c64)


def time_plan(plan: gpp.BatchedPlan, reps: int) -> float:
    plan.run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batched(dps, precision: str = "fp64", occ_mode: str = "all",
                 proxy_fraction: float = 1.0 / 32, reps: int = 2, candidates=CANDIDATES,
                 use_cache: bool = True) -> dict:
    """Best ``{"block_threads", "ig_per_thread"}`` for this batch (and the timings)."""
    key = batch_key(dps, precision, occ_mode)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key], cached=True)
    proxy = [_proxy(d, proxy_fraction) for d in dps]
    timings = {}
    for bt, k in candidates:
        plan = gpp.BatchedPlan(proxy, use_graph=True, precision=precision, occ_mode=occ_mode,
                               block_threads=bt, ig_per_thread=k)
        timings[f"{bt}x{k}"] = time_plan(plan, reps)
        plan.close()
    best = min(timings, key=timings.get)
    bt, k = (int(v) for v in best.split("x"))
    result = {"block_threads": bt, "ig_per_thread": k, "proxy_ms": timings}
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        cache[key] = result
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return dict(result, cached=False)
