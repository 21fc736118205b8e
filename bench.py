"""Benchmark of the GPP self-energy summation on GB300.

Workload: the paper-shaped benchmark instance (number_bands=512, ngpown=1638, ncouls=32768,
nw=3; synthetic seeded inputs standing in for BerkeleyGW's Si-214/Si-510). One step is one
``gpp_sigma`` FP64 call (column gather, main sum, final reduction) on inputs resident in
HBM. The metric is FP64 TFLOP/s from the fixed model FLOP count (159 per band x igp x ig at
nw=3), with the fraction of the FP64 peak measured in the same run by DFMA-chain kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpp|reference]

Prints one JSON line on rank 0. ``--impl reference`` times the CPU oracle (the plain FP64
reference implementation) on a band sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GPP FP64 TFLOP/s & %peak at 512x1638x32768x3; FP32-bulk speedup at <=1e-6 err"
UNIT = "TFLOP/s"
WORKLOAD = "gpp_benchmark_B512_P1638_G32768_nw3"
ORACLE_SAMPLE_BANDS = 8          # bands per step of the reference arm (the oracle)
CPU_BASELINE_SAMPLE_BANDS = 32   # bands of the cpu_baseline sample (~10 s on 16 cores)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpp", "reference"], default="gpp")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint and batched measurements")
    ap.add_argument("--pipe-rates", action="store_true",
                    help="print the throughput of every instruction kind of the library's "
                         "throughput kernels (machine characterisation) and exit")
    ap.add_argument("--profile-case", choices=["fwd_f64", "fwd_f64_b512", "fwd_f32",
                                               "fwd_f32_sorted", "bwd", "batched"],
                    default=None,
                    help="run only a small case three times, for ncu captures: fwd_f64, "
                         "fwd_f32 and bwd use B=64, P=256, G=32768, nw=3 (0.3 GB of (igp, ig) "
                         "arrays, more than L2); fwd_f64_b512 B=512, P=64, G=32768 (the "
                         "benchmark's band count and G on 64 columns, 0.3 GB); "
                         "fwd_f32_sorted B=256, P=128 (the FP32-bulk "
                         "kernel sorts from 128 bands); batched uses 8 instances with G "
                         "in [2048, 32768] and B=32")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def base_config(args, world):
    from paper_2008_11326_gb300 import inputs
    c = inputs.CONFIGS["benchmark"]
    return {"workload": WORKLOAD, "number_bands": c["number_bands"], "ngpown": c["ngpown"],
            "ncouls": c["ncouls"], "nw": c["nw"], "nvband": c["nvband"], "occ_mode": "all",
            "seed": c["seed"], "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "inputs (2.0 GB) larger than L2 (129 MB); no flush needed"}


# ----------------------------------------------------------------------------- oracle leg

def oracle_sample(prob, bands: int, nthreads: int, want_result: bool = False):
    """Time the CPU oracle, as it stands, on the first ``bands`` bands of the instance."""
    import oracle
    from paper_2008_11326_gb300 import inputs
    sub = prob.bands(slice(0, bands))
    t0 = time.perf_counter()
    res = oracle.sigma(sub, nthreads=nthreads)
    dt = time.perf_counter() - t0
    flops = inputs.model_flops(sub.number_bands, sub.ngpown, sub.ncouls, sub.nw)
    if want_result:
        return flops / dt / 1e12, dt, sub, res
    return flops / dt / 1e12, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2008_11326_gb300 import inputs
    oracle.build()
    prob = inputs.config("benchmark")
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(prob, 1, cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample(prob, ORACLE_SAMPLE_BANDS, cores)
        times.append(dt)
    flops = inputs.model_flops(ORACLE_SAMPLE_BANDS, prob.ngpown, prob.ncouls, prob.nw)
    t = statistics.mean(times)
    value = flops / t / 1e12
    sample = (f"first {ORACLE_SAMPLE_BANDS} of 512 bands of the benchmark instance per step "
              f"({flops:.3e} model FLOP), OpenMP over igp")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # let nvidia-smi finish starting (its driver initialisation delayed the host-to-device
        # copies of a timed region that began at the same moment) before the caller times
        deadline = time.perf_counter() + 5.0
        while (time.perf_counter() < deadline and self.proc.poll() is None
               and os.path.getsize(self.file.name) == 0):
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        pw = [num(r[3]) for r in rows if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows),
                "reasons": reasons}


def recorded_counters():
    """The committed ncu record of the main kernel (DRAM bytes per full-size launch,
    executed FP64 FLOP per unit), if the kernel's sources are unchanged since (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    return rec if h.hexdigest() == rec["sources_sha256"] else None


def measure_peaks(torch, gpp, device):
    """FP64 (DFMA) and FP32 (FFMA) peaks from the library's throughput kernels."""
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    sink = torch.zeros(1, dtype=torch.float64, device=device)
    out = {}
    for kind, iters, bps in (("dfma", 256, 4), ("ffma", 8192, 8), ("drcp", 128, 4)):
        blocks, threads = sms * bps, 256
        gpp.peak_launch(kind, iters // 8, blocks, threads, sink)  # warm
        torch.cuda.synchronize(device)
        best = 0.0
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = gpp.peak_launch(kind, iters, blocks, threads, sink)
            e1.record()
            e1.synchronize()
            best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
        out[kind] = best
    return {"fp64_tflops": 2 * out["dfma"] / 1e12, "fp32_tflops": 2 * out["ffma"] / 1e12,
            "fp64_rcp_per_s": out["drcp"], "sms": sms}


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def measure_adjoint(torch, gpp, inputs, device, reps=3):
    """Adjoint workload (B=128, P=410, G=8192, nw=3): backward time against forward time."""
    prob = inputs.config("adjoint")
    ga, gs = inputs.cotangents(3, prob.nw)
    dp = gpp.DeviceProblem.from_host(prob, device=device)
    ga_t = torch.from_numpy(ga).to(device)
    gs_t = torch.from_numpy(gs).to(device)
    gpp.sigma(dp)
    gpp.sigma_backward(dp, ga_t, gs_t)
    torch.cuda.synchronize(device)
    fwd, bwd = [], []
    for _ in range(reps):
        e = _events(torch, 3)
        e[0].record()
        gpp.sigma(dp)
        e[1].record()
        gpp.sigma_backward(dp, ga_t, gs_t)
        e[2].record()
        e[2].synchronize()
        fwd.append(e[0].elapsed_time(e[1]))
        bwd.append(e[1].elapsed_time(e[2]))
    f, b = min(fwd), min(bwd)
    return {"workload": "B128_P410_G8192_nw3", "forward_ms": f, "backward_ms": b,
            "backward_over_forward": b / f, "target_max_ratio": 3.0}


BATCH_REPS = 5             # timed repetitions of every arm of the batched comparison
BATCH_FP64_BANDS = 64      # bands per instance in the FP64 batched comparison


def _spread(ms):
    return {"median_ms": statistics.median(ms), "min_ms": min(ms), "max_ms": max(ms),
            "reps": len(ms)}


def measure_batched(torch, gpp, inputs, device, reps=BATCH_REPS):
    """64 uneven instances: one graph-replayed persistent launch (autotuned tile shape)
    against loops of per-instance gpp_sigma calls, both at the default tile and at the tuned
    one, each arm timed ``reps`` times (median and spread). FP32-bulk on the full instances;
    FP64 on the first BATCH_FP64_BANDS bands of every instance (the full FP64 batch takes
    ~24 s per run)."""
    from paper_2008_11326_gb300 import autotune
    shapes = inputs.batched_shapes()
    full = [gpp.DeviceProblem(**inputs.make_device_arrays(**s, device=device)) for s in shapes]

    def first_bands(d, nb):
        nb = min(nb, d.number_bands)
        return gpp.DeviceProblem(nb, d.nvband, d.ncouls, d.ngpown, d.nw, d.aqsmtemp[:nb],
                                 d.aqsntemp[:nb], d.I_eps_array, d.wtilde_array, d.vcoul,
                                 d.inv_igp_index, d.indinv, d.wx_array[:nb])

    out = {"workload": "64 instances, G log-uniform in [2048, 32768], P = G/20, B ~ U{64..512}, "
                       "nw=3 (inputs drawn on the device)"}

    def timed(fn):
        fn()
        torch.cuda.synchronize(device)
        ms = []
        for _ in range(reps):
            e = _events(torch, 2)
            e[0].record()
            fn()
            e[1].record()
            e[1].synchronize()
            ms.append(e[0].elapsed_time(e[1]))
        return ms

    for precision in ("fp64", "fp32_bulk"):
        dps = [first_bands(d, BATCH_FP64_BANDS) for d in full] if precision == "fp64" else full
        if precision == "fp32_bulk":
            for d in dps:
                d.make_c64()
        units = sum(d.number_bands * d.ngpown * d.ncouls for d in dps)
        flops = sum(inputs.model_flops(d.number_bands, d.ngpown, d.ncouls, d.nw) for d in dps)
        tuned = autotune.tune_batched(dps, precision=precision, reps=1,
                                      proxy_fraction=1 / 16 if precision == "fp64" else 1 / 32)
        tile = dict(block_threads=tuned["block_threads"], ig_per_thread=tuned["ig_per_thread"])
        plan = gpp.BatchedPlan(dps, use_graph=True, precision=precision, **tile)
        g_ms = timed(plan.run)
        batched_res = [torch.cat(o).cpu() for o in plan.outputs]
        plan.close()
        arms = {}
        loop_res = None
        for name, opts in (("loop_default_tile", {}), ("loop_tuned_tile", tile)):
            wss = [torch.empty(gpp.workspace_size(d, precision=precision, **opts),
                               dtype=torch.uint8, device=device) for d in dps]
            res = []

            def loop():
                res[:] = [gpp.sigma(d, workspace=w, precision=precision, **opts)
                          for d, w in zip(dps, wss)]
            arms[name] = timed(loop)
            if name == "loop_default_tile":
                loop_res = [torch.cat(r).cpu() for r in res]
            del wss
        diff = max(float(((a - b).abs() / b.abs()).max()) for a, b in zip(batched_res, loop_res))
        g_med = statistics.median(g_ms)
        out[precision] = {
            "bands": f"first {BATCH_FP64_BANDS} of each instance" if precision == "fp64" else "all",
            "units": units, "model_flop": flops,
            "graph": _spread(g_ms),
            **{k: _spread(v) for k, v in arms.items()},
            "speedup_vs_loop_default_tile": statistics.median(arms["loop_default_tile"]) / g_med,
            "speedup_vs_loop_tuned_tile": statistics.median(arms["loop_tuned_tile"]) / g_med,
            "tflops_model_graph": flops / (g_med * 1e-3) / 1e12,
            "tile": {**tile, "from_cache": tuned["cached"]},
            "max_rel_diff_vs_loop": diff}
    del full
    torch.cuda.empty_cache()
    return out


def measure_large(torch, gpp, inputs, device):
    """Three times the benchmark on every loop (B=1536, P=4915, G=98304, nw=3), drawn on the
    device: the full FP32-bulk sum, and the FP64 sum on its first 32 bands (the full FP64
    sum takes over a minute)."""
    c = inputs.CONFIGS["large"]
    dp = gpp.DeviceProblem(**inputs.make_device_arrays(**c, device=device))
    dp.make_c64()
    B, P, G, W = dp.number_bands, dp.ngpown, dp.ncouls, dp.nw
    nb = 32
    sub = gpp.DeviceProblem(nb, dp.nvband, G, P, W, dp.aqsmtemp[:nb], dp.aqsntemp[:nb],
                            dp.I_eps_array, dp.wtilde_array, dp.vcoul, dp.inv_igp_index,
                            dp.indinv, dp.wx_array[:nb])
    out = {"workload": f"B{B}_P{P}_G{G}_nw{W} (inputs drawn on the device)",
           "input_gb": (2 * B * G + 2 * P * G) * 16 / 1e9}
    for name, prob, prec in (("fp32_bulk", dp, "fp32_bulk"), ("fp64_first_32_bands", sub, "fp64")):
        ws = torch.empty(gpp.workspace_size(prob, precision=prec), dtype=torch.uint8,
                         device=device)
        gpp.sigma(prob, workspace=ws, precision=prec)
        e = _events(torch, 2)
        e[0].record()
        gpp.sigma(prob, workspace=ws, precision=prec)
        e[1].record()
        e[1].synchronize()
        ms = e[0].elapsed_time(e[1])
        flops = inputs.model_flops(prob.number_bands, P, G, W)
        out[name] = {"ms": ms, "tflops_model": flops / (ms * 1e-3) / 1e12}
        del ws
    del dp, sub
    torch.cuda.empty_cache()
    return out


def max_over_ranks(value: float, pg=None, device="cpu") -> float:
    """The largest of the ranks' values (each rank passes its own; all ranks get the
    result). Without a process group, the value itself."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank: float, seconds_per_step: float, world: int) -> float:
    """Every rank sums its own copy of the instance (replicas, weak scaling): the job does
    world x the work in the slowest rank's time."""
    return world * flops_per_rank / seconds_per_step / 1e12


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2008_11326_gb300 import gpp, inputs

    rank, world, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    prob = inputs.config("benchmark")
    dp = gpp.DeviceProblem.from_host(prob, device=device)
    flops = inputs.model_flops(prob.number_bands, prob.ngpown, prob.ncouls, prob.nw)
    # bytes moved host -> device per end-to-end step: every input, except that the host
    # entry point's gather reads only aqsmtemp's gathered columns (B x P elements) in place
    # when the array is page-locked (as the benchmark's host arrays are)
    h2d_bytes = (prob.nbytes() - prob.aqsmtemp.nbytes
                 + prob.number_bands * prob.ngpown * 16)
    ws = torch.empty(gpp.workspace_size(dp), dtype=torch.uint8, device=device)
    ach = torch.empty(prob.nw, dtype=torch.complex128, device=device)
    asx = torch.empty(prob.nw, dtype=torch.complex128, device=device)

    peaks = measure_peaks(torch, gpp, device)

    K, W = args.steps, args.warmup
    stage = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for evs in stage:  # materialise the events so their handles exist
        for e in evs:
            e.record()
    torch.cuda.synchronize(device)

    for _ in range(W):
        gpp.sigma(dp, out=(ach, asx), workspace=ws)
    torch.cuda.synchronize(device)
    ref_a = ach.cpu().numpy().copy()
    ref_s = asx.cpu().numpy().copy()

    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(device)
    with ClockSampler(local) as clk:
        t0.record()
        for k in range(K):
            gpp.sigma(dp, out=(ach, asx), workspace=ws, stage_events=stage[k])
        t1.record()
        torch.cuda.synchronize(device)
    barrier()
    total_ms = t0.elapsed_time(t1)
    main_ms = [stage[k][1].elapsed_time(stage[k][2]) for k in range(K)]
    step_ms_each = [stage[k][0].elapsed_time(stage[k][3]) for k in range(K)]
    step_ms = max_over_ranks(total_ms / K, pg, device)
    value = whole_job_tflops(flops, step_ms * 1e-3, world)
    deterministic = bool(np.array_equal(ach.cpu().numpy(), ref_a) and
                         np.array_equal(asx.cpu().numpy(), ref_s))

    # end to end through the host-array entry point: H2D of every input, sum, D2H (right
    # after the device-resident steps, on the same GPU state)
    hp = gpp.DeviceProblem.from_host(prob, device="cpu", pin=True)
    if not hp.aqsmtemp.is_pinned():   # then the host entry point copies all of aqsmtemp
        h2d_bytes = prob.nbytes()
    hws = torch.empty(gpp.host_workspace_size(hp), dtype=torch.uint8, device=device)
    hout = (torch.empty(prob.nw, dtype=torch.complex128).pin_memory(),
            torch.empty(prob.nw, dtype=torch.complex128).pin_memory())
    gpp.sigma_host(hp, workspace=hws, out=hout)
    # the box's pinned host-to-device rate right now (one 268 MB copy of aqsntemp): the
    # host entry point's copies overlap the sum, but the first chunk and aqsmtemp (which
    # the column gather needs) are waited for
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    probe_dst = torch.empty_like(hp.aqsntemp, device=device)
    h0.record()
    probe_dst.copy_(hp.aqsntemp, non_blocking=True)
    h1.record()
    torch.cuda.synchronize(device)
    h2d_gbs = hp.aqsntemp.numel() * 16 / (h0.elapsed_time(h1) * 1e-3) / 1e9
    del probe_dst
    e2e_steps = max(1, args.e2e_steps)
    e2e_stage = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(e2e_steps)]
    e2e_start = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps)]
    for evs in e2e_stage:
        for e in evs:
            e.record()
    barrier()
    torch.cuda.synchronize(device)
    with ClockSampler(local) as e2e_clk:
        s0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_start[k].record()
            gpp.sigma_host(hp, workspace=hws, out=hout, stage_events=e2e_stage[k])
        e2e_s = (time.perf_counter() - s0) / e2e_steps
    barrier()
    e2e_s = max_over_ranks(e2e_s, pg, device)
    e2e_ok = bool(np.array_equal(hout[0].numpy(), ref_a) and np.array_equal(hout[1].numpy(), ref_s))
    e2e_h2d_ms = statistics.mean(e2e_start[k].elapsed_time(e2e_stage[k][0]) for k in range(e2e_steps))
    e2e_main_ms = statistics.mean(e2e_stage[k][1].elapsed_time(e2e_stage[k][2])
                                  for k in range(e2e_steps))
    del hws, hp
    torch.cuda.empty_cache()

    # FP32-bulk forward on the same instance: speedup over FP64 and error against it.
    # (a) each call converts aqsntemp to complex64 in its own workspace (no copy kept by the
    # caller); (b) the caller keeps the copy, made once by the library's conversion kernel.
    def time_f32(dpx, ws_x):
        for _ in range(W):
            gpp.sigma(dpx, out=(ach, asx), workspace=ws_x, precision="fp32_bulk")
        st = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        for evs in st:
            for e in evs:
                e.record()
        torch.cuda.synchronize(device)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for k in range(K):
            gpp.sigma(dpx, out=(ach, asx), workspace=ws_x, precision="fp32_bulk",
                      stage_events=st[k])
        f1.record()
        torch.cuda.synchronize(device)
        return (f0.elapsed_time(f1) / K,
                statistics.mean(st[k][0].elapsed_time(st[k][1]) for k in range(K)),
                statistics.mean(st[k][1].elapsed_time(st[k][2]) for k in range(K)))

    import dataclasses
    dp_nc = dataclasses.replace(dp, aqsntemp_c64=None)
    ws32 = torch.empty(gpp.workspace_size(dp_nc, precision="fp32_bulk"), dtype=torch.uint8,
                       device=device)
    f32c_step_ms, f32c_prep_ms, _ = time_f32(dp_nc, ws32)
    got_c = np.concatenate([ach.cpu().numpy(), asx.cpu().numpy()])
    del ws32, dp_nc
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record()
    dp.make_c64()
    c1.record()
    torch.cuda.synchronize(device)
    conv_ms = c0.elapsed_time(c1)
    ws32 = torch.empty(gpp.workspace_size(dp, precision="fp32_bulk"), dtype=torch.uint8,
                       device=device)
    f32_step_ms, f32_prep_ms, f32_main_ms = time_f32(dp, ws32)
    got = np.concatenate([ach.cpu().numpy(), asx.cpu().numpy()])
    ref = np.concatenate([ref_a, ref_s])
    f32_err = float(np.max(np.abs(got - ref) / np.abs(ref)))
    conv_bytes = prob.number_bands * prob.ncouls * (16 + 8)
    fp32_bulk = {"ms_per_step": f32_step_ms, "main_kernel_ms": f32_main_ms,
                 "tflops_model": flops / (f32_step_ms * 1e-3) / 1e12,
                 "speedup_vs_fp64": step_ms / f32_step_ms,
                 "ms_per_step_converting_in_call": f32c_step_ms,
                 "speedup_incl_c64_conversion": step_ms / f32c_step_ms,
                 "gather_ms": f32_prep_ms,
                 "gather_plus_conversion_ms": f32c_prep_ms,
                 "c64_conversion_ms": conv_ms,
                 "c64_conversion_gbs": conv_bytes / (conv_ms * 1e-3) / 1e9,
                 "conversion_in_call_bit_equal": bool(np.array_equal(got_c, got)),
                 "max_rel_err_vs_fp64_gpu": f32_err,
                 "per_output_rel_err": [float(v) for v in np.abs(got - ref) / np.abs(ref)],
                 "fp32_peak_frac_model": flops / (f32_main_ms * 1e-3) / 1e12 / peaks["fp32_tflops"]}
    del ws32

    adjoint = None if args.no_extras else measure_adjoint(torch, gpp, inputs, device)
    batched = None if args.no_extras else measure_batched(torch, gpp, inputs, device)
    large = None if args.no_extras else measure_large(torch, gpp, inputs, device)

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    main_avg_s = statistics.mean(main_ms) * 1e-3
    achieved = flops / main_avg_s / 1e12
    rec = recorded_counters()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peaks["fp64_tflops"],
                "unit": "TFLOP/s", "frac": achieved / peaks["fp64_tflops"],
                "traffic": rec["traffic_bytes_per_launch"] if rec else None,
                "algorithmic_bytes": 2.0 * prob.ngpown * prob.ncouls * 16 + prob.number_bands * prob.ncouls * 16
                + prob.number_bands * prob.ngpown * 16 + prob.ncouls * 8 + prob.number_bands * prob.nw * 8,
                "kernel": "gpp_batched_kernel_f64<3> (main sum of gpp_sigma)",
                "peak_source": "DFMA-chain throughput kernel measured in this run, all SMs "
                               "(FP64 pipe; FMA = 2 FLOP)",
                "achieved_source": "model FLOP (159 per band x igp x ig) / mean CUDA-event "
                                   "duration of the main kernel over the timed steps"}
    if rec and "executed" in rec:
        # The model FLOP count above the executed one is why frac exceeds 1: the kernel
        # executes fewer FP64 FLOPs per unit than the model counts (one reciprocal for both
        # denominators, I w applied once per G-vector).
        ex = rec["executed"]
        exe = achieved * ex["fp64_flop_per_unit"] / inputs.model_flops(1, 1, 1, prob.nw)
        adj = (1 + ex["fma_ratio"]) / 2 * peaks["fp64_tflops"]
        roofline["executed"] = {"flop_per_unit": ex["fp64_flop_per_unit"],
                                "achieved": exe, "frac": exe / peaks["fp64_tflops"],
                                "fma_ratio": ex["fma_ratio"], "fma_adjusted_peak": adj,
                                "frac_of_fma_adjusted_peak": exe / adj,
                                "source": "ncu SASS counters of the same kernel, " + ex["workload"]}
        # the same two fractions at the top of the roofline object: executed FP64 FLOP/s
        # against the DFMA-chain peak, and against the FMA-adjusted peak (paper §III v8)
        roofline["frac_executed"] = exe / peaks["fp64_tflops"]
        roofline["frac_fma_adjusted"] = exe / adj

    cpu = None
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, dt, sub, ref = oracle_sample(prob, CPU_BASELINE_SAMPLE_BANDS, cores, want_result=True)
        v1, dt1 = oracle_sample(prob, 1, 1)
        ref = np.concatenate(ref)
        parity, scaled, per_output = {}, {}, {}
        sdp = gpp.DeviceProblem.from_host(sub, device=device, c64=True)
        for prec in ("fp64", "fp32_bulk"):
            a, s = gpp.sigma(sdp, precision=prec)
            got = np.concatenate([a.cpu().numpy(), s.cpu().numpy()])
            parity[prec] = float(np.max(np.abs(got - ref) / np.abs(ref)))
            # the same errors against the sample's output scale (its largest |output|): an
            # output much smaller than the others (cancellation over bands) has a relative
            # error above the terms' rounding level
            scaled[prec] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
            per_output[prec] = [float(e) for e in np.abs(got - ref) / np.abs(ref)]
        del sdp
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {CPU_BASELINE_SAMPLE_BANDS} of 512 bands of the benchmark instance "
                         f"({dt:.1f} s, OpenMP over igp on all host cores)",
               "value_1_core": v1,
               "sample_1_core": f"first band of the benchmark instance ({dt1:.1f} s, one thread)",
               "full_instance_s_extrapolated": dt * prob.number_bands / CPU_BASELINE_SAMPLE_BANDS,
               "gpu_max_rel_err_on_sample": parity,
               "gpu_max_err_on_sample_vs_largest_output": scaled,
               "gpu_rel_err_on_sample_per_output": per_output,
               "sample_output_magnitudes": [float(a) for a in np.abs(ref)]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config(args, world),
            "fp64_peak_frac": value / world / peaks["fp64_tflops"],
            "main_kernel_ms": statistics.mean(main_ms),
            "step_ms_median": statistics.median(step_ms_each),
            "step_ms_spread": [min(step_ms_each), max(step_ms_each)],
            "peaks_measured": peaks,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_tflops(flops, e2e_s, world), "unit": UNIT,
                    "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": 2 * prob.nw * 16,
                    "steps": e2e_steps, "matches_device_result": e2e_ok,
                    "h2d_ms": e2e_h2d_ms, "main_kernel_ms": e2e_main_ms,
                    "pinned_h2d_gbs": h2d_gbs,
                    "clocks": e2e_clk.summary()},
            "gpu_launches": 3 * K,
            "deterministic_across_steps": deterministic,
            "clocks": clk.summary(),
            "fp32_bulk": fp32_bulk,
            "adjoint": adjoint,
            "batched": batched,
            "large": large}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_profile_case(args):
    import torch

    from paper_2008_11326_gb300 import gpp, inputs
    if args.profile_case == "batched":
        shapes = inputs.batched_shapes(8)
        dps = [gpp.DeviceProblem(**inputs.make_device_arrays(**dict(s, number_bands=32),
                                                             device="cuda")) for s in shapes]
        plan = gpp.BatchedPlan(dps, use_graph=False, block_threads=64, ig_per_thread=4)
        for _ in range(3):
            outs = plan.run()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "batched", "achtemp0": str(outs[0][0][0].item())}))
        return 0
    if args.profile_case == "fwd_f32_sorted":   # enough bands for the tile sort by Re w
        prob = inputs.make_problem(256, 2, 32768, 128, 3, seed=1)
    elif args.profile_case == "fwd_f64_b512":   # the benchmark's B and G, 64 columns
        prob = inputs.make_problem(512, 2, 32768, 64, 3, seed=1)
    else:
        prob = inputs.make_problem(64, 2, 32768, 256, 3, seed=1)
    precision = "fp32_bulk" if args.profile_case.startswith("fwd_f32") else "fp64"
    dp = gpp.DeviceProblem.from_host(prob, device="cuda", c64=precision == "fp32_bulk")
    if args.profile_case == "bwd":
        ga, gs = inputs.cotangents(3, prob.nw)
        for _ in range(3):
            g = gpp.sigma_backward(dp, torch.from_numpy(ga).cuda(), torch.from_numpy(gs).cuda())
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "bwd", "grad0": str(g["wtilde"][0, 0].item())}))
        return 0
    for _ in range(3):
        ach, asx = gpp.sigma(dp, precision=precision)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "achtemp0": str(ach[0].item())}))
    return 0


def run_pipe_rates():
    """Throughput of each instruction kind on all SMs (8 independent chains per thread)."""
    import torch

    from paper_2008_11326_gb300 import gpp
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {}
    for kind, iters in (("dfma", 256), ("dadd", 256), ("dmul", 256), ("drcp", 128),
                        ("drcp_approx", 512), ("drcp_rn", 64), ("f2f", 256), ("ffma", 8192),
                        ("fsetp", 8192), ("isel", 8192), ("fsel", 8192)):
        blocks, threads = sms * 4, 256
        gpp.peak_launch(kind, max(iters // 8, 1), blocks, threads, sink)
        torch.cuda.synchronize(dev)
        best = 0.0
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = gpp.peak_launch(kind, iters, blocks, threads, sink)
            e1.record()
            e1.synchronize()
            best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
        out[kind] = {"ops_per_s": best, "per_clk_per_sm_at_2070MHz": best / (sms * 2.07e9)}
    print(json.dumps({"pipe_rates": out, "sms": sms}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.pipe_rates:
        return run_pipe_rates()
    if args.profile_case:
        return run_profile_case(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
