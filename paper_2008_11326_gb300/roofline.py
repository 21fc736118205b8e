"""Hierarchical roofline from Nsight Compute counters, in the paper's style (§II-B, Eqs. 1-2).

For one captured kernel launch it forms
  * the executed FLOPs per precision from the SASS instruction counters: adds and
    multiplies count 1, fused multiply-adds 2, and GB300's paired FP32 instructions
    (FADD2 / FMUL2 / FFMA2) twice that;
  * the bytes moved at each level: L1/TEX (l1tex__t_bytes), L2 (lts__t_bytes) and DRAM
    (dram__bytes_read + dram__bytes_write);
  * the arithmetic intensity at each level (FLOPs / bytes) and the achieved FLOP/s (FLOPs /
    the launch's duration);
  * the FMA ratio f = FMA / (add + mul + FMA) of the dominant precision and the FMA-adjusted
    peak (1 + f) / 2 x peak: a kernel that issues one instruction per cycle with that mix
    reaches it (the paper's §III v8 analysis);
and compares them with the peaks the caller passes (measured throughput of the FP pipes,
measured memory bandwidth).

It is a measurement tool beside the library: ``ncu_command`` builds the capture command,
``load_raw_csv`` reads ``ncu -i REPORT --page raw --csv``, ``summarize`` computes the
roofline and ``to_markdown`` renders it; ``collect`` runs the capture and the first three
steps in one call. ``python -m paper_2008_11326_gb300.roofline REPORT
--fp64-peak-tflops X --hbm-gbs Y`` does all three on an existing report.
"""

from __future__ import annotations

import argparse
import csv
import io
import json
import subprocess
import sys

_OPS = {
    "fp64": [("dadd", 1), ("dmul", 1), ("dfma", 2)],
    "fp32": [("fadd", 1), ("fmul", 1), ("ffma", 2), ("fadd2", 2), ("fmul2", 2), ("ffma2", 4)],
}

METRICS = (
    ["gpu__time_duration.sum", "sm__cycles_elapsed.avg.per_second",
     "l1tex__t_bytes.sum", "lts__t_bytes.sum", "dram__bytes_read.sum",
     "dram__bytes_write.sum", "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
     "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"]
    + [f"smsp__sass_thread_inst_executed_op_{op}_pred_on.sum"
       for ops in _OPS.values() for op, _ in ops])

_SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12,
          "nsecond": 1e-9, "ns": 1e-9, "usecond": 1e-6, "us": 1e-6, "msecond": 1e-3,
          "ms": 1e-3, "second": 1.0, "s": 1.0, "inst": 1.0, "": 1.0, "%": 1.0,
          "cycle/second": 1.0, "cycle/nsecond": 1e9, "cycle/usecond": 1e6,
          "cycle/msecond": 1e3, "Kcycle/second": 1e3, "Mcycle/second": 1e6,
          "Gcycle/second": 1e9, "hz": 1.0, "Khz": 1e3, "Mhz": 1e6, "Ghz": 1e9,
          "Kinst": 1e3, "Minst": 1e6, "Ginst": 1e9}


def ncu_command(cmd, kernel_regex: str, report: str, skip: int = 0, count: int = 1,
                extra_metrics=()):
    """The capture command for the roofline metrics of ``count`` launches of the kernels
    matching ``kernel_regex`` (after ``skip``); the clocks are left to the GPU."""
    return (["ncu", "--metrics", ",".join(list(METRICS) + list(extra_metrics)),
             "--clock-control", "none", "-k", f"regex:{kernel_regex}", "-s", str(skip),
             "-c", str(count), "-o", report] + list(cmd))


def load_raw_csv(text: str, launch: int = 0) -> dict:
    """Metric name -> value in base units (bytes, seconds, instructions) for one launch of
    an ``ncu --page raw --csv`` export (the first row is names, the second units)."""
    rows = [r for r in csv.reader(io.StringIO(text)) if r]
    if len(rows) < 3:
        raise ValueError("not an ncu raw-page CSV export with at least one launch")
    names, units, vals = rows[0], rows[1], rows[2 + launch]
    out = {}
    for n, u, v in zip(names, units, vals):
        try:
            x = float(v.replace(",", ""))
        except ValueError:
            continue
        if u in _SCALE:  # metrics in other units are not used here
            out[n] = x * _SCALE[u]
    return out


def report_metrics(report: str, launch: int = 0, run=subprocess.run) -> dict:
    text = run(["ncu", "-i", report, "--page", "raw", "--csv"], check=True,
               capture_output=True, text=True).stdout
    return load_raw_csv(text, launch)


def collect(cmd, kernel_regex: str, report: str, peaks: dict, units: float | None = None,
            skip: int = 0, count: int = 1, launch: int = 0, run=subprocess.run) -> dict:
    """Capture, read back and summarise in one call: runs ``ncu_command`` on ``cmd`` (which
    must already have exited 0 on the same GPU without ncu), then ``summarize`` on launch
    ``launch`` of the report. Capture a small case of the kernel: the metric set takes
    several replay passes per launch."""
    run(ncu_command(cmd, kernel_regex, report, skip, count), check=True)
    path = report if report.endswith(".ncu-rep") else report + ".ncu-rep"
    return summarize(report_metrics(path, launch, run), peaks, units)


def _count(m, op):
    for prefix in ("smsp", "sm"):
        k = f"{prefix}__sass_thread_inst_executed_op_{op}_pred_on.sum"
        if k in m:
            return m[k]
    return 0.0


def summarize(m: dict, peaks: dict, units: float | None = None) -> dict:
    """The roofline of one launch. ``peaks``: any of fp64_tflops, fp32_tflops (FMA-chain
    throughput, 2 FLOP per FMA), hbm_gbs. ``units``: work units of the launch, for
    per-unit counts."""
    t = m["gpu__time_duration.sum"]
    out = {"duration_s": t}
    levels = {"l1": m.get("l1tex__t_bytes.sum"), "l2": m.get("lts__t_bytes.sum"),
              "dram": (m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"])
              if "dram__bytes_read.sum" in m else None}
    out["bytes"] = levels
    for prec, ops in _OPS.items():
        counts = {op: _count(m, op) for op, _ in ops}
        flops = sum(counts[op] * w for op, w in ops)
        r = {"flops": flops, "tflops": flops / t / 1e12 if t > 0 else 0.0,
             "instructions": counts,
             "ai": {lv: (flops / b if b else None) for lv, b in levels.items()}}
        fma = sum(v for k, v in counts.items() if "fma" in k)
        total = sum(counts.values())
        if total:
            f = fma / total
            r["fma_ratio"] = f
            peak = peaks.get(f"{prec}_tflops")
            if peak:
                r["peak_tflops"] = peak
                r["fma_adjusted_peak_tflops"] = (1 + f) / 2 * peak
                r["frac_of_peak"] = r["tflops"] / peak
                r["frac_of_fma_adjusted_peak"] = r["tflops"] / r["fma_adjusted_peak_tflops"]
        if units:
            r["instructions_per_unit"] = {k: v / units for k, v in counts.items()}
            r["flops_per_unit"] = flops / units
        out[prec] = r
    if levels["dram"] is not None and t > 0:
        out["dram_gbs"] = levels["dram"] / t / 1e9
        if peaks.get("hbm_gbs"):
            out["dram_frac_of_peak"] = out["dram_gbs"] / peaks["hbm_gbs"]
    for k in ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
              "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"):
        if k in m:
            out[k.split("__")[1].split("_cycles")[0] + "_busy_pct"] = m[k]
    return out


def to_markdown(s: dict, title: str = "Hierarchical roofline") -> str:
    lines = [f"## {title}", "", f"duration {s['duration_s'] * 1e3:.3f} ms", ""]
    lines += ["| level | bytes | FP64 FLOP/B | FP32 FLOP/B |", "|---|---:|---:|---:|"]
    for lv in ("l1", "l2", "dram"):
        b = s["bytes"][lv]
        if b is None:
            continue
        ai64, ai32 = s["fp64"]["ai"][lv], s["fp32"]["ai"][lv]
        lines.append(f"| {lv} | {b:.4g} | {ai64 if ai64 is None else f'{ai64:.4g}'} | "
                     f"{ai32 if ai32 is None else f'{ai32:.4g}'} |")
    lines += ["", "| precision | executed FLOP | TFLOP/s | FMA ratio | peak | FMA-adjusted peak |"
              " of peak | of adjusted |", "|---|---:|---:|---:|---:|---:|---:|---:|"]
    for prec in ("fp64", "fp32"):
        r = s[prec]
        if not r["flops"]:
            continue
        g = lambda k, f="{:.4g}": f.format(r[k]) if k in r else "-"  # noqa: E731
        lines.append(f"| {prec} | {r['flops']:.4g} | {r['tflops']:.4g} | {g('fma_ratio', '{:.3f}')} | "
                     f"{g('peak_tflops')} | {g('fma_adjusted_peak_tflops')} | "
                     f"{g('frac_of_peak', '{:.3f}')} | {g('frac_of_fma_adjusted_peak', '{:.3f}')} |")
    if "dram_gbs" in s:
        lines += ["", f"DRAM {s['dram_gbs']:.1f} GB/s"
                  + (f" ({s['dram_frac_of_peak']:.3f} of peak)" if "dram_frac_of_peak" in s else "")]
    return "\n".join(lines) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("report", help="an .ncu-rep file, or '-' for a raw-page CSV on stdin")
    ap.add_argument("--launch", type=int, default=0)
    ap.add_argument("--fp64-peak-tflops", type=float)
    ap.add_argument("--fp32-peak-tflops", type=float)
    ap.add_argument("--hbm-gbs", type=float)
    ap.add_argument("--units", type=float, help="work units of the launch (per-unit counts)")
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args(argv)
    m = (load_raw_csv(sys.stdin.read(), a.launch) if a.report == "-"
         else report_metrics(a.report, a.launch))
    peaks = {k: v for k, v in (("fp64_tflops", a.fp64_peak_tflops),
                               ("fp32_tflops", a.fp32_peak_tflops), ("hbm_gbs", a.hbm_gbs)) if v}
    s = summarize(m, peaks, a.units)
    print(json.dumps(s, indent=1) if a.json else to_markdown(s))
    return 0


if __name__ == "__main__":
    sys.exit(main())
