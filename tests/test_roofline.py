"""The hierarchical-roofline tool on a hand-made ncu raw-page export (no GPU needed)."""

import io
import json
import sys

import pytest

from paper_2008_11326_gb300 import roofline

CSV = (
    '"ID","Kernel Name","gpu__time_duration.sum","l1tex__t_bytes.sum","lts__t_bytes.sum",'
    '"dram__bytes_read.sum","dram__bytes_write.sum",'
    '"smsp__sass_thread_inst_executed_op_dadd_pred_on.sum",'
    '"smsp__sass_thread_inst_executed_op_dmul_pred_on.sum",'
    '"smsp__sass_thread_inst_executed_op_dfma_pred_on.sum",'
    '"smsp__sass_thread_inst_executed_op_ffma_pred_on.sum",'
    '"smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum","sm__cycles_elapsed.avg.per_second"\n'
    '"","","msecond","Gbyte","Mbyte","Mbyte","Kbyte","inst","inst","inst","inst","inst","Ghz"\n'
    '"0","k","2.5","1.5","300","200","500","1,000,000","2,000,000","7,000,000","100","50","2.07"\n')


def test_counts_bytes_and_intensity():
    m = roofline.load_raw_csv(CSV)
    assert m["gpu__time_duration.sum"] == pytest.approx(2.5e-3)
    assert m["l1tex__t_bytes.sum"] == pytest.approx(1.5e9)
    s = roofline.summarize(m, {"fp64_tflops": 1.2, "hbm_gbs": 6785.5}, units=1e6)
    fp64 = s["fp64"]
    assert fp64["flops"] == pytest.approx(1e6 + 2e6 + 2 * 7e6)            # 17e6
    assert fp64["tflops"] == pytest.approx(17e6 / 2.5e-3 / 1e12)
    assert fp64["fma_ratio"] == pytest.approx(0.7)
    assert fp64["fma_adjusted_peak_tflops"] == pytest.approx(0.85 * 1.2)
    assert fp64["ai"]["l2"] == pytest.approx(17e6 / 300e6)
    assert s["bytes"]["dram"] == pytest.approx(200e6 + 500e3)
    assert fp64["instructions_per_unit"]["dfma"] == pytest.approx(7.0)
    assert s["fp32"]["flops"] == pytest.approx(2 * 100 + 4 * 50)
    assert s["dram_gbs"] == pytest.approx(200.5e6 / 2.5e-3 / 1e9)
    assert "| l2 |" in roofline.to_markdown(s)


def test_command_keeps_the_clocks_and_limits_the_capture():
    cmd = roofline.ncu_command(["python", "bench.py"], "gpp_batched_kernel", "out", 1, 2)
    assert cmd[cmd.index("--clock-control") + 1] == "none"
    assert cmd[cmd.index("-c") + 1] == "2" and cmd[-2:] == ["python", "bench.py"]
    metrics = cmd[cmd.index("--metrics") + 1].split(",")
    assert "lts__t_bytes.sum" in metrics and "dram__bytes_write.sum" in metrics


def test_cli_reads_csv_on_stdin(monkeypatch, capsys):
    monkeypatch.setattr(sys, "stdin", io.StringIO(CSV))
    assert roofline.main(["-", "--fp64-peak-tflops", "1.2", "--json"]) == 0
    s = json.loads(capsys.readouterr().out)
    assert s["fp64"]["frac_of_peak"] == pytest.approx(17e6 / 2.5e-3 / 1e12 / 1.2)


def test_collect_runs_the_capture_then_reads_the_report():
    calls = []

    class Done:
        stdout = CSV

    def fake_run(args, **kw):
        calls.append(list(args))
        return Done()

    s = roofline.collect(["python", "bench.py", "--profile-case", "fwd_f64"], "gpp_batched",
                         "prof", {"fp64_tflops": 1.2}, units=1e6, run=fake_run)
    assert calls[0][0] == "ncu" and calls[0][-4:] == ["python", "bench.py", "--profile-case",
                                                      "fwd_f64"]
    assert calls[0][calls[0].index("--clock-control") + 1] == "none"
    assert calls[1] == ["ncu", "-i", "prof.ncu-rep", "--page", "raw", "--csv"]
    assert s["fp64"]["flops_per_unit"] == pytest.approx(17.0)
