"""The benchmark's JSON contract, checked on the host with the oracle arm
(`bench.py --impl reference`, no GPU): one JSON line with the contract's
keys, the warm-up floor of 3, and under torchrun with two ranks a line from
rank 0 only while every rank exits 0.  The 64^3 FP64 workload keeps each
run to seconds.  Also the roofline's inputs: the peak from the measured-peaks
record and the DRAM traffic from the committed ncu summary, used only while
its kernel source hash matches."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def _json_lines(stdout):
    return [json.loads(l) for l in stdout.splitlines() if l.startswith("{")]


def _run(args, timeout=600):
    return subprocess.run([sys.executable] + args, cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["bench.py", "--impl", "reference", "--config", "dense64-f64", "--steps", "2",
              "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2
    assert d["warmup"] == 3  # raised to the timing rule's floor
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "iter/s"
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"]["workload"] == "nncp-dense-3way-64x64x64-fp64-R8"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_on_rank_0_only():
    r = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
              "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
              "bench.py", "--impl", "reference", "--gpus", "2", "--config", "dense64-f64",
              "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_is_reported_only_for_the_profiled_kernel_source():
    """`roofline.traffic` comes from the committed ncu summary, and only while
    the kernel source hash recorded there matches."""
    b = _bench_module()
    path = os.path.join(ROOT, "profiles", "pm_tcr_traffic_512x512x512_fp32_r32.txt")
    kv = dict(l.split(":", 1) for l in open(path) if ":" in l and not l.startswith("#"))
    kv = {k.strip(): v.strip() for k, v in kv.items()}
    wl = b.CONFIGS["dense512-f32"]["workload"]
    assert kv["workload"] == wl
    got = b.profiled_traffic(wl, kv["kernel_source_sha"])
    assert got == float(kv["dram_bytes_per_launch"])
    assert b.profiled_traffic(wl, "0" * 16) is None
    assert b.profiled_traffic("another-workload", kv["kernel_source_sha"]) is None
    assert len(b.pm_source_sha(True)) == 16


def test_roofline_peak_is_the_measured_copy_bandwidth():
    b = _bench_module()
    peak, kind = b.measured_peak()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0


def test_default_step_counts():
    """Without --steps the oracle arm takes 10 bounded samples (the solve arm
    takes 60, which needs a GPU and is not run here)."""
    r = _run(["bench.py", "--impl", "reference", "--config", "dense64-f64"])
    assert r.returncode == 0, r.stderr[-2000:]
    d = _json_lines(r.stdout)[0]
    assert d["steps"] == 10 and d["warmup"] == 3
