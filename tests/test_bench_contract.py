"""bench.py's output contract on the host: the reference arm (the CPU oracle)
prints exactly one JSON line with the keys the driver reads.  The GPU arm
prints the same keys plus roofline, cpu_baseline, e2e and clocks; it needs a
GPU and is exercised by running bench.py there."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "cnot_m16", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "M16_c128_cnot64"


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_roofline_record_from_traced_passes():
    """The roofline record is the dominant kernel's algorithmic bytes per
    launch over its mean launch time, against the measured copy bandwidth."""
    bench = _bench()
    passes = [("qsim_jit_closed", 18.5, 103.0e9)] * 3 + [("probs_kernel", 1.0, 1.0e9)]
    roof, kernel_ms, launches = bench._roofline(passes, "no_such_workload")
    peak, src = bench.hbm_peak()
    assert roof["kernel"] == "qsim_jit_closed" and roof["launches"] == 3
    assert abs(roof["achieved"] - 103.0e9 / 18.5e-3 / 1e9) < 1e-6
    assert abs(roof["frac"] - roof["achieved"] / peak) < 1e-12 and roof["peak"] == peak
    assert abs(roof["share_of_device_time"] - 3 * 18.5 / (3 * 18.5 + 1.0)) < 1e-12
    assert roof["traffic"] is None  # no record for this workload
    assert kernel_ms == {"qsim_jit_closed": 18.5, "probs_kernel": 1.0}
    assert launches == {"qsim_jit_closed": 3, "probs_kernel": 1}


def test_traffic_records_follow_the_kernel_source():
    """profiles/traffic.json: each record names its capture and the source
    hash it was taken on; a record is returned only while that hash is the
    kernel's current one."""
    bench = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    n = 0
    for wl, kernels in rec.items():
        if wl.startswith("_"):
            continue
        for kernel, e in kernels.items():
            assert e["dram_bytes_per_launch"] > 0 and e["source"]
            got = bench.ncu_traffic(kernel, wl)
            if e["kernel_source_sha256_16"] == bench.kernel_source_hash(kernel):
                assert got == float(e["dram_bytes_per_launch"])
            else:
                assert got is None
            n += 1
    assert n > 0


def test_reference_arm_without_room_for_the_fp64_state(monkeypatch, capsys):
    """On a host that cannot hold the oracle's FP64 copy of the state the
    reference arm times single rows through every step instead."""
    bench = _bench()
    monkeypatch.setattr(bench, "_host_free_bytes", lambda: 1)
    import argparse
    args = argparse.Namespace(workload="cnot_m16", steps=1, warmup=0, ref_steps_per_step=0)
    assert bench.run_reference(args, 0, 1) == 0
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0
    assert "single-row evaluation" in d["cpu_baseline"]["sample"]


def test_profile_summaries_name_their_commands():
    """Each ncu summary under profiles/ gives the command that made it, and
    every ncu command there leaves the GPU clocks alone."""
    d = os.path.join(ROOT, "profiles")
    mds = [f for f in os.listdir(d) if f.endswith(".md")]
    assert mds
    for f in mds:
        text = open(os.path.join(d, f)).read()
        lines = text.splitlines()
        starts = [i for i, l in enumerate(lines) if l.strip().startswith("ncu ")]
        assert starts, f
        for i in starts:
            cmd = lines[i]
            while cmd.rstrip().endswith("\\") and i + 1 < len(lines):
                i += 1
                cmd += lines[i]
            assert "--clock-control none" in cmd, (f, cmd)
