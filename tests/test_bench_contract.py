"""The benchmark's JSON line (CPU): the reference arm, which times the FP64
oracle, runs on any machine; its line must carry the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "nozzle_re500_24x24x160", "--steps", "2", "--warmup", "1", "--ref-seconds", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["config"]["workload"] == "nozzle_re500_24x24x160"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_roofline_bookkeeping():
    """The per-cell bytes and recorded DRAM traffic that the benchmark's
    roofline figures rest on."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2204_10566_gb300 import inputs as I

    # 27 populations read and written in the storage type, plus the link word
    assert [bench.algorithmic_bytes_per_cell(p) for p in ("fp64", "fp32", "fp16s")] == [436, 220, 112]
    # the committed ncu traffic: one line per precision of the default workload,
    # read + write = total, a little above the algorithmic bytes of a launch
    path = os.path.join(ROOT, "profiles", "step_kernel_dram_traffic.txt")
    rows = [dict(kv.split("=", 1) for kv in line.split()) for line in open(path)
            if line.strip() and not line.startswith("#")]
    cells = I.active_count(I.workload_flags(bench.DEFAULT_WORKLOAD))
    for p in ("fp32", "fp16s"):
        (r,) = [r for r in rows if r["workload"] == bench.DEFAULT_WORKLOAD and r["precision"] == p]
        total, rd, wr, alg = (float(r[k]) for k in ("dram_bytes_per_launch", "read", "write", "algorithmic"))
        assert abs(rd + wr - total) <= 2.0
        assert abs(alg - cells * bench.algorithmic_bytes_per_cell(p)) < 0.01 * alg
        assert 1.0 < total / alg < 1.3
