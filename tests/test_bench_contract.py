"""The benchmark's reference arm on a CPU-only machine."""
import os


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the timed oracle on a bounded slice) prints one JSON line
    with the keys of the benchmark contract, on a CPU-only machine."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-rows", "8"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] >= 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("nao1200")
    # the step is a bounded sample of one evaluation: the line says so and its step time is
    # the measured one
    assert "value_projection" in d and d["ms_per_step"] < 60e3


def test_roofline_of_both_split_layouts():
    """The half transform's roofline entry for both digit layouts of B: digit-product flops over
    the stage time against the sustained BF16 peak, and the measured per-row DRAM traffic scaled
    to the workload's rows (the packed planes move about two thirds of the full-row bytes)."""
    import sys
    from types import SimpleNamespace
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    s = SimpleNamespace(naux=4800, nao=1200)
    work = bench.algorithmic_work(1200, 4800, 150, 40)
    r = {"stage_ms": [42.0, 12.0, 3.0, 8.0, 0.2]}
    peaks = {"bf16_tflops_sustained": 1728.1}
    out = {k: bench.roofline_for(k, r, work, peaks, s) for k in ("split", "split_packed")}
    for rf in out.values():
        assert rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s"
        assert abs(rf["achieved"] - 21 * work["s1"] / 0.042 / 1e12) < 1e-6
        assert abs(rf["frac"] - rf["achieved"] / 1728.1) < 1e-12
        assert rf["traffic"] is not None
    full, packed = out["split"]["traffic"], out["split_packed"]["traffic"]
    # full rows: six BF16 planes of a 1200-long row (14.4 KB) plus 192 FP64 outputs, read and
    # written once; packed: 45 tiles and 48 ragged rows per b^L, 0.55 of the digits
    assert 0.95 * 5.76e6 * 15.9e3 < full < 1.1 * 5.76e6 * 15.9e3
    assert 0.6 * full < packed < 0.7 * full
