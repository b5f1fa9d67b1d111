"""Host-side arithmetic of bench.py (no GPU): the grouped launch's roofline
times on a hand-worked group."""
import pytest


def test_grouped_rooflines_hand_worked():
    import bench

    # (1000, 1000, 1000): 2e9 flops, 6e6 bytes; (1, 1000, 1000): 2e6 flops,
    # 2.004e6 bytes. At 1 TFLOP/s and 10 GB/s the first is tensor-bound
    # (2 ms against 0.6 ms), the second HBM-bound (0.2004 ms against 0.002 ms).
    shapes = [(1000, 1000, 1000), (1, 1000, 1000)]
    peaks = {"bf16_tflops": 1.0, "hbm_gbs": 10.0, "bf16_tflops_sustained": 0.5}
    overlap, overlap_sust, per_problem = bench.grouped_rooflines_ms(shapes, peaks)
    assert overlap == pytest.approx(2.002)        # max(2.002 ms of flops, 0.8004 ms of bytes)
    assert overlap_sust == pytest.approx(4.004)   # the flops at 0.5 TFLOP/s
    assert per_problem == pytest.approx(2.2004)   # 2 ms + 0.2004 ms: no overlap
    # without a sustained figure the burst peak stands in for it
    peaks.pop("bf16_tflops_sustained")
    assert bench.grouped_rooflines_ms(shapes, peaks)[1] == pytest.approx(2.002)


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` runs the oracle's maps step on the host
    cores and prints one JSON line in the benchmark's form: impl, metric and
    unit as the GPU line, a positive value, the cores it used, and an e2e
    figure with no host-device copies."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "30", "--warmup", "0"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "TB/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 30
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == bench.WORKLOAD
