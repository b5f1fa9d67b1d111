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
