"""bench.py's per-kernel report on the CPU: shares, the dominant kernel's roofline, the whole
apply against the FP32 peak, and the tensor-core switch against the TF32 peak, from a profile
shaped like the headline run (N=1024, q=9, 32 RHS, s=3, e=2)."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

INFO = types.SimpleNamespace(N=1024, q=9, s=3, l0=3, precision=1, pairs_per_level=4 * 1024 * 1024)
# {kind: (launches, total ms)} over two applies
PROF = {"init": (2, 89.1), "trans_p": (4, 306.7), "switch": (2, 316.8), "trans_x": (4, 352.8), "term": (2, 70.3)}
MS_STEP = 567.9


@pytest.mark.parametrize("switch_impl", [0, 3])
def test_kernel_report(switch_impl):
    kernels, roof = bench.kernel_report(PROF, INFO, 2, MS_STEP, switch_impl)
    assert sum(v["share"] for v in kernels.values()) == pytest.approx(1.0)
    assert roof["kernel"] == "trans_x"  # 352.8 ms of 1135.7: the largest share
    fl, _ = bench.kernel_flops_bytes("trans_x", INFO, bench.NRHS)
    assert roof["achieved"] == pytest.approx(fl / 88.2e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] * 1e12 / bench.FP32_PEAK)
    assert roof["traffic"] == bench.MEASURED_TRAFFIC["trans_x"]
    per_step = sum(bench.kernel_flops_bytes(k, INFO, bench.NRHS)[0] * n for k, (n, _) in PROF.items()) / 2
    assert roof["apply_achieved"] == pytest.approx(per_step / (MS_STEP * 1e-3) / 1e12)
    assert 0.0 < roof["apply_frac"] < 1.0
    sw = kernels["switch"]
    if switch_impl == 3:
        # 5 MMAs of 128 x 64 x 168 per pair, 4 Mi pairs, one 32-RHS tile
        tc = 5 * 2 * 128 * 64 * 168 * INFO.pairs_per_level
        assert sw["tensor_tflops"] == pytest.approx(tc / 158.4e-3 / 1e12)
        assert 0.0 < sw["tensor_frac_of_tf32_peak"] < 1.0
    else:
        assert "tensor_tflops" not in sw


def test_tf32_peak_is_derived_from_the_bf16_figure():
    assert 500.0 < bench.TF32_PEAK_FROM_BF16 < 1200.0


def test_wave_timing_reports_instead_of_raising():
    # without a usable device the wave leg returns an error record; the headline line survives
    args = types.SimpleNamespace(steps=1, warmup=0)
    rec = bench.run_wave(args, "cpu", lambda x: x, 1)
    assert set(rec) == {"error"} or rec.get("unit") == "outputs/s"
