"""bench.py's per-kernel report on the CPU: shares, the dominant kernel's roofline, each kernel
against the peak of its own pipe (the tensor-core switch against the TF32 peak), and the whole
apply against the roofline time max(B_min/BW, F32/P_fp32, F64/P_fp64, 2E/P_mufu, F_tc/P_tf32),
from a profile shaped like the headline run (N=1024, q=9, 32 RHS, s=3, e=2)."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

INFO = types.SimpleNamespace(N=1024, q=9, s=3, l0=3, lm=5, l1=7, e=2, precision=1, pairs_per_level=4 * 1024 * 1024)
# {kind: (launches, total ms)} over two applies
PROF = {"init": (2, 89.1), "trans_p": (4, 306.7), "switch": (2, 316.8), "trans_x": (4, 352.8), "term": (2, 70.3)}
MS_STEP = 567.9


@pytest.mark.parametrize("switch_impl", [0, 3, 5, 6])
def test_kernel_report(switch_impl):
    kernels, roof = bench.kernel_report(PROF, INFO, 2, switch_impl)
    assert sum(v["share"] for v in kernels.values()) == pytest.approx(1.0, abs=2e-3)
    assert roof["kernel"] == "trans_x"  # 352.8 ms of 1135.7: the largest share
    fl, by = bench.kernel_flops_bytes("trans_x", INFO, bench.NRHS)
    # 24 q^3 + 30 q^2 flops per pair and RHS, 4 Mi pairs, 32 RHS; the state read and written once
    assert fl == (24 * 729 + 30 * 81) * INFO.pairs_per_level * 32
    assert by == 2 * INFO.pairs_per_level * 32 * 81 * 8
    # compute-bound: 2.67e12 flops at the FP32 peak (33 ms) exceed 174 GB at the HBM peak (26 ms)
    assert roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(fl / 88.2e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] * 1e12 / bench.FP32_PEAK)
    assert roof["traffic"] == bench.MEASURED_TRAFFIC["trans_x"]
    # the switch: 8 q^4 flops per pair and RHS are 7.0e12, ~6 ms at a TF32 peak (then its 174 GB of
    # state, 26 ms at the HBM peak, bound it) but 87 ms on the FP32 FMA pipe
    sw = kernels["switch"]
    swfl = 8 * 9 ** 4 * INFO.pairs_per_level * 32
    tensor = switch_impl in (3, 5, 6)  # the tcgen05 forms (5 or 3 split-TF32 products, narrow or wide)
    if tensor:
        assert sw["bound"] == "hbm"
        assert sw["frac"] == pytest.approx(by / (bench._hbm_peak_gbs() * 1e9) / 158.4e-3, abs=1e-3)
    else:
        assert sw["bound"] == "alu"
        assert sw["frac"] == pytest.approx(swfl / bench.FP32_PEAK / 158.4e-3, abs=1e-3)
    assert sw["pipe"] == ("tf32 tensor" if tensor else "fp32 fma")
    # init and term move 87 GB (13 ms) against 0.7-0.8e12 flops (9-10 ms): HBM-bound too
    assert kernels["init"]["bound"] == "hbm" and kernels["term"]["bound"] == "hbm"


def test_apply_roofline_by_hand():
    # the five terms recomputed from the per-unit counts of the design notes
    probes = {"fp32": 78.0e12, "fp64": 1.06e12, "sfu": 4.9e12}
    r = bench.apply_roofline(INFO, 32, 567.9, probes)
    P, q, R = INFO.pairs_per_level, 9, 32
    F32 = (64 * 1024 ** 2 * R * (4 * q * q + 8) + 4 * (24 * q ** 3 + 30 * q * q) * P * R
           + (4 * 8 * q * q + 4 * 64 * q + 6 * (64 + q * q)) * P * R)
    assert r["F32"] == F32
    assert r["F_tc"] == 8 * q ** 4 * P * R
    assert r["E"] == q ** 4 * P + 4 * 5 * q * q * P + 64 * 1024 ** 2 + q * q * P + (q * q + 64) * P
    assert r["B_min"] == 2 * 1024 ** 2 * R * 8 + 2 * P * R * q * q * 8
    assert r["terms_ms"]["fp32_ms"] == pytest.approx(F32 / bench.FP32_PEAK * 1e3, abs=0.01)
    assert r["t_roof_ms"] == max(r["terms_ms"].values())
    assert r["apply_frac"] == pytest.approx(r["t_roof_ms"] / 567.9, abs=1e-4)
    # at the headline the FP32 term decides: ~151 ms, ~0.27 of the 568 ms apply
    assert r["t_roof_ms"] == r["terms_ms"]["fp32_ms"]
    assert 0.25 < r["apply_frac"] < 0.29


def test_tf32_peak_is_derived_from_the_bf16_figure():
    assert 500.0 < bench.TF32_PEAK_FROM_BF16 < 1200.0


def test_wave_timing_reports_instead_of_raising():
    # without a usable device the wave leg returns an error record; the headline line survives
    args = types.SimpleNamespace(steps=1, warmup=0)
    rec = bench.run_wave(args, "cpu", lambda x: x, 1)
    assert set(rec) == {"error"} or rec.get("unit") == "outputs/s"
