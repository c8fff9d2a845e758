"""The bench's roofline arithmetic on the host (no GPU): achieved = algorithmic work per launch over
the live average launch time, frac = achieved / peak, the bound chosen by the larger of the HBM
and tensor times, traffic scaled from the per-column capture only for the captured M, and the
measured peaks read from MEASURED_PEAKS.json (the sustained BF16 figure for kernels timed inside
a long step)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeH:
    def __init__(self, flops):
        self.f = flops

    def flops_per_column(self):
        return self.f


def test_defect_roofline_split():
    H = FakeH(311_000.0)
    ncols, M, per_point = 523_776 * 2, 512, 7.85e6
    cnt = {"defect_launches": 5, "defect_ms": 5 * 25.0}
    r = bench.roofline_defect(H, cnt, 300.0, ncols, M, per_point, 1748.4, "measured")
    t = 25.0e-3
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(per_point * ncols / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1748.4)
    assert r["fp64_equivalent_tflops"] == pytest.approx(311_000.0 * ncols / t / 1e12)
    assert r["share_of_step"] == pytest.approx(125.0 / 300.0)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_COLUMN["defect"][1] * ncols)
    # the capture holds for M = 512 only
    assert bench.roofline_defect(H, cnt, 300.0, ncols, 1024, per_point, 1748.4, "measured")["traffic"] is None


def test_defect_roofline_double_float():
    H = FakeH(2.0e5)
    cnt = {"defect_launches": 2, "defect_ms": 2 * 50.0}
    r = bench.roofline_defect(H, cnt, 400.0, 1000, 512, None, 1748.4, "measured")
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(bench.DF_PEAK_TFLOPS)
    assert r["achieved"] == pytest.approx(2.0e5 * 1000 / 0.05 / 1e12)
    assert bench.DF_PEAK_TFLOPS == pytest.approx(152 * 128 * 2.07e9 * 2 / 11 / 1e12)


def test_smoother_roofline_picks_the_longer_bound():
    cnt = {"smooth_launches": 10, "smooth_ms": 10 * 2.0}
    M, ncols = 512, 523_776
    # few flops per column: HBM-bound, achieved = 12 M bytes per column over the launch time
    r = bench.roofline_smoother(FakeH(1.0e3), cnt, 300.0, ncols, M, 6674.2, 1748.4, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(12.0 * M * ncols / 2.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6674.2)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_COLUMN["smooth"][1] * ncols)
    # many flops per column: tensor-bound
    r = bench.roofline_smoother(FakeH(1.0e9), cnt, 300.0, ncols, M, 6674.2, 1748.4, "measured")
    assert r["bound"] == "tensor" and r["frac"] == pytest.approx(1.0e9 * ncols / 2.0e-3 / 1e12 / 1748.4)


def test_peaks_read_the_measured_file():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("no measured peaks in this checkout")
    with open(path) as fh:
        d = json.load(fh)
    hbm, bf16, kind = bench.peaks()
    assert kind == "measured"
    assert hbm == pytest.approx(float(d["hbm_gbs"]))
    assert bf16 == pytest.approx(float(d.get("bf16_tflops_sustained", d["bf16_tflops"])))
