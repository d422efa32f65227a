"""Host logic of bench.py's roofline record (no GPU): the dominant kernel class, achieved work over
time against the measured peak, and the ncu traffic figure that is reported only while the source it
was captured from is unchanged."""
import hashlib
import os

import pytest

import bench


def _kernels(ms_matvec=6000.0, ms_update=900.0):
    return {"matvec": {"ms": ms_matvec, "launches": 27200, "work": 27200 * 663552},
            "gs_update": {"ms": ms_update, "launches": 1275, "work": 1.8e11},
            "ritz": {"ms": 10.0, "launches": 34, "work": 0}}


def test_fp32_op_count_of_the_fused_product():
    bound, per_site, unit = bench.LEARNED_UNIT_WORK["matvec"]
    assert (bound, unit) == ("alu", "FP32 op")
    assert per_site == 1152 * 5 + 12 * 42 + 12 * 8 * 5 + 12 * 2 * 3 + 3 * (3 + 8) + 450 == 7299


def test_roofline_picks_the_dominant_class_and_divides_by_the_measured_peak():
    peaks = {"fp32_fma_tflops": 78.4}
    r = bench.learned_roofline(_kernels(), "stencil_24x24x24x48", peaks)
    assert r["kernel"] == "matvec" and r["bound"] == "alu" and r["unit"] == "Tops/s"
    achieved = 27200 * 663552 * 7299 / 6.0 / 1e12
    assert r["achieved"] == pytest.approx(achieved, abs=0.01)
    assert r["peak"] == pytest.approx(39.2, abs=0.01)              # one op per FMA
    assert r["frac"] == pytest.approx(achieved / 39.2, abs=1e-3)
    assert r["avg_launch_us"] == pytest.approx(6000.0 * 1e3 / 27200, abs=0.01)
    r2 = bench.learned_roofline(_kernels(ms_matvec=500.0), "stencil_24x24x24x48", peaks)
    assert r2["kernel"] == "gs_update" and r2["bound"] == "hbm" and r2["unit"] == "GB/s"


def test_traffic_is_reported_only_for_the_captured_source_and_workload(monkeypatch):
    t = bench.NCU_TRAFFIC["matvec"]
    with open(os.path.join(bench.ROOT, t["source"]), "rb") as f:
        current = hashlib.sha256(f.read()).hexdigest()
    assert t["sha256"] == current                 # the recorded capture is of the kernel as committed
    assert bench.ncu_traffic("matvec", "stencil_24x24x24x48") == t["bytes"]
    assert bench.ncu_traffic("matvec", "stencil_16x16x16x16") is None
    assert bench.ncu_traffic("no_such_class", "stencil_24x24x24x48") is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "matvec", dict(t, sha256="0" * 64))
    assert bench.ncu_traffic("matvec", "stencil_24x24x24x48") is None
