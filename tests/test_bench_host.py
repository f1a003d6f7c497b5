"""Host logic of bench.py's roofline: the per-launch algorithmic rate and the stored DRAM
traffic, which is used only at the workload and delay rank it was captured at (CPU)."""
import pytest

import bench
from synthetic import spec_for

PEAKS = {"hbm_gbs": 6789.3, "bf16_tflops": 1899.6}


def _cls(name, preset="sj512", precision="fp32", k=32, ms=96.25, n=800, steps=50):
    spec = spec_for(preset)
    return bench.class_roofline(name, ms, n, spec, precision, spec.n_walkers * spec.n_elec,
                                steps, PEAKS, k, 128, 2070.0)


def test_sweep_rate_and_traffic_at_the_captured_rank():
    spec = spec_for("sj512")
    r = _cls("sweep")                              # 800 launches, 96.25 ms over 50 steps
    moves_per_launch = spec.n_walkers * spec.n_elec * 50 / 800
    per_move = 5 * spec.n_orb * 4 + 3 * spec.n_up * 4
    launch_s = 96.25e-3 / 800
    assert r["kernel"] == "k_sweep_win"
    assert r["achieved"] == pytest.approx(per_move * moves_per_launch / launch_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
    assert r["traffic"] == pytest.approx((46.3e6 + 7.1e6) / 8192 * moves_per_launch)
    # captured at k = 32 only
    assert _cls("sweep", k=16)["traffic"] is None


def test_flush_traffic_follows_the_delay_rank():
    t16 = _cls("flush", k=16)["traffic"]
    t32 = _cls("flush", k=32)["traffic"]
    assert t16 is None                     # captured at k = 32 only
    assert t32 == pytest.approx((80.9e6 + 6.6e6) / 256 * 256)
    assert _cls("flush", k=8)["traffic"] is None


def test_traffic_only_for_the_captured_workload_and_kernel_names():
    assert _cls("vgl", preset="sj128")["traffic"] is None
    assert _cls("vgl", precision="bf16")["traffic"] is None
    assert _cls("vgl")["traffic"] is not None            # k-independent entry
    fp64 = _cls("sweep", precision="fp64", k=1)
    assert fp64["kernel"] == "k_sweep"                   # rank 1: the original sweep
    assert _cls("flush", precision="fp64", k=16)["kernel"] == "k_flush"


def test_dominant_class_leads_the_roofline():
    import paper_1802_06922_gb300.qmcgb as qb
    spec = spec_for("sj512")
    ms = {"sweep": 87.0, "flush": 96.0, "vgl": 63.0}
    n = {"sweep": 800, "flush": 800, "vgl": 100}
    prof_ms = [ms.get(c, 0.0) for c in qb.KERNEL_CLASSES]
    prof_n = [n.get(c, 0) for c in qb.KERNEL_CLASSES]
    top, per = bench.roofline(prof_ms, prof_n, spec, "fp32", spec.n_walkers * spec.n_elec, 50,
                              PEAKS, 32, 128, 2070.0)
    assert top["cls"] == "flush" and top["kernel"] == "k_flush_tc"
    assert sum(v["share"] for v in per.values()) == pytest.approx(1.0)
