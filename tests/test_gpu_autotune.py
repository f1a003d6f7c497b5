"""The delay-rank tuner times every candidate on the caller's inputs and returns the fastest;
the system it leaves behind is unchanged (each candidate runs on its own system)."""
import numpy as np
import pytest

from synthetic import build_inputs, small_spec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402


def test_tune_delay_returns_the_fastest_candidate():
    inputs = build_inputs(small_spec(40, 40, grid=16), n_walkers=8)
    best, times = q.tune_delay(inputs, candidates=(4, 8, 16), precision="fp32",
                               reinv_period=32, warm_sweeps=1, timed_sweeps=1)
    assert set(times) == {4, 8, 16}
    assert all(np.isfinite(v) and v > 0 for v in times.values())
    assert best == min(times, key=times.get)
    # the chosen rank runs a normal sweep
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=best, reinv_period=32)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(1)
    e, _ = w.measure()
    assert np.all(np.isfinite(e))
    w.close()
    s.close()


def test_tune_launch_covers_delays_and_batches():
    inputs = build_inputs(small_spec(32, 32, grid=12), n_walkers=6)
    best, times = q.tune_launch(inputs, delays=(8, 16), precision="fp32", reinv_period=32,
                                warm_sweeps=2, timed_sweeps=1)
    # batches 2k, 4k and the whole block (0)
    assert set(times) == {(8, 16), (8, 32), (8, 0), (16, 32), (16, 64), (16, 0)}
    assert all(np.isfinite(v) and v > 0 for v in times.values())
    assert best == min(times, key=times.get)
