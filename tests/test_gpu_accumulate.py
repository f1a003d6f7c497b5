"""GPU: the FP64 walker reductions of qmc_accumulate_energy (Sec. "Variational Monte
Carlo", Eq. pmc:weighted_average: sums of W, W E_L and W E_L^2 over walkers, W = 1 in VMC)
and the acceptance ratio, against the FP64 oracle's local energies at the GPU's walker
positions and the per-move accept bits of the trace; the counters reset after each call."""
import numpy as np
import pytest

from synthetic import build_inputs, small_spec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.vmc import OracleSystem   # noqa: E402


@pytest.mark.parametrize("precision,delay_k", [("fp64", 1), ("fp32", 8)])
def test_accumulate_energy_against_oracle(precision, delay_k):
    n_w = 37                              # not a multiple of the reduction's 32-lane warps
    inputs = build_inputs(small_spec(9, 8, grid=12), n_walkers=n_w)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=delay_k)
    w = q.Walkers(s, inputs["pos"])
    ne = s.n_up + s.n_dn
    buf = torch.zeros((2, n_w, ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    w.sweep(2)
    out = w.accumulate()
    tr = buf.cpu().numpy()
    pos = w.positions()
    osys = OracleSystem(inputs)
    e_ref = np.array([osys.wf.local_energy(pos[k])[0] for k in range(n_w)])
    # E_L tolerance per walker: 1e-10 relative (FP64), 1e-5 Ha per electron (single precision)
    tol = (1e-10 * np.abs(e_ref)) if precision == "fp64" else np.full(n_w, 1e-5 * ne)
    assert abs(out[0] - n_w) == 0.0
    assert abs(out[1] - e_ref.sum()) <= tol.sum()
    e2_tol = (2 * np.abs(e_ref) * tol + tol * tol).sum()
    assert abs(out[2] - (e_ref ** 2).sum()) <= e2_tol
    acc_ratio = tr[..., 7].mean()
    assert out[3] == pytest.approx(acc_ratio, rel=0, abs=1e-15)
    assert 0.05 < acc_ratio < 0.99
    # the device sums equal the read-back energies summed in FP64 (same walkers, W = 1)
    e_gpu, _ = w.measure()
    assert out[1] == pytest.approx(e_gpu.sum(), rel=1e-13)
    assert out[2] == pytest.approx((e_gpu ** 2).sum(), rel=1e-13)
    # a second call without new moves: same energy sums, no accepted or proposed moves
    out2 = w.accumulate()
    assert np.array_equal(out2[:3], out[:3]) and out2[3] == 0.0
    # one more sweep: the ratio counts that sweep only
    w.trace_enable(buf)
    w.sweep(1)
    out3 = w.accumulate()
    assert out3[3] == pytest.approx(buf[0].cpu().numpy()[..., 7].mean(), rel=0, abs=1e-15)
    w.close()
    s.close()


def test_accumulate_energy_into_device_memory():
    inputs = build_inputs(small_spec(5, 4, grid=8), n_walkers=300)
    s = q.system_from_inputs(inputs)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(1)
    dev = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    w.accumulate(dev)
    torch.cuda.synchronize()
    e, _ = w.measure()
    got = dev.cpu().numpy()
    assert got[0] == 300.0
    assert got[1] == pytest.approx(e.sum(), rel=1e-13)
    assert got[2] == pytest.approx((e * e).sum(), rel=1e-13)
    assert 0.0 < got[3] < 1.0
    w.close()
    s.close()
