"""GPU parity of the Coulomb energy by Ewald summation (Sec. "Hamiltonian": periodic
Coulomb sums by the Ewald technique; Sec. "Long-Range Interactions") against the FP64
oracle at the GPU's own walker positions.

E_L with the Ewald potential is compared with the oracle's kinetic energy plus its direct
restatement of the Ewald sums. FP64: 1e-10 relative. Single precision, per walker:
max(1e-5 Ha per electron, 2^-24 cond K) with K the magnitude of the kinetic energy's
determinant terms (``parity_util.el_gate``); the Ewald terms themselves add far less (a few
ulp per real-space pair, about 2^-24 per structure-factor phase, summed in double per 32
electrons).
"""
import math

import numpy as np
import pytest

from synthetic import build_inputs, small_spec, spec_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.ewald import coulomb_potential, kvectors   # noqa: E402
from oracle.vmc import OracleSystem   # noqa: E402
from parity_util import el_gate   # noqa: E402


def _params(L, x=4.5):
    """alpha with erfc(alpha L / 2) = erfc(x) and kcut with exp(-kcut^2 / (4 alpha^2)) = e^{-x^2}."""
    alpha = 2.0 * x / L
    return alpha, 2.0 * alpha * x


def _oracle_el(osys, R, alpha, kcut):
    wf = osys.wf
    kin = wf.local_energy(R)[1]
    return kin + coulomb_potential(R, wf.ions, wf.Z, wf.L, alpha, kcut)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_ewald_energy_small_charged_cell(precision):
    """15 electrons and 3 ions of charge 4: a charged cell, so the background term is live."""
    inputs = build_inputs(small_spec(8, 7, grid=12), n_walkers=6)
    coef = None
    if precision == "bf16":
        from parity_util import bf16_round
        coef = bf16_round(inputs["coef"])
        inputs = dict(inputs, coef=coef)
    spec = inputs["spec"]
    alpha, kcut = _params(spec.L)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=4)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(2)
    e_yukawa, _ = w.measure()
    s.set_ewald(alpha, kcut)
    assert s.ewald_count == kvectors(spec.L, kcut).shape[0]
    e_gpu, _ = w.measure()                       # the same state, measured again
    pos = w.positions()
    osys = OracleSystem(inputs, coef=coef)
    ne = spec.n_elec
    errs, gates = [], []
    for k in range(pos.shape[0]):
        ref = _oracle_el(osys, pos[k], alpha, kcut)
        errs.append(abs(e_gpu[k] - ref))
        gates.append(1e-10 * max(1.0, abs(ref)) if precision == "fp64" else el_gate(osys.wf, pos[k]))
    print(f"ewald {precision}: max |E_L error| {max(errs):.2e} Ha ({max(errs) / ne:.2e} per "
          f"electron); error / gate {np.round(np.array(errs) / np.array(gates), 3)}")
    assert np.all(np.array(errs) <= np.array(gates))
    # alpha = 0 goes back to the Yukawa form, bit for bit
    s.set_ewald(0.0)
    assert s.ewald_count == -1
    e_back, _ = w.measure()
    assert np.array_equal(e_back, e_yukawa)
    w.close()
    s.close()


def test_ewald_rejects_bad_arguments():
    inputs = build_inputs(small_spec(3, 2, grid=8), n_walkers=2)
    s = q.system_from_inputs(inputs)
    for a, kc in ((-1.0, 1.0), (float("nan"), 1.0), (1.0, 0.0), (1.0, float("inf")),
                  (1.0, 2 * math.pi / inputs["spec"].L * 65)):
        with pytest.raises(q.QMCError):
            s.set_ewald(a, kc)
    assert s.ewald_count == -1
    s.close()


def test_ewald_full_size_sampled_and_split_independent():
    """The 512-electron workload in the bench's launch configuration (FP32, k = 32):
    sampled walkers against the oracle, and E_L unchanged by the split parameter once both
    truncations have converged (a property of the Ewald sum, independent of the oracle)."""
    spec = spec_for("sj512")
    inputs = build_inputs(spec)
    alpha, kcut = _params(spec.L)
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=32, reinv_period=128,
                             logdet_period=1024)
    s.set_ewald(alpha, kcut)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(2)
    e1, _ = w.measure()
    pos = w.positions()
    osys = OracleSystem(inputs)
    for k in (0, 200):
        ref = _oracle_el(osys, pos[k], alpha, kcut)
        gate = el_gate(osys.wf, pos[k])
        print(f"walker {k}: E_L {e1[k]:.6f} oracle {ref:.6f} error {e1[k] - ref:.2e} gate {gate:.2e}")
        assert abs(e1[k] - ref) <= gate
    a2, k2 = _params(spec.L, 5.2)
    s.set_ewald(a2, k2)
    e2, _ = w.measure()
    d = np.abs(e2 - e1)
    print(f"alpha {alpha:.4f} -> {a2:.4f}: max |dE_L| {d.max():.2e} Ha over {e1.size} walkers")
    assert d.max() / spec.n_elec < 1e-5
    w.close()
    s.close()
