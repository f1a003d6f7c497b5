"""The batched delayed update over many launches without re-inversion.

Every Metropolis launch of the batched mode forms its moves from the per-launch pair matrix
and hands its window (new value rows, inverse rows, C^-1) to the batched flush kernel; the
accepted moves' VGL rows reach the current set by bulk copies. Without re-inversion nothing
repairs an error in that hand-off, so after several sweeps the device inverse must still be
the inverse of the Slater matrix of the device's orbital rows, those rows must be the
orbitals at the final positions, and E_L there must match the oracle's."""
import numpy as np
import pytest

from synthetic import build_inputs, small_spec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.vmc import OracleSystem   # noqa: E402


@pytest.mark.parametrize("precision,delay_k,n_up,n_dn", [
    ("fp64", 16, 37, 35),     # ragged spin blocks, rows not 16-byte aligned
    ("fp32", 32, 40, 40),
    ("fp32", 8, 37, 35),
])
def test_batched_window_keeps_the_inverse(precision, delay_k, n_up, n_dn):
    spec = small_spec(n_up, n_dn, grid=16, n_walkers=6)
    inputs = build_inputs(spec, n_walkers=6)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=delay_k, reinv_period=0)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(5)
    e_gpu, _ = w.measure()
    final = w.positions()
    osys = OracleSystem(inputs, coef=inputs["coef"])
    # A hand-off error shows as O(1); the bounds are the storage precision's
    tol_inv = 1e-9 if precision == "fp64" else 1e-2
    tol_orb = 1e-12 if precision == "fp64" else 1e-5
    tol_e = 1e-10 if precision == "fp64" else 1e-4
    ne = n_up + n_dn
    for wid in range(6):
        orb = w.orbitals(wid)
        fw = osys.walker(final[wid], wid)
        for spin, (first, ns) in enumerate(((0, n_up), (n_up, n_dn))):
            A = orb[first:first + ns, 0, :ns]
            # the current orbital rows are the orbitals at the final positions
            assert np.abs(A - fw.A[spin]).max() / np.abs(fw.A[spin]).max() < tol_orb, (wid, spin)
            res = np.abs(A @ w.inverse(wid, spin).T - np.eye(ns)).max()
            assert res < tol_inv, (wid, spin, res)
        e_ref = osys.measure(fw)[0]
        assert abs(e_gpu[wid] - e_ref) / ne < tol_e, (wid, e_gpu[wid], e_ref)
    w.close()
    s.close()
