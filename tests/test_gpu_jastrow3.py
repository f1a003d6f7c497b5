"""GPU parity of the three-body electron-electron-ion Jastrow factor (Sec. "Jastrow factor":
the polynomial of Drummond et al. in r_iI, r_jI and r_ij, cut off at r_c / 2) against the
FP64 oracle with J = J1 + J2 + J3.

Every path that evaluates J carries the term, and each has a case here: the rank-1 and
the windowed Metropolis sweeps (the windowed form adds pair corrections for two moves of one
window near the same ion), the drift-diffusion sweep (gradient at r'), the local energy
(gradient and Laplacian of every electron), ln|Psi| and the pseudopotential's virtual moves.
FP64: per-move traces, E_L and ln|Psi| to 1e-10. Single precision (lockstep on the oracle's
decisions): the per-move ratio gate, the ln|Psi| gate and the per-walker E_L gate of the
other single-precision tests.
"""
import numpy as np
import pytest

from synthetic import build_inputs, jastrow3_coefficients, small_spec, spec_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.jastrow3 import JastrowSum, ThreeBodyJastrow   # noqa: E402
from oracle.nlpp import NonLocalPP, nonlocal_energy   # noqa: E402
from oracle.vmc import OracleSystem, run_vmc   # noqa: E402
from parity_util import (assert_logpsi, assert_ratio_gate, assert_trace_close, el_gate,   # noqa: E402
                         logpsi_tol, ratio_gate, rel_err)


def _inputs(move="metropolis", n_walkers=3, m=(2, 3)):
    spec = small_spec(9, 8, grid=12, n_ion=8, move=move, step=0.3 if move == "metropolis" else 0.02)
    inputs = build_inputs(spec, n_walkers=n_walkers)
    rc3 = 0.5 * spec.L
    gs, go = jastrow3_coefficients(m[0], m[1], rc3, seed=3)
    return inputs, rc3, gs, go


def _oracle(inputs, rc3, gs, go):
    osys = OracleSystem(inputs)
    spec = inputs["spec"]
    osys.wf.jas = JastrowSum(osys.wf.jas,
                             ThreeBodyJastrow(spec.L, spec.n_up, inputs["ions"], gs, go, rc3))
    return osys


def _gpu(inputs, rc3, gs, go, n_sweeps, precision="fp64", delay_k=1, reinv_period=0,
         forced=None, logdet_period=0):
    s = q.system_from_inputs(inputs, precision=precision, delay_k=delay_k,
                             reinv_period=reinv_period, logdet_period=logdet_period)
    s.set_jastrow3(gs, go, rc3)
    nw = inputs["pos"].shape[0]
    w = q.Walkers(s, inputs["pos"])
    ne = s.n_up + s.n_dn
    buf = torch.zeros((n_sweeps, nw, ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    if forced is not None:
        bits = np.ascontiguousarray(
            forced.reshape(nw, n_sweeps, ne).transpose(1, 0, 2).astype(np.uint8))
        w.replay(bits, n_sweeps)
    en = []
    for _ in range(n_sweeps):
        w.sweep(1)
        en.append(w.measure())
    tr = buf.cpu().numpy().transpose(1, 0, 2, 3).reshape(nw, n_sweeps * ne, 8)
    pos = w.positions()
    w.close()
    s.close()
    return tr, np.array(en), pos


@pytest.mark.parametrize("move,delay_k", [("metropolis", 1), ("metropolis", 8),
                                          ("drift", 1), ("drift", 8)])
def test_jastrow3_fp64_parity(move, delay_k):
    inputs, rc3, gs, go = _inputs(move)
    osys = _oracle(inputs, rc3, gs, go)
    ids = np.arange(inputs["pos"].shape[0])
    walkers, ref, ref_en = run_vmc(osys, inputs["pos"], ids, 2)
    # the term is live: J3 of the final configurations is far from zero
    j3 = [osys.wf.jas.terms[1].value(wk.R) for wk in walkers]
    assert max(abs(v) for v in j3) > 1e-3, j3
    tr, en, pos = _gpu(inputs, rc3, gs, go, 2, delay_k=delay_k)
    assert_trace_close(tr, ref, 1e-10)
    assert np.all(rel_err(en[:, 0, :].T, ref_en[..., 0], 1.0) < 1e-10)
    assert np.all(rel_err(en[:, 1, :].T, ref_en[..., 2], 1.0) < 1e-10)
    assert np.allclose(pos, np.array([wk.R for wk in walkers]), rtol=0, atol=1e-10)


@pytest.mark.parametrize("precision,delay_k", [("fp32", 1), ("fp32", 8), ("bf16", 16)])
def test_jastrow3_single_precision_lockstep(precision, delay_k):
    inputs, rc3, gs, go = _inputs(n_walkers=3)
    coef = None
    if precision == "bf16":
        from parity_util import bf16_round
        coef = bf16_round(inputs["coef"])
        inputs = dict(inputs, coef=coef)
    osys = _oracle(inputs, rc3, gs, go)
    ids = np.arange(3)
    ne = inputs["spec"].n_elec
    cond = np.zeros((3, 2 * ne))
    walkers, ref, ref_en = run_vmc(osys, inputs["pos"], ids, 2, conds=cond)
    batched = delay_k >= 4
    tr, en, pos = _gpu(inputs, rc3, gs, go, 2, precision=precision, delay_k=delay_k,
                       reinv_period=16 if batched else 0, forced=ref[..., 7],
                       logdet_period=16 if batched else 0)
    assert_ratio_gate(tr[..., 0], ref[..., 0], cond, f"J3 {precision} k={delay_k}")
    # Delta J of every move, J3 included: FP32 pair sums
    assert np.max(np.abs(tr[..., 1] - ref[..., 1])) < 1e-4
    assert_logpsi(en[:, 1, :].T, ref_en[..., 2], ne, f"J3 {precision} k={delay_k}")
    for k, wk in enumerate(walkers):
        err = abs(en[-1, 0, k] - ref_en[k, -1, 0])
        assert err <= el_gate(osys.wf, wk.R), (k, err)


def test_jastrow3_in_pseudopotential_ratios():
    inputs, rc3, gs, go = _inputs(n_walkers=4)
    amp, width, rcut = np.array([1.5, -1.0]), np.array([1.0, 0.9]), 1.9
    s = q.system_from_inputs(inputs, precision="fp64", delay_k=1)
    s.set_jastrow3(gs, go, rc3)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(1)
    s.set_nonlocal(amp, width, rcut)
    w.sweep(1)
    vnl = w.nonlocal_energy()
    pos = w.positions()
    osys = _oracle(inputs, rc3, gs, go)
    pp = NonLocalPP(amp, width, rcut)
    live = 0
    for k in range(4):
        ref = nonlocal_energy(osys.wf, pp, pos[k], seed=inputs["seed"], t=2, walker_id=k)
        assert abs(vnl[k] - ref) <= 1e-10 * max(1.0, abs(ref)), (k, vnl[k], ref)
        live += ref != 0.0
    assert live >= 2
    w.close()
    s.close()


def test_jastrow3_rejects_bad_coefficients_and_removal_restores_j12():
    inputs, rc3, gs, go = _inputs(n_walkers=2)
    s = q.system_from_inputs(inputs, precision="fp64")
    bad = gs.copy()
    bad[1, 0, 0] += 1e-3
    for args in ((bad, go, rc3), (gs, go, 0.6 * inputs["spec"].L), (gs, go, 0.0)):
        with pytest.raises(q.QMCError):
            s.set_jastrow3(*args)
    big = np.zeros((6, 6, 2))
    with pytest.raises(q.QMCError):
        s.set_jastrow3(big, big, rc3)
    w = q.Walkers(s, inputs["pos"])
    e0, l0 = w.measure()
    s.set_jastrow3(gs, go, rc3)
    e1, l1 = w.measure()
    assert not np.array_equal(l0, l1)
    s.set_jastrow3(None)
    e2, l2 = w.measure()
    assert np.array_equal(e0, e2) and np.array_equal(l0, l2)
    w.close()
    s.close()


def test_jastrow3_full_size_sampled():
    """The 512-electron workload in the bench's launch configuration (FP32, k = 32, batched
    re-inversion every 128 moves) with the three-body term (r_c = 5 bohr, orders 2 and 3):
    the first 40 moves of two walkers against the oracle (per-move ratio gate, Delta J, the
    same decisions up to the first one at u ~ A), then ln|Psi| at the GPU's final
    configuration."""
    spec = spec_for("sj512")
    inputs = build_inputs(spec)
    rc3 = 5.0
    gs, go = jastrow3_coefficients(2, 3, rc3, seed=5)
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=32, reinv_period=128,
                             logdet_period=128)
    s.set_jastrow3(gs, go, rc3)
    w = q.Walkers(s, inputs["pos"])
    ne = spec.n_elec
    buf = torch.zeros((spec.n_walkers, ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    w.sweep(1)
    _, lp_gpu = w.measure()
    tr = buf.cpu().numpy()
    final = w.positions()
    osys = _oracle(inputs, rc3, gs, go)
    dj_err = []
    for wid in (0, 200):
        ow = osys.walker(inputs["pos"][wid], wid)
        rows, conds = [], []
        osys.sweep(ow, 0, trace=rows, electrons=range(40), conds=conds)
        ref = np.array(rows)
        got = tr[wid, :40]
        for mv in range(40):
            err, bound = ratio_gate(got[mv, 0], ref[mv, 0], conds[mv])
            assert err <= bound, (wid, mv, float(err), float(bound))
            dj_err.append(abs(got[mv, 1] - ref[mv, 1]))
            assert dj_err[-1] < 1e-4, (wid, mv, got[mv, 1], ref[mv, 1])
            if got[mv, 7] != ref[mv, 7]:
                assert abs(ref[mv, 5] - ref[mv, 6]) <= 2 * bound * ref[mv, 6] + 1e-12, (wid, mv)
                break
        fw = osys.walker(final[wid], wid)
        lp_ref = osys.log_psi(fw)
        j3 = osys.wf.jas.terms[1].value(final[wid])
        print(f"sj512 J3 walker {wid}: J3 {j3:.4f}, ln|Psi| error {lp_gpu[wid] - lp_ref:.2e}")
        assert abs(j3) > 1e-3
        assert abs(lp_gpu[wid] - lp_ref) <= logpsi_tol(ne), (wid, lp_gpu[wid] - lp_ref)
    print(f"sj512 J3: Delta J error max {max(dj_err):.2e} over {len(dj_err)} moves")
    w.close()
    s.close()
