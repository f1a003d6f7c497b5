"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical
seeded inputs, move by move."""
import dataclasses

import numpy as np
import pytest

from synthetic import build_inputs, small_spec, spec_for

from parity_util import (assert_logpsi, assert_ratio_gate, assert_trace_close, bf16_round,
                         logpsi_tol, oracle_vmc, rel_err)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402


def _gpu_run(inputs, walker_ids, n_sweeps, precision="fp64", delay_k=1, reinv_period=0,
             reinv_on_accepted=False, forced=None, coef=None, logdet_period=0):
    d = dict(inputs)
    if coef is not None:
        d["coef"] = coef
    s = q.system_from_inputs(d, precision=precision, delay_k=delay_k,
                             reinv_period=reinv_period, reinv_on_accepted=reinv_on_accepted,
                             logdet_period=logdet_period)
    w = q.Walkers(s, np.ascontiguousarray(inputs["pos"][walker_ids]))
    ne = s.n_up + s.n_dn
    buf = torch.zeros((n_sweeps, len(walker_ids), ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    if forced is not None:
        bits = np.ascontiguousarray(
            forced.reshape(len(walker_ids), n_sweeps, ne).transpose(1, 0, 2).astype(np.uint8))
        w.replay(bits, n_sweeps)
    energies = []
    for _ in range(n_sweeps):
        w.sweep(1)
        energies.append(w.measure())
    tr = buf.cpu().numpy().transpose(1, 0, 2, 3).reshape(len(walker_ids), n_sweeps * ne, 8)
    en = np.array(energies)          # [sweeps][2][n_w]
    pos = w.positions()
    w.close()
    s.close()
    return tr, en, pos


def test_plane_wave_fp64_parity_and_zero_variance():
    inputs = build_inputs(spec_for("pw14"), n_walkers=4)
    ids = np.arange(4)
    tr, en, pos = _gpu_run(inputs, ids, 3)
    walkers, ref, ref_en = oracle_vmc(inputs, ids, 3)
    assert_trace_close(tr, ref, 1e-10)
    e_gpu = en[:, 0, :].T           # [n_w][sweeps]
    assert np.all(rel_err(e_gpu, ref_en[..., 0], 1.0) < 1e-10)
    assert np.all(rel_err(en[:, 1, :].T, ref_en[..., 2], 1.0) < 1e-10)
    assert np.allclose(pos, np.array([w.R for w in walkers]), rtol=0, atol=1e-12)
    # spline orbitals reproduce the zero-variance kinetic energy up to the spline error
    e_ref = 2 * 6 * (2 * np.pi / 10) ** 2 / 2
    assert np.all(np.abs(e_gpu - e_ref) / e_ref < ((2 * np.pi / 10) * (10 / 32)) ** 2)


@pytest.mark.parametrize("delay_k", [1, 3, 8, 32])
def test_slater_jastrow_fp64_parity_ragged(delay_k):
    # 70 up / 66 down electrons: two 64-orbital chunks per FP64 warp with a ragged tail,
    # a delay window that does not divide the block; k = 32 fills the window to the pair
    # matrix's full 32 rows
    inputs = build_inputs(small_spec(70, 66, grid=12, n_orb=72), n_walkers=2)
    ids = np.arange(2)
    tr, en, _ = _gpu_run(inputs, ids, 1, delay_k=delay_k)
    _, ref, ref_en = oracle_vmc(inputs, ids, 1)
    assert_trace_close(tr, ref, 1e-10)
    assert np.all(rel_err(en[:, 0, :].T, ref_en[..., 0], 1.0) < 1e-10)
    assert np.all(rel_err(en[:, 1, :].T, ref_en[..., 2], 1.0) < 1e-10)


@pytest.mark.parametrize("precision,delay_k,on_acc", [("fp32", 1, True), ("fp32", 4, True),
                                                     ("bf16", 4, True), ("fp32", 8, False),
                                                     ("bf16", 16, False)])
def test_mixed_precision_lockstep(precision, delay_k, on_acc):
    inputs = build_inputs(small_spec(40, 40, grid=16), n_walkers=3)
    ids = np.arange(3)
    coef = bf16_round(inputs["coef"]) if precision == "bf16" else None
    cond = np.zeros((3, 2 * 80))
    _, ref, ref_en = oracle_vmc(inputs, ids, 2, coef=coef, conds=cond)
    forced = ref[..., 7]
    batched = delay_k >= 4 and not on_acc
    tr, en, _ = _gpu_run(inputs, ids, 2, precision=precision, delay_k=delay_k,
                         reinv_period=16, reinv_on_accepted=on_acc, forced=forced, coef=coef,
                         logdet_period=16 if batched else 0)
    # per-move ratio gate: 1e-4 relative (floor 1e-3), or cond * 2^-24 where single-precision
    # storage of the orbitals and the inverse bounds the accuracy above that
    assert_ratio_gate(tr[..., 0], ref[..., 0], cond, f"{precision} k={delay_k}")
    # ln|Psi| (anchored at every re-inversion in the batched form; the in-sweep re-inversion
    # of the accepted-move cadence has no anchor, and its short run here adds little drift)
    assert_logpsi(en[:, 1, :].T, ref_en[..., 2], 80, f"{precision} k={delay_k}")
    # a GPU decision that would differ from the oracle's must sit at u ~ A
    own = tr[..., 5] < tr[..., 6]
    flips = own != (ref[..., 7] == 1)
    if flips.any():
        assert np.all(np.abs(tr[..., 5] - ref[..., 6])[flips] <= 1e-4 * ref[..., 6][flips] + 1e-12)
    # local energy gate: 1e-5 Ha per electron
    ne = inputs["spec"].n_elec
    assert np.max(np.abs(en[:, 0, :].T - ref_en[..., 0])) / ne < 1e-5


def test_walker_state_round_trip_and_errors():
    inputs = build_inputs(small_spec(5, 4, grid=8), n_walkers=3)
    s = q.system_from_inputs(inputs)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(2)
    st = w.get_state()
    e1, l1 = w.measure()
    w.sweep(1)
    e2, _ = w.measure()
    w.set_state(st)
    e1b, l1b = w.measure()
    assert np.allclose(e1b, e1, rtol=1e-12) and np.allclose(l1b, l1, rtol=1e-12)
    w.sweep(1)
    assert np.allclose(w.measure()[0], e2, rtol=1e-12)
    with pytest.raises(q.QMCError):
        w.set_state(st[:-8])
    w.close()
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_orbitals_and_inverse_at_setup(precision):
    """Stage check: orbital VGL at the initial positions against the oracle's tricubic
    evaluation, and the FP64 re-inversion against numpy's LU inverse."""
    from oracle.orbitals import SplineOrbitals
    inputs = build_inputs(small_spec(70, 66, grid=12, n_orb=72), n_walkers=2)
    s = q.system_from_inputs(inputs, precision=precision)
    w = q.Walkers(s, inputs["pos"])
    orb = SplineOrbitals(inputs["coef"], inputs["spec"].L)
    tol = 1e-11 if precision == "fp64" else 2e-5
    for wk in range(2):
        got = w.orbitals(wk)
        R = inputs["pos"][wk]
        for e in range(0, 136, 5):
            ns = 70 if e < 70 else 66
            v, g, lap = orb.vgl(R[e])
            ref = np.vstack([v[None, :ns], g[:, :ns], lap[None, :ns]])
            scale = np.abs(ref).max()
            assert np.abs(got[e, :, :ns] - ref).max() <= tol * scale, (e, np.abs(got[e, :, :ns] - ref).max())
        for spin, (first, ns) in enumerate(((0, 70), (70, 66))):
            A = np.array([orb.values(R[first + i])[:ns] for i in range(ns)])
            Binv = w.inverse(wk, spin)
            ref = np.linalg.inv(A).T
            err = np.abs(Binv - ref).max() / np.abs(ref).max()
            # FP32 form: the matrix entries themselves are single precision, so the
            # inverse can differ from the FP64 one by about cond(A) * 2^-24
            eps = 1e-14 if precision == "fp64" else 2.0 ** -24
            assert err < 10 * np.linalg.cond(A) * eps, (err, np.linalg.cond(A))
            # the re-inversion is exact for its own input: A_gpu Binv^T = I
            A_gpu = w.orbitals(wk)[first:first + ns, 0, :ns]
            res = np.abs(A_gpu @ Binv.T - np.eye(ns)).max()
            assert res < (1e-11 if precision == "fp64" else 2e-5), res
    # ln|Psi| at the initial positions (single precision: FP32 Gauss-Jordan, two Newton steps
    # and the log-det anchor) against the oracle's from-scratch value
    from oracle.vmc import OracleSystem
    _, lp = w.measure()
    osys = OracleSystem(inputs)
    for wk in range(2):
        ref = osys.wf.log_psi(inputs["pos"][wk])[0]
        tol = 1e-10 * max(1.0, abs(ref)) if precision == "fp64" else logpsi_tol(136)
        assert abs(lp[wk] - ref) <= tol, (wk, lp[wk], ref)
    w.close()
    s.close()


@pytest.mark.parametrize("ns,bound", [(64, 64 * 2.0 ** -24), (256, 1e-5)])
def test_fp32_refinement_reaches_storage_accuracy(ns, bound):
    """The single-precision re-inversion (one Newton step with the error-free residual
    computed from BF16 slice products on the tensor cores: 8-bit slices at both sizes here)
    leaves an inverse whose error is set by FP32 storage, not by the condition number or the
    number of rank-k updates since the last re-inversion."""
    inputs = build_inputs(small_spec(ns, ns, grid=12, n_orb=ns + 8), n_walkers=2)
    errs = {}
    for period in (0, 16):
        s = q.system_from_inputs(inputs, precision="fp32", delay_k=4, reinv_period=period)
        w = q.Walkers(s, inputs["pos"])
        w.sweep(3)
        worst = 0.0
        for wk in range(2):
            orb = w.orbitals(wk)
            for spin in range(2):
                A = orb[ns * spin:ns * (spin + 1), 0, :ns]
                ref = np.linalg.inv(A).T
                worst = max(worst, np.abs(w.inverse(wk, spin) - ref).max() / np.abs(ref).max())
        errs[period] = worst
        w.close()
        s.close()
    print(f"N_s = {ns}: max inverse error relative to max |A^-1|: {errs}")
    assert errs[16] < bound, errs
    assert errs[16] <= errs[0], errs


@pytest.mark.parametrize("precision,delay_k", [("fp32", 8), ("bf16", 4)])
def test_mixed_precision_lockstep_odd_sizes(precision, delay_k):
    """Spin blocks of 37 and 35 electrons (not multiples of 4): the scalar load paths of the
    batched flush, the error-free residual and the Newton update, with the refinement every
    16 moves; same gates as the even-sized lockstep test."""
    inputs = build_inputs(small_spec(37, 35, grid=16), n_walkers=3)
    ids = np.arange(3)
    coef = bf16_round(inputs["coef"]) if precision == "bf16" else None
    cond = np.zeros((3, 2 * 72))
    _, ref, ref_en = oracle_vmc(inputs, ids, 2, coef=coef, conds=cond)
    forced = ref[..., 7]
    tr, en, _ = _gpu_run(inputs, ids, 2, precision=precision, delay_k=delay_k,
                         reinv_period=16, reinv_on_accepted=False, forced=forced, coef=coef,
                         logdet_period=16)
    assert_ratio_gate(tr[..., 0], ref[..., 0], cond, f"{precision} k={delay_k} 37/35")
    assert_logpsi(en[:, 1, :].T, ref_en[..., 2], 72, f"{precision} k={delay_k} 37/35")
    ne = inputs["spec"].n_elec
    assert np.max(np.abs(en[:, 0, :].T - ref_en[..., 0])) / ne < 1e-5


def test_refinement_beyond_the_exact_slice_bound_falls_back_to_fp64():
    """A spin block of 520 electrons exceeds the 512 for which the BF16 slice products of
    the error-free residual sum exactly; its re-inversion takes the FP64 Gauss-Jordan path and
    leaves an inverse at single-precision storage accuracy."""
    inputs = build_inputs(small_spec(520, 1, grid=8, n_orb=520), n_walkers=2)
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=16, reinv_period=32)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(1)
    w.check()
    for wk in range(2):
        orb = w.orbitals(wk)
        A = orb[:520, 0, :520]
        ref = np.linalg.inv(A).T
        err = np.abs(w.inverse(wk, 0) - ref).max() / np.abs(ref).max()
        assert err < 1e-4 * max(1.0, np.linalg.cond(A) * 2.0 ** -24 / 1e-4), err
    w.close()
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_proposal_batch_does_not_change_the_chain(precision):
    """The proposal batch (moves whose proposals and orbital rows one launch pair forms) is a
    launch parameter: batches of 8 and 24 moves and the whole block give identical chains.
    Delay windows end at batch ends, so bit-identical single-precision results need window
    ends that do not depend on the batch: spin blocks and the re-inversion period are
    multiples of k here, as at the benched workload (with other sizes the chains still make
    the same decisions, and the flushes round differently)."""
    inputs = build_inputs(small_spec(40, 32, grid=12), n_walkers=3)
    out = []
    for chunk in (0, 8, 24):
        s = q.system_from_inputs(inputs, precision=precision, delay_k=8, prop_chunk=chunk,
                                 reinv_period=16 if precision == "fp32" else 0,
                                 logdet_period=16 if precision == "fp32" else 0)
        w = q.Walkers(s, inputs["pos"])
        w.sweep(3)
        e, l = w.measure()
        out.append((w.positions(), e, l))
        w.close()
        s.close()
    for pos, e, l in out[1:]:
        assert np.array_equal(pos, out[0][0])
        assert np.array_equal(e, out[0][1]) and np.array_equal(l, out[0][2])
