"""GPU parity at the full workload sizes, in the launch configuration the bench times
(all walkers, mixed precision, delayed rank-k, re-inversion cadence), on sampled outputs
the FP64 oracle can compute one by one:

* the first moves of sampled walkers: every move's relative ratio error (floor 1e-3) within
  the per-move gate max(1e-4, cond 2^-24) of parity_util, with cond the oracle's condition
  number of the moved spin block, and the same accept decisions up to the first decision
  that sits at u ~ A within twice that gate (after a legitimate flip the chains differ, so
  the comparison stops there);
* the local energy of sampled walkers at the GPU's final configuration within
  1e-5 Ha per electron of the oracle's value at the same positions;
* the inverse of sampled walkers against the orbital matrix at the final positions.
"""
import numpy as np
import pytest

from synthetic import build_inputs, spec_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.vmc import OracleSystem   # noqa: E402
from parity_util import logpsi_tol, ratio_gate   # noqa: E402

CASES = [
    # preset, precision, delay k, re-inversion period, counted on accepted moves,
    # sampled walkers, sampled moves
    ("sj512", "fp32", 32, 128, False, (0, 129), 40),    # the benched configuration
    ("sj512", "fp32", 16, 128, False, (3,), 40),
    ("sj512", "bf16", 16, 128, False, (7,), 24),
    ("sj128", "fp32", 16, 64, True, (0, 300), 64),
    ("sj1024", "fp32", 32, 256, False, (5,), 20),
]


@pytest.mark.parametrize("preset,precision,k,period,on_acc,sample,n_moves", CASES)
def test_full_size_sampled_parity(preset, precision, k, period, on_acc, sample, n_moves):
    spec = spec_for(preset)
    inputs = build_inputs(spec)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=k, reinv_period=period,
                             reinv_on_accepted=on_acc, logdet_period=0 if on_acc else period)
    w = q.Walkers(s, inputs["pos"])
    ne, nw = spec.n_elec, spec.n_walkers
    buf = torch.zeros((nw, ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    w.sweep(1)
    e_gpu, lp_gpu = w.measure()
    tr = buf.cpu().numpy()
    final = w.positions()
    acc = tr[..., 7].mean()
    assert 0.3 < acc < 0.95, acc
    coef = inputs["coef"]
    if precision == "bf16":
        from parity_util import bf16_round
        coef = bf16_round(coef)
    osys = OracleSystem(inputs, coef=coef)
    errs, worst = [], 0.0
    for wid in sample:
        ow = osys.walker(inputs["pos"][wid], wid)
        rows, conds = [], []
        osys.sweep(ow, 0, trace=rows, electrons=range(n_moves), conds=conds)
        ref = np.array(rows)
        got = tr[wid, :n_moves]
        for mv in range(n_moves):
            err, bound = ratio_gate(got[mv, 0], ref[mv, 0], conds[mv])
            errs.append(float(err))
            worst = max(worst, float(err / bound))
            assert err <= bound, (wid, mv, float(err), float(bound), conds[mv])
            assert got[mv, 5] == ref[mv, 5]
            if got[mv, 7] != ref[mv, 7]:
                assert abs(ref[mv, 5] - ref[mv, 6]) <= 2 * bound * ref[mv, 6] + 1e-12, (wid, mv)
                break
        # local energy at the GPU's final configuration
        fw = osys.walker(final[wid], wid)
        e_ref, _, lp_ref = osys.measure(fw)
        assert abs(e_gpu[wid] - e_ref) / ne < 1e-5, (wid, e_gpu[wid], e_ref)
        print(f"{preset} {precision} k={k} walker {wid}: ln|Psi| error {lp_gpu[wid] - lp_ref:.2e}")
        if not on_acc:       # anchored at every re-inversion (the batched form)
            assert abs(lp_gpu[wid] - lp_ref) <= logpsi_tol(ne), (wid, lp_gpu[wid] - lp_ref)
        # the inverse of each spin block against the orbital values at the final positions
        orb = w.orbitals(wid)
        for spin, (first, ns) in enumerate(((0, spec.n_up), (spec.n_up, spec.n_dn))):
            A = orb[first:first + ns, 0, :ns]
            res = np.abs(A @ w.inverse(wid, spin).T - np.eye(ns)).max()
            assert res < 1e-3, (wid, spin, res)
    errs = np.array(errs)
    print(f"{preset} {precision} k={k}: ratio rel err median {np.median(errs):.2e} "
          f"p90 {np.quantile(errs, 0.9):.2e} p99 {np.quantile(errs, 0.99):.2e} "
          f"max {errs.max():.2e}; worst err/bound {worst:.3f}")
    w.close()
    s.close()


@pytest.mark.parametrize("precision,anchor", [("fp32", 128), ("bf16", 128), ("fp32", 1024)])
def test_logpsi_over_many_sweeps(precision, anchor):
    """ln|Psi| and E_L of the single-precision forms stay tied to the FP64 oracle over 56
    sweeps of the 512-electron workload in the bench's launch form (k = 32, whole-block
    proposal batches formed beside the other block's moves, every sweep a CUDA-graph replay,
    re-inversion every 128 moves, log-determinant anchor every `anchor` moves; 1024 is the
    bench's cadence): the oracle recomputes both from scratch at the GPU's final positions of
    sampled walkers. 56 sweeps (14336 moves per spin block) end right after an anchor for both
    cadences, so the ln|Psi| gate is the single-precision floor; the drift the anchors removed
    along the way (their shifts) is reported."""
    spec = spec_for("sj512")
    inputs = build_inputs(spec)
    coef = inputs["coef"]
    if precision == "bf16":
        from parity_util import bf16_round
        coef = bf16_round(coef)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=32, reinv_period=128,
                             logdet_period=anchor)
    w = q.Walkers(s, inputs["pos"])
    shifts, resid = [], []
    for _ in range(56):
        w.sweep(1)
        res, shift = w.precision_report()
        shifts.append(shift.ravel())
        resid.append(res.ravel())
    assert w.graph_stats()[1] == 56                   # every sweep replayed, as in the bench
    e_gpu, lp = w.measure()
    final = w.positions()
    osys = OracleSystem(inputs, coef=coef)
    errs = [lp[wid] - osys.wf.log_psi(final[wid])[0] for wid in (0, 101, 255)]
    for wid in (0, 101, 255):
        e_ref = osys.measure(osys.walker(final[wid], wid))[0]
        assert abs(e_gpu[wid] - e_ref) / spec.n_elec < 1e-5, (wid, e_gpu[wid], e_ref)
    sh = np.abs(np.concatenate(shifts))
    sh = sh[np.isfinite(sh)]                      # NaN before a walker's first anchor
    print(f"{precision} anchor {anchor}: ln|Psi| error after 56 sweeps {np.round(errs, 7)}; anchor "
          f"shifts median {np.median(sh):.2e} p99 {np.quantile(sh, 0.99):.2e} max {sh.max():.2e}")
    assert sh.size > 0
    assert np.max(np.abs(errs)) <= logpsi_tol(spec.n_elec), errs
    # max |I - A X| before the Newton step of each re-inversion (the last one of each spin
    # block per sweep): one step leaves about its square, so values up to 2^-12 end at
    # single-precision storage accuracy
    r = np.concatenate(resid)
    r = r[np.isfinite(r)]
    edges = [0, 1e-6, 3e-6, 1e-5, 3e-5, 1e-4, 2.0 ** -12, 5e-4, 1e-3, 1e-2, np.inf]
    print(f"{precision} anchor {anchor}: residual before the Newton step: n {r.size} median "
          f"{np.median(r):.2e} p90 {np.quantile(r, 0.9):.2e} p99 {np.quantile(r, 0.99):.2e} "
          f"max {r.max():.2e}; histogram over {[f'{e:.3g}' for e in edges]}: "
          f"{np.histogram(r, bins=edges)[0].tolist()}")
    assert np.mean(r <= 2.0 ** -12) > 0.98
    w.close()
    s.close()
