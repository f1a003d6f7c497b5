"""GPU parity of drift-diffusion moves and branching DMC against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from synthetic import build_inputs, small_spec, spec_for

from parity_util import (assert_ratio_gate, assert_trace_close, bf16_round, logpsi_tol,
                         rel_err)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.dmc import DMCPopulation   # noqa: E402
from oracle.vmc import OracleSystem, run_vmc   # noqa: E402


def _drift_inputs(n_up, n_dn, tau, n_walkers, grid=10):
    spec = dataclasses.replace(small_spec(n_up, n_dn, grid=grid), move="drift", step=tau)
    return build_inputs(spec, n_walkers=n_walkers)


@pytest.mark.parametrize("delay_k", [1, 4])
def test_drift_vmc_fp64_parity(delay_k):
    inputs = _drift_inputs(9, 8, 0.05, 2)
    ids = np.arange(2)
    s = q.system_from_inputs(inputs, precision="fp64", delay_k=delay_k)
    w = q.Walkers(s, inputs["pos"])
    buf = torch.zeros((2, 2, 17, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    en = []
    for _ in range(2):
        w.sweep(1)
        en.append(w.measure())
    tr = buf.cpu().numpy().transpose(1, 0, 2, 3).reshape(2, 34, 8)
    _, ref, ref_en = run_vmc(OracleSystem(inputs), inputs["pos"], ids, 2)
    assert_trace_close(tr, ref, 1e-10)
    assert np.all(rel_err(np.array(en)[:, 0, :].T, ref_en[..., 0], 1.0) < 1e-10)
    w.close()
    s.close()


@pytest.mark.parametrize("delay_k", [1, 4])
def test_branching_dmc_fp64_parity(delay_k):
    tau, nw, steps = 0.02, 8, 3
    inputs = _drift_inputs(6, 5, tau, nw)
    osys = OracleSystem(inputs)
    e0 = np.mean([osys.measure(osys.walker(R, i))[0] for i, R in enumerate(inputs["pos"])])
    pop = DMCPopulation(osys, inputs["pos"], list(range(nw)), E_T=e0, capacity=2 * nw)
    s = q.system_from_inputs(inputs, precision="fp64", delay_k=delay_k, move="drift", step=tau)
    d = q.DMC([s], [inputs["pos"]], [e0], capacity_factor=2)
    branched = False
    for t in range(steps):
        sum_w, e_mean, _ = pop.step(t)
        d.step(1)
        st = d.read(0)
        pos, ids, el = d.walkers(0)
        ref_ids = np.array([w.wid for w in pop.walkers])
        assert st["population"] == len(pop.walkers) > 0
        assert np.array_equal(ids, ref_ids), (ids, ref_ids)
        assert np.allclose(pos, np.array([w.R for w in pop.walkers]), rtol=0, atol=1e-10)
        assert np.allclose(el, pop.E_L, rtol=1e-10, atol=1e-10)
        assert abs(st["sum_w"] - sum_w) < 1e-10 * sum_w
        assert abs(st["e_mean"] - e_mean) < 1e-10 * max(1.0, abs(e_mean))
        assert abs(st["e_trial_next"] - pop.E_T) < 1e-10 * max(1.0, abs(pop.E_T))
        assert st["next_id"] == pop.next_id
        branched |= st["population"] != st["population_before"] or len(set(ids)) != len(ids) or max(ids) >= nw
    assert branched, "no branching event: the test does not exercise copies or deaths"
    d.close()
    s.close()


def test_dmc_three_uneven_systems_run_together():
    """The three systems of the batched DMC workload (64, 192, 384 electrons) at reduced
    walker counts advance together; populations stay within capacity, energies finite."""
    systems, pos, et = [], [], []
    for name, nw in (("dmc64", 24), ("dmc192", 16), ("dmc384", 8)):
        inputs = build_inputs(spec_for(name), n_walkers=nw)
        s = q.system_from_inputs(inputs, precision="fp32", delay_k=16)
        w = q.Walkers(s, inputs["pos"])
        e, _ = w.measure()
        w.close()
        systems.append(s)
        pos.append(inputs["pos"])
        et.append(float(np.mean(e)))
    d = q.DMC(systems, pos, et, capacity_factor=2)
    d.step(3)
    for i, nw in enumerate((24, 16, 8)):
        st = d.read(i)
        assert 0 < st["population"] <= 2 * nw
        assert np.isfinite(st["e_mean"]) and np.isfinite(st["e_trial_next"])
        _, ids, el = d.walkers(i)
        assert len(set(ids.tolist())) == len(ids) and np.all(np.isfinite(el))
    assert d.launch_count() > 0
    d.close()
    for s in systems:
        s.close()


def test_branching_saturates_at_capacity_with_huge_weights():
    """A trial energy 2000 Ha above E_L gives weights near e^40 (beyond 2^31 copies): the
    population fills the capacity with copies in parent order, exactly as the oracle drops
    every copy beyond it, and the next step proceeds normally."""
    tau, nw = 0.02, 8
    inputs = _drift_inputs(6, 5, tau, nw)
    osys = OracleSystem(inputs)
    e0 = np.mean([osys.measure(osys.walker(R, i))[0] for i, R in enumerate(inputs["pos"])])
    et = e0 + 2000.0
    pop = DMCPopulation(osys, inputs["pos"], list(range(nw)), E_T=et, capacity=2 * nw)
    s = q.system_from_inputs(inputs, precision="fp64", delay_k=1, move="drift", step=tau)
    d = q.DMC([s], [inputs["pos"]], [et], capacity_factor=2)
    for t in range(2):
        sum_w, e_mean, _ = pop.step(t)
        d.step(1)
        st = d.read(0)
        _, ids, el = d.walkers(0)
        assert st["population"] == len(pop.walkers)
        assert np.array_equal(ids, np.array([w.wid for w in pop.walkers]))
        assert np.allclose(el, pop.E_L, rtol=1e-10, atol=1e-10)
        assert abs(st["sum_w"] - sum_w) < 1e-10 * sum_w
        assert st["next_id"] == pop.next_id
    assert len(pop.walkers) > 0
    d.close()
    s.close()


def test_dmc_uneven_systems_with_refinement():
    """Batched DMC with the single-precision inverse refined every 32 moves: empty slots of
    the capacity-padded buffers are skipped by every kernel (no error flag), populations stay
    within capacity and energies finite over several steps."""
    systems, pos, et, caps = [], [], [], []
    for name, nw in (("dmc64", 48), ("dmc192", 24), ("dmc384", 12)):
        inputs = build_inputs(spec_for(name), n_walkers=nw)
        s = q.system_from_inputs(inputs, precision="fp32", delay_k=16, reinv_period=32)
        w = q.Walkers(s, inputs["pos"])
        e, _ = w.measure()
        w.close()
        systems.append(s)
        pos.append(inputs["pos"])
        et.append(float(np.mean(e)))
        caps.append(2 * nw)
    d = q.DMC(systems, pos, et, capacity_factor=2)
    for _ in range(6):
        d.step(1)
        for i, cap in enumerate(caps):
            st = d.read(i)                   # raises on any device error flag
            assert 0 < st["population"] <= cap
            assert np.isfinite(st["e_mean"])
    d.close()
    for s in systems:
        s.close()


@pytest.mark.parametrize("precision,delay_k", [("fp32", 4), ("bf16", 8)])
def test_drift_vmc_mixed_precision_lockstep(precision, delay_k):
    """Drift-diffusion VMC in the single-precision forms (the DMC workload's arithmetic) with
    the error-free refinement every 16 moves, replaying the oracle's decisions: the per-move
    ratio gate of parity_util (1e-4 relative, or cond 2^-24); E_L at the GPU's positions
    within 1e-5 Ha per electron, or within the single-precision storage bound
    cond(A) 2^-24 |T_L| of a near-node configuration. The proposal r' uses the GPU's own
    gradient, which differs from the oracle's by ~1e-5 relative, far below these gates."""
    inputs = _drift_inputs(20, 18, 0.05, 3, grid=12)
    ids = np.arange(3)
    coef = bf16_round(inputs["coef"]) if precision == "bf16" else None
    osys = OracleSystem(inputs, coef=coef)
    move_cond = np.zeros((3, 2 * 38))
    _, ref, ref_en = run_vmc(osys, inputs["pos"], ids, 2, conds=move_cond)
    d = dict(inputs)
    if coef is not None:
        d["coef"] = coef
    s = q.system_from_inputs(d, precision=precision, delay_k=delay_k, reinv_period=16,
                             logdet_period=16)
    w = q.Walkers(s, inputs["pos"])
    ne = s.n_up + s.n_dn
    buf = torch.zeros((2, 3, ne, 8), dtype=torch.float64, device="cuda")
    w.trace_enable(buf)
    bits = np.ascontiguousarray(ref[..., 7].reshape(3, 2, ne).transpose(1, 0, 2).astype(np.uint8))
    w.replay(bits, 2)
    el_err = []
    lp_err = []
    for _ in range(2):
        w.sweep(1)
        e_gpu, lp_gpu = w.measure()
        pos = w.positions()
        lp_err += [abs(lp_gpu[i] - osys.wf.log_psi(pos[i])[0]) for i in range(3)]
        # E_L against the oracle at the GPU's own positions. Gate: 1e-5 Ha per electron, or
        # the single-precision storage bound cond(A) 2^-24 |T_L| where that is larger (a
        # configuration next to a node: E_L an outlier, A ill-conditioned)
        for i in range(3):
            e_ref, t_ref = osys.wf.local_energy(pos[i])
            cond = max(np.linalg.cond(osys.wf.slater_matrix(pos[i], sp)) for sp in (0, 1))
            bound = max(1e-5, cond * 2.0 ** -24 * abs(t_ref) / ne)
            el_err.append(abs(e_gpu[i] - e_ref) / ne / bound)
    tr = buf.cpu().numpy().transpose(1, 0, 2, 3).reshape(3, 2 * ne, 8)
    print(f"drift {precision} k={delay_k}: E_L error / gate {np.round(el_err, 3)}; "
          f"ln|Psi| error max {max(lp_err):.2e}")
    assert_ratio_gate(tr[..., 0], ref[..., 0], move_cond, f"drift {precision} k={delay_k}")
    assert max(el_err) < 1.0
    assert max(lp_err) <= logpsi_tol(ne), (max(lp_err), logpsi_tol(ne))
    # the trajectories agree closely: same decisions, proposals from nearly equal gradients
    ref_pos = np.array([wk.R for wk in run_vmc(osys, inputs["pos"], ids, 2)[0]])
    assert np.abs(pos - ref_pos).max() < 1e-3
    w.close()
    s.close()


@pytest.mark.parametrize("reconfigure", [False, True])
def test_dmc_driver_fp64_parity_three_uneven_systems(reconfigure):
    """The full DMC driver (Sec. "Diffusion Monte Carlo"): drift rescaled near nodes
    (Umrigar, Nightingale and Runge, a = 1), the effective time step in the branching factor,
    and either branching or stochastic reconfiguration at a fixed walker count, for three
    systems of uneven size advancing together in one driver. FP64: walker IDs, positions,
    local energies, weight sums, E_T and the next free ID equal the oracle's to 1e-10."""
    tau, steps = 0.05, 3
    specs = ((6, 5, 8), (8, 7, 6), (12, 11, 4))
    systems, pops, pos0, e0s = [], [], [], []
    for n_up, n_dn, nw in specs:
        inputs = _drift_inputs(n_up, n_dn, tau, nw)
        osys = OracleSystem(inputs, drift_a=1.0)
        e0 = float(np.mean([osys.measure(osys.walker(R, i))[0] for i, R in enumerate(inputs["pos"])]))
        pops.append(DMCPopulation(osys, inputs["pos"], list(range(nw)), E_T=e0, capacity=2 * nw,
                                  tau_eff=True, reconfigure=reconfigure))
        systems.append(q.system_from_inputs(inputs, precision="fp64", delay_k=4, move="drift",
                                            step=tau, drift_a=1.0))
        pos0.append(inputs["pos"])
        e0s.append(e0)
    d = q.DMC(systems, pos0, e0s, capacity_factor=2)
    d.set_mode(effective_tau=True, reconfigure=reconfigure)
    copied = False
    for t in range(steps):
        ref = [pop.step(t) for pop in pops]
        d.step(1)
        for i, (pop, (sum_w, e_mean, w)) in enumerate(zip(pops, ref)):
            st = d.read(i)
            pos, ids, el = d.walkers(i)
            ref_ids = np.array([x.wid for x in pop.walkers])
            assert st["population"] == len(pop.walkers) > 0
            if reconfigure:
                assert st["population"] == specs[i][2]
            assert np.array_equal(ids, ref_ids), (i, t, ids, ref_ids)
            assert np.allclose(pos, np.array([x.R for x in pop.walkers]), rtol=0, atol=1e-10)
            assert np.allclose(el, pop.E_L, rtol=1e-10, atol=1e-10)
            assert abs(st["sum_w"] - sum_w) < 1e-10 * sum_w
            assert abs(st["e_mean"] - e_mean) < 1e-10 * max(1.0, abs(e_mean))
            assert abs(st["e_trial_next"] - pop.E_T) < 1e-10 * max(1.0, abs(pop.E_T))
            assert st["next_id"] == pop.next_id
            assert np.any(pop.last_tau_eff < tau)        # some moves rejected: tau_eff active
            copied |= max(ids) >= specs[i][2]
    assert copied, "no walker was copied: the test does not exercise the population control"
    d.close()
    for s in systems:
        s.close()
