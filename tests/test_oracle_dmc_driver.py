"""Pins of the full DMC driver in the oracle (CPU): the nodal drift rescaling of Umrigar,
Nightingale and Runge, the effective time step and the stochastic reconfiguration at a
fixed walker count (Sec. "Projector Monte Carlo", Sec. "Diffusion Monte Carlo")."""
import copy
import dataclasses
import math

import numpy as np
import pytest

from oracle.dmc import DMCPopulation, comb_counts
from oracle.philox import move_draws
from oracle.vmc import OracleSystem, drift_displacement
from synthetic import SystemSpec, build_inputs, small_spec, spec_for


# ------------------------------------------------------------------ drift rescaling
def test_rescaled_drift_closed_forms():
    tau = 0.5
    v = np.array([2.0, 0.0, 0.0])
    # a = 1: 2 a |v|^2 tau = 4, vbar tau = tau v 2 / (1 + sqrt 5)
    assert np.allclose(drift_displacement(v, tau, 1.0), [0.5 * 2.0 * 2.0 / (1.0 + math.sqrt(5.0)), 0, 0],
                       rtol=1e-15, atol=0)
    # the same from the unsimplified form (-1 + sqrt(1 + 2 a v^2 tau)) / (a v^2 tau) v tau
    a, v2 = 0.25, 4.0
    ref = (-1.0 + math.sqrt(1.0 + 2.0 * a * v2 * tau)) / (a * v2 * tau) * 2.0 * tau
    assert drift_displacement(v, tau, a)[0] == pytest.approx(ref, rel=1e-14)
    # a = 0 is the plain step
    assert np.array_equal(drift_displacement(v, tau, 0.0), tau * v)


def test_rescaled_drift_limits():
    tau, a = 0.02, 1.0
    d = np.array([0.3, -0.4, 1.2]) / 1.3
    # far from a node (|v|^2 tau << 1): the plain drift, to second order
    for vm in (1e-3, 1e-2, 0.1):
        v = vm * d
        rel = np.linalg.norm(drift_displacement(v, tau, a) - tau * v) / np.linalg.norm(tau * v)
        assert rel <= a * vm * vm * tau * 0.5 * 1.01 + 1e-15
    # next to a node (|v| -> infinity): the displacement stays below sqrt(2 tau / a), grows
    # monotonically with |v| and keeps the direction of v
    cap = math.sqrt(2.0 * tau / a)
    prev = 0.0
    for vm in (1.0, 10.0, 1e2, 1e4, 1e8):
        disp = drift_displacement(vm * d, tau, a)
        n = np.linalg.norm(disp)
        assert prev < n < cap
        assert np.allclose(disp / n, d, atol=1e-14)
        prev = n
    assert cap - prev < 1e-3 * cap


def _one_electron_system(move, step, drift_a, node=False):
    """One up electron, one orbital: 2 + cos(2 pi x / L) (no node) or cos(2 pi x / L)."""
    L = 6.0
    spec = SystemSpec("one", 1, 0, L, 16, 1, 0, "none", 0, 1, 1, move=move, step=step,
                      with_potential=False)
    amp = np.array([[0.0, 1.0]]) if node else np.array([[2.0, 1.0]])
    inputs = dict(spec=spec, seed=11, ions=np.zeros((0, 3)),
                  nvec=np.array([[[0, 0, 0], [1, 0, 0]]]), kind=np.array([[0, 0]]),
                  amp=amp, jastrow={}, rcut=L / 2, pos=np.array([[[1.0, 2.0, 3.0]]]))
    return OracleSystem(inputs, orbitals="planewave", drift_a=drift_a), L


@pytest.mark.parametrize("node", [False, True])
def test_rescaled_drift_chain_samples_psi_squared(node):
    """Drift-diffusion moves with the rescaled drift still sample |Psi|^2: the proposal and
    the Green's-function ratio of the acceptance use the same rescaled drift (a ratio built
    with the plain drift would bias the density)."""
    s, L = _one_electron_system("drift", 0.4, 1.0, node=node)
    w = s.walker([[1.0, 2.0, 3.0]], 0)
    xs = []
    for t in range(8000):
        s.sweep(w, t)
        xs.append(w.R[0, 0])
    xs = np.array(xs[200:])
    nb = 12
    edges = np.linspace(0, L, nb + 1)
    frac = np.histogram(xs, edges)[0] / xs.size
    xf = np.linspace(0, L, 20001)
    phi = np.cos(2 * np.pi * xf / L) + (0.0 if node else 2.0)
    probs = np.array([(phi[(xf >= a) & (xf < b)] ** 2).sum() for a, b in zip(edges[:-1], edges[1:])])
    probs /= probs.sum()
    assert np.abs(frac - probs).max() < 0.03, np.round(frac - probs, 3)


def test_drift_proposal_uses_the_rescaled_drift():
    """An accepted drift move lands at r + vbar tau + sqrt(tau) xi, vbar the rescaled drift
    of the current configuration."""
    spec = dataclasses.replace(small_spec(3, 3, grid=8), move="drift", step=0.3)
    d = build_inputs(spec, n_walkers=1)
    for a in (0.0, 1.0):
        s = OracleSystem(d, drift_a=a)
        w = s.walker(d["pos"][0], 0)
        R0 = w.R.copy()
        g = s.wf.grad_log_psi(w.R, 0, np.linalg.inv(w.A[0]))
        xi, _ = move_draws(s.seed, 0, 0, 0)
        forced = np.zeros(6)
        forced[0] = 1
        s.sweep(w, 0, forced=forced)
        expect = np.mod(R0[0] + drift_displacement(g, 0.3, a) + math.sqrt(0.3) * xi, spec.L)
        assert np.allclose(w.R[0], expect, rtol=0, atol=1e-12)
        assert np.array_equal(w.R[1:], R0[1:])


# ------------------------------------------------------------------ effective time step
def test_effective_time_step_bounds():
    spec = dataclasses.replace(small_spec(3, 3, grid=8), move="drift", step=0.05)
    d = build_inputs(spec, n_walkers=1)
    s = OracleSystem(d)
    for forced, frac in ((np.ones(6), 1.0), (np.zeros(6), 0.0)):
        w = s.walker(d["pos"][0], 0)
        r2 = [0.0, 0.0]
        s.sweep(w, 0, forced=forced, r2=r2)
        assert r2[0] > 0.0
        assert r2[1] == frac * r2[0]          # tau_eff = tau r2[1] / r2[0] is tau or 0


def _constant_el(tau, n, offset):
    spec = dataclasses.replace(spec_for("pw14"), move="drift", step=tau)
    d = build_inputs(spec, n_walkers=n)
    s = OracleSystem(d, orbitals="planewave")
    e_kin = 2 * 6 * (2 * np.pi / 10) ** 2 / 2
    return s, d, e_kin


def test_dmc_weights_use_the_effective_time_step():
    """With a constant E_L every weight is exp(-tau_eff (E - E_T)), tau_eff from the walker's
    own accepted and proposed squared displacements of the step."""
    tau, n = 0.4, 6
    s, d, E = _constant_el(tau, n, 0.0)
    E_T = E + 0.7
    pop = DMCPopulation(s, d["pos"], list(range(n)), E_T=E_T, capacity=4 * n, tau_eff=True)
    twins = [copy.deepcopy(w) for w in pop.walkers]
    _, _, w = pop.step(0)
    for k, tw in enumerate(twins):
        r2 = [0.0, 0.0]
        s.sweep(tw, 0, fixed_node=True, r2=r2)
        te = tau * r2[1] / r2[0]
        assert pop.last_tau_eff[k] == pytest.approx(te, rel=1e-15)
        assert w[k] == pytest.approx(math.exp(-te * (E - E_T)), rel=1e-12)
    # at this large time step some moves are rejected: tau_eff < tau for some walkers
    assert np.all(pop.last_tau_eff <= tau) and np.any(pop.last_tau_eff < tau)


# ------------------------------------------------------------------ reconfiguration
def test_comb_counts_floor_or_ceiling_and_fixed_total():
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 64):
        for _ in range(50):
            w = rng.exponential(size=n) * rng.integers(0, 2, size=n)   # some zero weights
            if w.sum() == 0:
                w[0] = 1.0
            xi = rng.uniform()
            m = comb_counts(w, xi)
            assert m.sum() == n
            exp = n * w / w.sum()
            assert np.all(m >= np.floor(exp) - 1e-9) and np.all(m <= np.ceil(exp) + 1e-9)
            assert np.all(m[w == 0] == 0)
    assert np.array_equal(comb_counts(np.ones(5), 0.37), np.ones(5))


def test_comb_counts_are_unbiased():
    w = np.array([0.1, 2.5, 0.7, 1.3, 0.05, 3.0, 0.35])
    K = 20000
    xis = (np.arange(K) + 0.5) / K          # uniform grid: the exact average over xi
    mean = np.mean([comb_counts(w, x) for x in xis], axis=0)
    assert np.allclose(mean, len(w) * w / w.sum(), atol=2.0 / K)


def test_reconfiguration_keeps_population_and_weight():
    tau, n = 0.05, 10
    s, d, E = _constant_el(tau, n, 0.0)
    # equal weights (E_T = E): the comb gives every walker exactly one copy
    pop = DMCPopulation(s, d["pos"], list(range(n)), E_T=E, capacity=4 * n, reconfigure=True)
    ids0 = [x.wid for x in pop.walkers]
    for t in range(3):
        pop.step(t)
        assert [x.wid for x in pop.walkers] == ids0
    # unequal weights (Jastrow + potential: E_L varies): N stays fixed, IDs stay unique, and
    # the total weight W of the step is what the N resampled walkers of weight W / N carry
    spec = dataclasses.replace(small_spec(4, 4, grid=8), move="drift", step=0.05)
    d2 = build_inputs(spec, n_walkers=n)
    s2 = OracleSystem(d2)
    e0 = np.mean([s2.measure(s2.walker(R, i))[0] for i, R in enumerate(d2["pos"])])
    pop2 = DMCPopulation(s2, d2["pos"], list(range(n)), E_T=e0, capacity=4 * n,
                         reconfigure=True)
    for t in range(4):
        sum_w, e_mean, w = pop2.step(t)
        assert len(pop2.walkers) == n
        ids = [x.wid for x in pop2.walkers]
        assert len(set(ids)) == n
        assert abs(n * (sum_w / n) - w.sum()) < 1e-12 * w.sum()
        assert np.ptp(w) > 0
        assert abs(pop2.E_T - e_mean) < 1e-12      # N at its target: no feedback term
