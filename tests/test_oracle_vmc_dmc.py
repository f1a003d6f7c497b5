"""Pins of the oracle's Monte Carlo steps: Metropolis and drift-diffusion chains sample
|Psi|^2, null moves are always accepted, DMC weights follow Eq. pmc:g_growth (CPU)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle.dmc import DMCPopulation
from oracle.vmc import OracleSystem, run_vmc
from synthetic import SystemSpec, build_inputs, small_spec, spec_for


def _one_electron_system(move, step):
    """One up electron, one orbital phi = 2 + cos(2 pi x / L): |phi|^2 is known exactly."""
    L = 6.0
    spec = SystemSpec("one", 1, 0, L, 16, 1, 0, "none", 0, 1, 1, move=move, step=step,
                      with_potential=False)
    inputs = dict(spec=spec, seed=11, ions=np.zeros((0, 3)),
                  nvec=np.array([[[0, 0, 0], [1, 0, 0]]]), kind=np.array([[0, 0]]),
                  amp=np.array([[2.0, 1.0]]), jastrow={}, rcut=L / 2,
                  pos=np.array([[[1.0, 2.0, 3.0]]]))
    return OracleSystem(inputs, orbitals="planewave"), L


@pytest.mark.parametrize("move,step", [("metropolis", 1.5), ("drift", 0.4)])
def test_chain_samples_psi_squared(move, step):
    s, L = _one_electron_system(move, step)
    w = s.walker([[1.0, 2.0, 3.0]], 0)
    xs = []
    for t in range(6000):
        s.sweep(w, t)
        xs.append(w.R[0, 0])
    xs = np.array(xs[200:])
    nb = 12
    edges = np.linspace(0, L, nb + 1)
    counts = np.histogram(xs, edges)[0]
    xf = np.linspace(0, L, 20001)
    dens = (2 + np.cos(2 * np.pi * xf / L)) ** 2
    probs = np.array([dens[(xf >= a) & (xf < b)].sum() for a, b in zip(edges[:-1], edges[1:])])
    probs /= probs.sum()
    # a Markov chain is correlated: compare with a loose bound on the binned deviations
    frac = counts / counts.sum()
    assert np.abs(frac - probs).max() < 0.025
    # a wrong acceptance rule (e.g. ratio instead of ratio^2) gives a visibly flatter density
    ratio_ends = frac[[0, -1]].mean() / frac[nb // 2 - 1: nb // 2 + 1].mean()
    assert abs(ratio_ends - 9.0) < 2.5           # (2+1)^2 / (2-1)^2 = 9


def test_null_move_always_accepted():
    d = build_inputs(small_spec(3, 3, grid=8, step=0.0), n_walkers=1)
    s = OracleSystem(d)
    _, tr, _ = run_vmc(s, d["pos"], [0], 1)
    assert np.allclose(tr[0, :, 0], 1.0, atol=1e-12)     # ratio
    assert np.allclose(tr[0, :, 1], 0.0, atol=1e-12)     # dJ
    assert np.all(tr[0, :, 7] == 1.0)


def test_trace_is_consistent_with_the_acceptance_rule():
    d = build_inputs(small_spec(4, 4, grid=10), n_walkers=2)
    s = OracleSystem(d)
    _, tr, en = run_vmc(s, d["pos"], [0, 1], 2)
    ratio, dJ, u, A, acc = tr[..., 0], tr[..., 1], tr[..., 5], tr[..., 6], tr[..., 7]
    assert np.allclose(A, np.minimum(1, ratio ** 2 * np.exp(2 * dJ)))
    assert np.all((u < A) == (acc == 1))
    assert 0.1 < acc.mean() < 0.95


def test_replayed_decisions_reproduce_the_trajectory():
    d = build_inputs(small_spec(3, 3, grid=8), n_walkers=1)
    s = OracleSystem(d)
    w1, tr, en = run_vmc(s, d["pos"], [0], 2)
    w2, tr2, en2 = run_vmc(s, d["pos"], [0], 2, forced=[tr[0, :, 7]])
    assert np.array_equal(tr, tr2) and np.array_equal(en, en2)
    flipped = tr[0, :, 7].copy()
    flipped[0] = 1 - flipped[0]
    _, tr3, _ = run_vmc(s, d["pos"], [0], 2, forced=[flipped])
    assert tr3[0, 0, 7] == flipped[0]


def test_dmc_weights_with_constant_local_energy():
    spec = dataclasses.replace(spec_for("pw14"), move="drift", step=0.01)
    d = build_inputs(spec, n_walkers=8)
    s = OracleSystem(d, orbitals="planewave")
    e_kin = 2 * 6 * (2 * np.pi / 10) ** 2 / 2
    E_T = e_kin + 0.3
    pop = DMCPopulation(s, d["pos"], list(range(8)), E_T=E_T, capacity=16)
    assert np.allclose(pop.E_L, e_kin, atol=1e-10)
    sum_w, e_mean, w = pop.step(0)
    assert np.allclose(w, math.exp(-0.01 * (e_kin - E_T)), rtol=1e-12)
    assert abs(e_mean - e_kin) < 1e-10
    assert abs(sum_w - 8 * w[0]) < 1e-12
    # weights ~ 1.003: every walker survives once, a few copy (draw-dependent), cap respected
    assert 8 <= len(pop.walkers) <= 16
    ids = [x.wid for x in pop.walkers]
    assert len(set(ids)) == len(ids)


def test_fixed_node_rejects_sign_changes():
    spec = dataclasses.replace(spec_for("pw14"), move="drift", step=0.5)
    d = build_inputs(spec, n_walkers=2)
    s = OracleSystem(d)
    for wid, R in enumerate(d["pos"]):
        w = s.walker(R, wid)
        rows = []
        for t in range(3):
            s.sweep(w, t, fixed_node=True, trace=rows)
        rows = np.array(rows)
        assert not np.any((rows[:, 0] < 0) & (rows[:, 7] == 1))


def _constant_el_population(offset, n=8, capacity=64, tau=0.05):
    """Plane-wave determinant without Jastrow or potential: E_L is the same constant for
    every configuration, so the branching weights depend on E_T alone."""
    spec = dataclasses.replace(spec_for("pw14"), move="drift", step=tau)
    d = build_inputs(spec, n_walkers=n)
    s = OracleSystem(d, orbitals="planewave")
    e_kin = 2 * 6 * (2 * np.pi / 10) ** 2 / 2
    return DMCPopulation(s, d["pos"], list(range(n)), E_T=e_kin + offset,
                         capacity=capacity), e_kin


def test_dmc_population_control_fixed_point():
    # E_T equal to the constant E_L and the population at its target: every weight is one,
    # each walker survives exactly once under its own ID, and E_T stays put
    pop, E = _constant_el_population(0.0)
    ids0 = [x.wid for x in pop.walkers]
    for t in range(6):
        sum_w, e_mean, w = pop.step(t)
        assert np.allclose(w, 1.0, rtol=0, atol=1e-12)
        assert [x.wid for x in pop.walkers] == ids0
        assert abs(pop.E_T - E) < 1e-10


def test_dmc_population_control_is_negative_feedback():
    # twelve walkers against a target of eight, E_T at the constant E_L: the trial-energy
    # feedback must lower E_T and bring the population back to the target instead of letting
    # it run away (a feedback of the wrong sign reaches the capacity within about 20 steps)
    pop, E = _constant_el_population(0.0, n=12, capacity=64)
    pop.n_target = 8
    sizes, e_t = [], []
    for t in range(60):
        pop.step(t)
        sizes.append(len(pop.walkers))
        e_t.append(pop.E_T)
    assert 0 < min(sizes) and max(sizes) < 24, sizes
    assert 4 <= np.mean(sizes[-30:]) <= 12, sizes
    assert e_t[0] < E                         # above the target: E_T drops below E_L
    assert abs(np.mean(e_t[-30:]) - E) < 1.0
    ids = [x.wid for x in pop.walkers]
    assert len(set(ids)) == len(ids)


def test_dmc_branching_ids_stay_unique_under_growth():
    # weights near 2.5: every walker leaves two or three copies; the IDs of the population
    # stay unique and the copies stay within the capacity
    pop, E = _constant_el_population(math.log(2.5) / 0.05, n=6, capacity=40)
    for t in range(3):
        pop.step(t)
        ids = [x.wid for x in pop.walkers]
        assert len(set(ids)) == len(ids)
        assert len(ids) <= 40
    assert len(pop.walkers) > 6
