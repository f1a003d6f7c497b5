"""CUDA-graph replay of sweeps and of batched DMC steps: the chain is the same, bit for bit,
as with direct launches, while graphs are captured once per starting state and replayed.

A sweep's launches follow from host state (parameters, buffer assignment, moves since the
last re-inversion and log-det anchor); the sweep index reaches the replayed kernels through
a device word. Both halves are exercised: states that recur (the re-inversion and anchor
cadences), changes of the Hamiltonian between sweeps (new graphs), and the per-sweep index
in the Metropolis proposals, the drift moves, the pseudopotential's quadrature rotation
(index + 1) and the DMC branching draws.
"""
import dataclasses

import numpy as np
import pytest

from synthetic import build_inputs, small_spec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402


def _assert_same(a, b, what):
    ea, la = a.measure()
    eb, lb = b.measure()
    assert np.array_equal(a.positions(), b.positions()), what
    assert np.array_equal(ea, eb), what
    assert np.array_equal(la, lb), what


@pytest.mark.parametrize("precision,move,delay_k", [("fp32", "metropolis", 8),
                                                    ("fp64", "metropolis", 1),
                                                    ("fp32", "drift", 4)])
def test_sweep_graphs_match_direct_launches(precision, move, delay_k):
    step = 0.4 if move == "metropolis" else 0.03
    spec = small_spec(8, 8, grid=12, n_ion=8, move=move, step=step)
    inputs = build_inputs(spec, n_walkers=5)
    single = precision != "fp64"
    s = q.system_from_inputs(inputs, precision=precision, delay_k=delay_k,
                             reinv_period=16 if single else 0,
                             logdet_period=32 if single else 0)
    a = q.Walkers(s, inputs["pos"])            # graphs on (the default)
    b = q.Walkers(s, inputs["pos"])
    b.graphs(False)
    l0a, l0b = a.launch_count(), b.launch_count()
    n = 0
    for phase, n_sweeps in enumerate((8, 4, 4)):
        if phase == 1:                         # a new Hamiltonian term: new graphs
            s.set_nonlocal(np.array([1.2, -0.8]), np.array([1.0, 0.9]), 1.8)
        if phase == 2:
            s.set_ewald(9.0 / spec.L, 2 * 9.0 / spec.L * 4.5)
        for _ in range(n_sweeps):
            a.sweep(1)
            b.sweep(1)
            n += 1
            _assert_same(a, b, f"{precision} {move} phase {phase} sweep {n}")
    captures, replays = a.graph_stats()
    assert replays == n
    assert 3 <= captures < n                    # states recur within a phase
    assert b.graph_stats() == (0, 0)
    # the graphs carry the same kernels, plus the one that sets the sweep index
    assert a.launch_count() - l0a == b.launch_count() - l0b + replays
    a.close()
    b.close()
    s.close()


def test_sweep_graphs_several_sweeps_per_call_and_toggling():
    """Several sweeps per call, and replay switched off and on between calls: the sweep
    counter and the host state stay consistent with the device."""
    spec = small_spec(8, 8, grid=12)
    inputs = build_inputs(spec, n_walkers=4)
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=8, reinv_period=16,
                             logdet_period=32)
    a = q.Walkers(s, inputs["pos"])
    b = q.Walkers(s, inputs["pos"])
    b.graphs(False)
    a.sweep(3)
    b.sweep(3)
    _assert_same(a, b, "three sweeps in one call")
    a.graphs(False)
    a.sweep(2)
    b.sweep(2)
    _assert_same(a, b, "replay off")
    a.graphs(True)
    a.sweep(3)
    b.sweep(3)
    _assert_same(a, b, "replay on again")
    assert a.graph_stats()[1] == 6
    a.close()
    b.close()
    s.close()


def _dmc_systems(precision):
    # spin blocks of 4, 8 and 12 electrons with a refinement every 4 moves and an anchor every
    # 8: every walker set returns to its starting state within two of its sweeps
    systems, pos, et = [], [], []
    for n_up, n_dn, nw in ((4, 4, 8), (8, 8, 6), (12, 12, 4)):
        spec = dataclasses.replace(small_spec(n_up, n_dn, grid=10), move="drift", step=0.05)
        inputs = build_inputs(spec, n_walkers=nw)
        kw = dict(delay_k=4)
        if precision == "fp32":
            kw.update(reinv_period=4, logdet_period=8)
        s = q.system_from_inputs(inputs, precision=precision, move="drift", step=0.05,
                                 drift_a=1.0, **kw)
        w = q.Walkers(s, inputs["pos"])
        e, _ = w.measure()
        w.close()
        systems.append(s)
        pos.append(inputs["pos"])
        et.append(float(np.mean(e)))
    return systems, pos, et


@pytest.mark.parametrize("precision,reconfigure", [("fp64", False), ("fp32", False),
                                                   ("fp32", True)])
def test_dmc_step_graphs_match_direct_launches(precision, reconfigure):
    """Three systems of uneven size in one driver: one graph per step over all of them,
    against the same driver stepping by direct launches on per-system streams."""
    systems, pos, et = _dmc_systems(precision)
    a = q.DMC(systems, pos, et, capacity_factor=2)
    b = q.DMC(systems, pos, et, capacity_factor=2)
    b.graphs(False)
    for d in (a, b):
        d.set_mode(effective_tau=True, reconfigure=reconfigure)
    steps = 8
    for t in range(steps):
        a.step(1)
        b.step(1)
        for i in range(len(systems)):
            ra, rb = a.read(i), b.read(i)
            assert ra == rb, (t, i, ra, rb)
            for x, y in zip(a.walkers(i), b.walkers(i)):
                assert np.array_equal(x, y), (t, i)
    captures, replays = a.graph_stats()
    assert replays == steps and 1 <= captures < steps
    a.close()
    b.close()
    for s in systems:
        s.close()
