"""The regrouping behind the pair-matrix sweep, checked on the CPU against the oracle.

Within a launch of the batched delayed update the inverse A0^-1 is fixed and the proposals
r'_t of the launch's moves are known. The sweep then takes every dot product from
D[a][b] = phi'_a . A0^-1[:, e_b] and every Jastrow difference from a value at the launch-start
positions plus pair corrections between the launch's own moves. This test restates those
formulas in numpy, replays a launch with a fixed accept/reject pattern, and compares each
move's determinant ratio and Jastrow difference with the oracle's direct values (ratio of
determinants of the current Slater matrices, J of the current configuration)."""
import numpy as np
import pytest

from oracle.jastrow import functor, min_image
from oracle.vmc import OracleSystem
from synthetic import build_inputs, small_spec


def _direct(osys, R0, moves, props, accepted):
    """The oracle's values move by move on the evolving configuration."""
    R = R0.copy()
    ratios, djs = [], []
    for t, e in enumerate(moves):
        A = osys.wf.slater_matrix(R, 0)
        Rn = R.copy()
        Rn[e] = props[t]
        An = osys.wf.slater_matrix(Rn, 0)
        ratios.append(np.linalg.det(An) / np.linalg.det(A))
        djs.append(osys.wf.jas.value(Rn) - osys.wf.jas.value(R))
        if accepted[t]:
            R = Rn
    return np.array(ratios), np.array(djs)


def _regrouped(osys, R0, moves, props, accepted, L, rc, p_same):
    """The pair-matrix form: D, the window solve by bordering, base + Q."""
    kk = len(moves)
    A0 = osys.wf.slater_matrix(R0, 0)
    A0inv = np.linalg.inv(A0)                     # column e: the inverse row of electron e
    ns = A0.shape[0]
    phi = np.array([osys.wf.orb.values(props[t])[:ns] for t in range(kk)])
    D = phi @ A0inv[:, moves]                     # D[a][b] = phi'_a . A0^-1[:, e_b]
    # Jastrow: the difference at the launch-start positions and the pair corrections
    J0 = osys.wf.jas.value(R0)
    base = np.empty(kk)
    for t, e in enumerate(moves):
        Rn = R0.copy()
        Rn[e] = props[t]
        base[t] = osys.wf.jas.value(Rn) - J0

    def u(a, b):
        d = min_image(np.asarray(a) - np.asarray(b), L)
        return functor(np.array([np.sqrt((d * d).sum())]), p_same, rc)[0][0]

    Q = np.zeros((kk, kk))
    for a in range(kk):
        for b in range(kk):
            if a != b:
                ra, rb = props[a], props[b]
                oa, ob = R0[moves[a]], R0[moves[b]]
                Q[a, b] = u(ra, rb) - u(ra, ob) - u(oa, rb) + u(oa, ob)
    win, Cinv = [], np.zeros((0, 0))
    ratios, djs = [], []
    for t in range(kk):
        m = len(win)
        d = np.array([D[l, t] for l in win])
        crow = np.array([D[t, l] for l in win])
        y = Cinv.T @ crow if m else np.zeros(0)
        z = Cinv @ d if m else np.zeros(0)
        R = D[t, t] - y @ d                       # the Schur complement of the bordered C
        ratios.append(R)
        djs.append(base[t] + sum(Q[t, l] for l in win))
        if accepted[t]:
            s = 1.0 / R
            Cn = np.empty((m + 1, m + 1))
            Cn[:m, :m] = Cinv + np.outer(z, y) * s
            Cn[:m, m] = -z * s
            Cn[m, :m] = -y * s
            Cn[m, m] = s
            Cinv = Cn
            win.append(t)
    return np.array(ratios), np.array(djs)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pair_matrix_regrouping_matches_direct_values(seed):
    spec = small_spec(9, 8, grid=12, n_walkers=1)
    inputs = build_inputs(spec, n_walkers=1, seed=seed)
    osys = OracleSystem(inputs)
    rng = np.random.default_rng(100 + seed)
    R0 = np.mod(inputs["pos"][0], spec.L)
    moves = [1, 2, 3, 5, 6, 8]                    # one launch: consecutive up-spin moves
    props = np.mod(R0[moves] + 0.3 * rng.standard_normal((len(moves), 3)), spec.L)
    accepted = [True, False, True, True, False, True]
    j = inputs["jastrow"]
    r_dir, j_dir = _direct(osys, R0, moves, props, accepted)
    r_reg, j_reg = _regrouped(osys, R0, moves, props, accepted, spec.L, inputs["rcut"], j["same"])
    np.testing.assert_allclose(r_reg, r_dir, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(j_reg, j_dir, rtol=1e-10, atol=1e-12)
