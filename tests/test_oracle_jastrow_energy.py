"""Pins of the oracle's Jastrow functors, Slater determinants, log-derivatives, local
energy and Yukawa potential (CPU)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle.hamiltonian import yukawa_potential
from oracle.jastrow import Jastrow, cubic_bspline_N, cusp_p0, functor
from oracle.vmc import OracleSystem
from synthetic import build_inputs, small_spec, spec_for

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ------------------------------------------------------------------ 1D functor
def test_B3_values_at_integers_and_unit_integral():
    for x, v in GOLD["jastrow_B3_at_integers"]["value"].items():
        assert abs(cubic_bspline_N(float(x) + 3.0)[0] - v) < 1e-15
    x = np.linspace(0, 4, 400001)
    v = cubic_bspline_N(x)[0]
    assert abs(np.trapezoid(v, x) - 1.0) < 1e-9
    assert np.allclose(v, v[::-1], atol=1e-12)          # symmetric about 2


@pytest.mark.parametrize("M", [8, 10])
def test_partition_of_unity(M):
    rc = 5.0
    r = np.linspace(0, rc * (M - 2) / M - 1e-9, 500)
    u, du, d2u = functor(r, np.ones(M + 1), rc)
    assert np.allclose(u, 1.0, atol=1e-14)
    assert np.allclose(du, 0.0, atol=1e-12)
    assert np.allclose(d2u, 0.0, atol=1e-10)


def test_cusp_condition_and_smooth_cutoff():
    rng = np.random.default_rng(0)
    M, rc = 8, 7.5
    for cusp in (0.0, 0.5, -0.25, -4.0):
        p = rng.uniform(-0.5, 0, M + 1)
        p[M] = 0.0
        p[0] = cusp_p0(p, rc, cusp)
        h = 1e-6
        fd = (functor(np.array([h]), p, rc)[0][0] - functor(np.array([0.0]), p, rc)[0][0]) / h
        assert abs(fd - cusp) < 1e-5
        assert abs(functor(np.array([0.0]), p, rc)[1][0] - cusp) < 1e-12
        rm = np.array([rc - 1e-7])
        u, du, d2u = functor(rm, p, rc)
        assert abs(u[0]) < 1e-12 and abs(du[0]) < 1e-8 and abs(d2u[0]) < 1e-5
        u, du, d2u = functor(np.array([rc, rc + 1.0]), p, rc)
        assert np.all(u == 0) and np.all(du == 0) and np.all(d2u == 0)


def test_functor_derivatives_finite_differences():
    rng = np.random.default_rng(1)
    M, rc = 10, 6.0
    p = rng.uniform(-0.5, 0, M + 1)
    p[M] = 0
    r = rng.uniform(0.01, rc - 0.01, 200)
    h = 1e-5
    u, du, d2u = functor(r, p, rc)
    up, dup, _ = functor(r + h, p, rc)
    um, dum, _ = functor(r - h, p, rc)
    assert np.allclose((up - um) / (2 * h), du, atol=1e-8)
    assert np.allclose((dup - dum) / (2 * h), d2u, atol=1e-6)


def test_two_body_pairs_and_minimum_image():
    M, rc, L = 8, 5.0, 10.0
    rng = np.random.default_rng(2)
    p_same, p_opp, p_eI = (rng.uniform(-0.5, 0, M + 1) for _ in range(3))
    for p in (p_same, p_opp, p_eI):
        p[M] = 0
    ions = np.array([[9.9, 0.2, 5.0]])
    jas = Jastrow(L, 1, ions, p_eI, p_same, p_opp, rc)
    R = np.array([[0.1, 0.3, 5.0], [9.8, 0.3, 5.0]])    # one up, one down, 0.3 apart
    expect = functor(np.array([0.3]), p_opp, rc)[0][0]
    expect += functor(np.array([0.2 * np.sqrt(1.25)]), p_eI, rc)[0][0]   # (0.2, 0.1, 0)
    expect += functor(np.array([np.hypot(0.1, 0.1)]), p_eI, rc)[0][0]
    assert abs(jas.value(R) - expect) < 1e-13
    jas2 = Jastrow(L, 2, ions, p_eI, p_same, p_opp, rc)       # both up: same-spin functor
    expect2 = expect - functor(np.array([0.3]), p_opp, rc)[0][0] + functor(np.array([0.3]), p_same, rc)[0][0]
    assert abs(jas2.value(R) - expect2) < 1e-13
    # relabelling electrons of the same spin leaves J unchanged
    d = build_inputs(small_spec(6, 5, grid=8), n_walkers=1)
    s = OracleSystem(d)
    R = d["pos"][0]
    perm = np.r_[np.random.default_rng(3).permutation(6), 6 + np.random.default_rng(4).permutation(5)]
    assert abs(s.wf.jas.value(R) - s.wf.jas.value(R[perm])) < 1e-12


def test_jastrow_gradient_laplacian_finite_differences():
    d = build_inputs(small_spec(6, 5, grid=8), n_walkers=1)
    s = OracleSystem(d)
    jas = s.wf.jas
    R = d["pos"][0].copy()
    h = 1e-4
    for i in (0, 5, 7, 10):
        g, lap = jas.grad_lap(R, i)
        fd_lap = 0.0
        for ax in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, ax] += h
            Rm[i, ax] -= h
            jp, jm, j0 = jas.value(Rp), jas.value(Rm), jas.value(R)
            assert abs((jp - jm) / (2 * h) - g[ax]) < 1e-7
            fd_lap += (jp - 2 * j0 + jm) / h ** 2
        assert abs(fd_lap - lap) < 1e-4


# ---------------------------------------------------------------- determinants
def _leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        sgn = 1
        p = list(perm)
        for a in range(n):            # parity by counting inversions
            for b in range(a + 1, n):
                if p[a] > p[b]:
                    sgn = -sgn
        tot += sgn * np.prod([A[k, perm[k]] for k in range(n)])
    return tot


def test_ratio_matches_permutation_expansion_and_sherman_morrison():
    d = build_inputs(small_spec(4, 3, grid=8, jastrow_M=0), n_walkers=1)
    s = OracleSystem(d)
    w = s.walker(d["pos"][0], 0)
    rng = np.random.default_rng(5)
    for e in range(7):
        spin, first, ns = s.wf.block(e)
        r_new = rng.uniform(0, s.L, 3)
        A = w.A[spin]
        A2 = A.copy()
        A2[e - first] = s.wf.orb.values(r_new)[:ns]
        ratio_brute = _leibniz_det(A2) / _leibniz_det(A)
        sg, ld = np.linalg.slogdet(A2)
        ratio = sg * w.sign[spin] * np.exp(ld - w.logdet[spin])
        assert abs(ratio - ratio_brute) < 1e-10 * max(1, abs(ratio_brute))
        # the identity used by the GPU: ratio = phi(r') . column e of inv(A)
        sm = A2[e - first] @ np.linalg.inv(A)[:, e - first]
        assert abs(ratio - sm) < 1e-10 * max(1, abs(ratio))


def test_log_psi_derivatives_match_finite_differences():
    d = build_inputs(small_spec(5, 4, grid=10), n_walkers=1)
    s = OracleSystem(d)
    R = d["pos"][0].copy()
    h = 1e-4
    for i in (0, 4, 5, 8):
        g = s.wf.grad_log_psi(R, i)
        gd, lapd = s.wf.grad_lap_log_det(R, i)
        _, lapj = s.wf.jas.grad_lap(R, i)
        lap = lapd + lapj
        f0 = s.wf.log_psi(R)[0]
        fd_lap = 0.0
        for ax in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, ax] += h
            Rm[i, ax] -= h
            fp, fm = s.wf.log_psi(Rp)[0], s.wf.log_psi(Rm)[0]
            assert abs((fp - fm) / (2 * h) - g[ax]) < 1e-6 * max(1, abs(g[ax]))
            fd_lap += (fp - 2 * f0 + fm) / h ** 2
        assert abs(fd_lap - lap) < 2e-3 * max(1, abs(lap))


def test_zero_variance_plane_wave_determinant():
    d = build_inputs(spec_for("pw14"), n_walkers=6)
    s = OracleSystem(d, orbitals="planewave")
    e_ref = GOLD["pw14_kinetic_energy"]["value"]
    for R in d["pos"]:
        e, kin = s.wf.local_energy(R)
        assert abs(kin - e_ref) < 1e-10
        assert e == kin          # no potential in this workload
    # with the B-spline orbitals the identity holds up to the spline error O((k D)^2)
    sp = OracleSystem(d)
    kd = (2 * np.pi / 10.0) * (10.0 / 32)
    for R in d["pos"]:
        _, kin = sp.wf.local_energy(R)
        assert abs(kin - e_ref) / e_ref < kd ** 2


# ------------------------------------------------------------------- potential
def test_yukawa_two_body_values_and_truncation():
    L, kap, Z = 10.0, 1.0, 4.0
    y = lambda r: np.exp(-kap * r) / r
    R = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 3.5]])
    assert abs(yukawa_potential(R, np.zeros((0, 3)), Z, kap, L) - y(2.5)) < 1e-15
    R = np.array([[0.5, 1.0, 1.0], [9.0, 1.0, 1.0]])             # min image 1.5
    assert abs(yukawa_potential(R, np.zeros((0, 3)), Z, kap, L) - y(1.5)) < 1e-15
    R = np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0]])              # r = L/2 -> truncated
    assert yukawa_potential(R, np.zeros((0, 3)), Z, kap, L) == 0.0
    ions = np.array([[1.0, 2.0, 1.0], [1.0, 2.0, 4.0]])
    R = np.array([[1.0, 1.0, 1.0]])
    expect = -Z * (y(1.0) + y(np.sqrt(1 + 9))) + Z * Z * y(3.0)
    assert abs(yukawa_potential(R, ions, Z, kap, L) - expect) < 1e-14


def test_potential_direct_double_sum():
    d = build_inputs(small_spec(5, 5, grid=8), n_walkers=1)
    R, ions, L = d["pos"][0], d["ions"], d["spec"].L
    tot = 0.0
    parts = [(R, R, 1.0, True), (R, ions, -4.0, False), (ions, ions, 16.0, True)]
    for A, B, q, same in parts:
        for a in range(len(A)):
            for b in range(len(B)):
                if same and b <= a:
                    continue
                dd = A[a] - B[b]
                dd -= L * np.round(dd / L)
                r = np.linalg.norm(dd)
                if r < L / 2:
                    tot += q * np.exp(-r) / r
    assert abs(yukawa_potential(R, ions, 4.0, 1.0, L) - tot) < 1e-12
