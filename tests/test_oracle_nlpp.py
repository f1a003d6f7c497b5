"""Pins of the oracle's non-local pseudopotential quadrature (CPU; Sec. "Hamiltonian",
semi-local pseudopotentials with a 12-point angular integration)."""
import math

import numpy as np
import pytest
from scipy.special import spherical_jn

from oracle.nlpp import NonLocalPP, icosahedron, legendre, nonlocal_energy, rotation
from oracle.orbitals import PlaneWaveOrbitals
from oracle.wavefunction import SlaterJastrow


def test_icosahedron_rule_is_exact_to_degree_five():
    """(1/12) sum_q P_l(u . O n_q) = delta_l0 for l <= 5, any unit u and rotation O; the rule
    is not exact at l = 6 (a 12-point rule cannot be)."""
    pts = icosahedron()
    assert pts.shape == (12, 3)
    assert np.allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-15)
    rng = np.random.default_rng(3)
    worst6 = 0.0
    for trial in range(20):
        O = rotation(trial, 5, 7)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        c = (pts @ O.T) @ u
        for l in range(6):
            assert abs(legendre(l, c).mean() - (1.0 if l == 0 else 0.0)) < 1e-14, (l, trial)
        worst6 = max(worst6, abs(legendre(6, c).mean()))
    assert worst6 > 1e-3


def test_legendre_closed_forms():
    x = np.linspace(-1, 1, 7)
    assert np.allclose(legendre(2, x), 0.5 * (3 * x ** 2 - 1), atol=1e-15)
    assert np.allclose(legendre(3, x), 0.5 * (5 * x ** 3 - 3 * x), atol=1e-15)


def test_rotations_are_proper_and_vary():
    Rs = [rotation(0, t, w) for t in range(5) for w in range(5)]
    for R in Rs:
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
    assert np.std([R[0, 0] for R in Rs]) > 0.1
    # a uniform random rotation: the mean of each matrix element vanishes
    many = np.array([rotation(1, t, 3) for t in range(4000)])
    assert np.abs(many.mean(0)).max() < 0.05


def _one_electron(orbitals, ions, L=8.0):
    return SlaterJastrow(orbitals, 1, 0, None, ions, 4.0, 1.0, L, False)


PP = NonLocalPP(amp=np.array([1.5, -1.0]), width=np.array([0.8, 0.7]), rcut=1.6)


def test_constant_orbital_leaves_the_s_channel():
    """A constant orbital makes every ratio 1: only l = 0 survives the exact rule."""
    L = 8.0
    orb = PlaneWaveOrbitals(np.zeros((1, 1, 3), int), np.zeros((1, 1), int), np.ones((1, 1)), L)
    ions = np.array([[1.0, 1.0, 1.0], [5.0, 5.0, 5.0]])
    wf = _one_electron(orb, ions, L)
    R = np.array([[1.7, 1.2, 0.6]])
    r = np.linalg.norm(R[0] - ions[0])
    e = nonlocal_energy(wf, PP, R, seed=0, t=1, walker_id=0)
    assert e == pytest.approx(1.5 * math.exp(-(r / 0.8) ** 2), rel=1e-13)


@pytest.mark.parametrize("t,offset", [(1, (0.55, 0.3, 0.2)), (2, (0.55, 0.3, 0.2)),
                                      (3, (0.12, -0.1, 0.05))])
def test_plane_wave_matches_the_angular_integral(t, offset):
    """One electron in phi = cos(k . r): the l-channel angular integral is
    Re[e^{i k.R_I} i^l j_l(k r) P_l(u . k^)] / cos(k . r_i) in closed form. Expanding the
    plane wave in Legendre polynomials, the 12-point rule is exact for the terms l' with
    l + l' <= 5 and errs by at most 2 on each product P_l P_l' beyond, so the quadrature
    differs from the closed form by at most
    sum_l (2l+1) |dv_l| sum_{l' >= 6-l} (2l'+1) |j_l'(k r)| / |cos(k . r_i)|."""
    L = 8.0
    n = np.array([[[1, 0, 0]]])
    orb = PlaneWaveOrbitals(n, np.zeros((1, 1), int), np.ones((1, 1)), L)
    k = 2 * np.pi / L * np.array([1.0, 0.0, 0.0])
    ions = np.array([[3.0, 2.0, 4.0]])
    wf = _one_electron(orb, ions, L)
    R = ions + np.array([offset])
    d = R[0] - ions[0]
    r = np.linalg.norm(d)
    u = d / r
    kn = np.linalg.norm(k)
    ref = 0.0
    for l in range(2):
        ang = (np.exp(1j * (k @ ions[0])) * (1j ** l) * spherical_jn(l, kn * r)
               * legendre(l, u @ (k / kn))).real / math.cos(k @ R[0])
        ref += (2 * l + 1) * PP.dv(l, r) * ang
    got = nonlocal_energy(wf, PP, R, seed=0, t=t, walker_id=0)
    bound = sum((2 * l + 1) * abs(PP.dv(l, r)) * sum(2 * (2 * lp + 1) * abs(spherical_jn(lp, kn * r))
                                                      for lp in range(6 - l, 30))
                for l in range(2)) / abs(math.cos(k @ R[0]))
    assert abs(got - ref) <= bound, (got, ref, bound)
    assert bound < 1e-3 * abs(ref)                  # the bound itself is tight enough to pin


def test_energy_outside_the_cutoff_is_zero():
    L = 8.0
    orb = PlaneWaveOrbitals(np.array([[[1, 0, 0]]]), np.zeros((1, 1), int), np.ones((1, 1)), L)
    wf = _one_electron(orb, np.array([[1.0, 1.0, 1.0]]), L)
    assert nonlocal_energy(wf, PP, np.array([[3.0, 1.0, 1.0]]), 0, 1, 0) == 0.0
