"""Pins of the oracle's Ewald summation (CPU; Sec. "Hamiltonian": periodic Coulomb sums by
the Ewald technique)."""
import math

import numpy as np
import pytest

from oracle.ewald import coulomb_potential, ewald_energy, kvectors

# Madelung constants (textbook lattice sums, not from any benchmark suite)
WIGNER_SC = -2.837297479480620    # one charge per cubic cell with a uniform background: E = xi / (2 L)
ROCK_SALT = 1.747564594633182     # E per ion pair = -M / (nearest-neighbour distance)


def _converged(L, r_frac=0.5):
    """alpha making the real-space terms beyond the nearest image negligible, and the k
    cutoff making the reciprocal terms beyond it negligible."""
    alpha = 6.0 / (r_frac * L)
    return alpha, 2 * alpha * math.sqrt(math.log(1e17))


def test_single_charge_with_background():
    for L in (1.0, 7.3):
        alpha, kcut = _converged(L, r_frac=1.0)
        e = ewald_energy([[0.3, 0.1, 0.2]], [1.0], L, alpha, kcut)
        assert e == pytest.approx(WIGNER_SC / (2 * L), rel=1e-12)


def test_rock_salt_madelung_constant():
    L = 5.64
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    pos = np.vstack([fcc, fcc + [0.5, 0, 0]]) * L + 0.37
    q = np.array([1.0] * 4 + [-1.0] * 4)
    alpha, kcut = _converged(L)
    e = ewald_energy(pos, q, L, alpha, kcut)
    assert e == pytest.approx(-4 * ROCK_SALT / (L / 2), rel=1e-11)


def test_total_is_independent_of_the_split():
    rng = np.random.default_rng(4)
    L = 6.0
    pos = rng.uniform(0, L, size=(7, 3))
    q = np.array([1, -1, 2, -2, 1, -1, 0.5])          # charged cell: background term active
    vals = []
    for a in (2.0, 2.6, 3.2):              # alpha L / 2 >= 6: nearest image suffices
        kc = 2 * a * math.sqrt(math.log(1e17))
        vals.append(ewald_energy(pos, q, L, a, kc))
    assert np.ptp(vals) < 1e-10 * max(1.0, abs(vals[0]))


def test_kvectors_half_set():
    k = kvectors(4.0, 2 * math.pi / 4.0 * 1.5)
    # |n| <= 1.5: the 18 nonzero vectors of the 3^3 cube minus the 8 corners, halved
    assert k.shape[0] == 9
    assert not np.any(np.all(np.isclose(k[:, None, :], -k[None, :, :]), -1))


def test_coulomb_potential_charges():
    """Electrons carry charge -1 and ions +Z: the potential equals the Ewald energy of the
    explicit list of point charges."""
    L = 5.0
    alpha, kcut = _converged(L)
    R = np.array([[1.0, 2.0, 3.0], [2.5, 0.5, 1.5]])
    ions = np.array([[4.0, 4.0, 1.0]])
    e = coulomb_potential(R, ions, 2.0, L, alpha, kcut)
    ref = ewald_energy(np.vstack([R, ions]), [-1.0, -1.0, 2.0], L, alpha, kcut)
    assert e == ref
