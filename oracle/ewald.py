"""Coulomb energy of a periodic cell by Ewald summation.

Sec. "Hamiltonian": in periodic boundary conditions every pair potential sums over the
images of the cell, v(|r_1 - r_2|) -> sum_n v(|r_1 - r_2 + n L|), and for the bare Coulomb
interaction v_C = 1/r these sums are evaluated by the Ewald technique (split into a short-
and a long-ranged part). For point charges q_a at r_a in a cubic cell of side L (volume
Omega = L^3) with a uniform neutralising background when sum_a q_a != 0, and splitting
parameter alpha:

  E = 1/2 sum_a sum_{b != a} q_a q_b erfc(alpha r_ab) / r_ab            (real space)
    + (2 pi / Omega) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2 |rho_k|^2  (reciprocal space)
    - alpha / sqrt(pi) sum_a q_a^2                                       (self terms)
    - pi (sum_a q_a)^2 / (2 Omega alpha^2)                               (background),

rho_k = sum_a q_a e^{i k.r_a}, k = 2 pi n / L over integer vectors n != 0 with |k| <= k_cut.
Adopted reading: the real-space sum runs over the nearest image of each pair only (alpha
large enough that erfc(alpha L / 2) is negligible), and the reciprocal sum is truncated at
k_cut; the two truncations are parameters of the system. The paper's optimised breakup is
not used: plain Ewald is one of the two evaluations it names.

This is test infrastructure (part of the FP64 oracle), a direct restatement of the sums
above.

Pins: the Madelung energy of a single charge in a cubic cell with background (the simple
cubic Wigner-lattice constant -2.837297479480620 / (2 L)); the rock-salt Madelung constant
1.747564594633; independence of the total from alpha at converged truncations.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def kvectors(L: float, kcut: float) -> np.ndarray:
    """Half of the reciprocal vectors 2 pi n / L with 0 < |k| <= kcut (one of each +-k
    pair: the first nonzero component of n is positive)."""
    nmax = int(math.floor(kcut * L / (2 * math.pi)))
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    k = 2 * math.pi / L * n
    keep = ((k * k).sum(1) <= kcut * kcut) & (
        (n[:, 0] > 0) | ((n[:, 0] == 0) & (n[:, 1] > 0)) | ((n[:, 0] == 0) & (n[:, 1] == 0) & (n[:, 2] > 0)))
    return k[keep]


def ewald_energy(pos, q, L: float, alpha: float, kcut: float) -> float:
    """Total Coulomb energy of charges q (n,) at pos (n, 3) in the periodic cube of side L."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    n = pos.shape[0]
    omega = L ** 3
    e_real = 0.0
    for a in range(n):
        d = pos[a + 1:] - pos[a]
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(1))
        e_real += float((q[a] * q[a + 1:] * erfc(alpha * r) / r).sum())
    k = kvectors(L, kcut)
    k2 = (k * k).sum(1)
    phase = pos @ k.T                                  # (n, K)
    rho_re = (q[:, None] * np.cos(phase)).sum(0)
    rho_im = (q[:, None] * np.sin(phase)).sum(0)
    # the half set of k covers each +-k pair once: factor 2
    e_recip = 2.0 * (2 * math.pi / omega) * float((np.exp(-k2 / (4 * alpha ** 2)) / k2
                                                 * (rho_re ** 2 + rho_im ** 2)).sum())
    e_self = -alpha / math.sqrt(math.pi) * float((q * q).sum())
    e_bg = -math.pi * float(q.sum()) ** 2 / (2 * omega * alpha ** 2)
    return e_real + e_recip + e_self + e_bg


def coulomb_potential(R, ions, Z: float, L: float, alpha: float, kcut: float) -> float:
    """Electrons (charge -1) at R and ions (charge +Z): the Coulomb energy of the
    configuration, including the ion-ion part."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    ions = np.asarray(ions, dtype=np.float64).reshape(-1, 3)
    pos = np.vstack([R, ions])
    q = np.concatenate([-np.ones(R.shape[0]), Z * np.ones(ions.shape[0])])
    return ewald_energy(pos, q, L, alpha, kcut)
