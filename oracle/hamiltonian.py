"""Potential energy: a short-range screened (Yukawa) stand-in for the Coulomb terms.

Sec. "Hamiltonian": H = -1/2 sum_i lap_i + sum_{i<j} v_ee + sum_{i,I} v_eI + sum_{I<J} v_II
with v_ee = v, v_eI = -Z v and v_II = Z^2 v. The periodic Coulomb sums need Ewald
(Sec. "Ewald" / optimised breakup), which is outside the hot path; the workloads here use
v(r) = exp(-kappa r) / r with minimum-image distances, truncated at r >= L/2
(adopted reading: Z = 4, kappa = 1 / bohr, no shift at the truncation).

Pins: two-particle values, the direct double sum, and invariance under relabelling.
"""
from __future__ import annotations

import numpy as np


def _min_image(d, L):
    return d - L * np.rint(d / L)


def yukawa(r, kappa, L):
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 0.5 * L, np.exp(-kappa * r) / r, 0.0)


def yukawa_potential(R, ions, Z, kappa, L):
    """sum_{i<j} v(r_ij) - Z sum_{i,I} v(r_iI) + Z^2 sum_{I<J} v(R_IJ)."""
    R = np.asarray(R, dtype=np.float64)
    ions = np.asarray(ions, dtype=np.float64).reshape(-1, 3)
    V = 0.0
    n = R.shape[0]
    if n > 1:
        i, j = np.triu_indices(n, 1)
        d = _min_image(R[i] - R[j], L)
        V += yukawa(np.sqrt((d * d).sum(-1)), kappa, L).sum()
    if ions.shape[0]:
        d = _min_image(R[:, None, :] - ions[None, :, :], L)
        V -= Z * yukawa(np.sqrt((d * d).sum(-1)), kappa, L).sum()
        if ions.shape[0] > 1:
            i, j = np.triu_indices(ions.shape[0], 1)
            d = _min_image(ions[i] - ions[j], L)
            V += Z * Z * yukawa(np.sqrt((d * d).sum(-1)), kappa, L).sum()
    return float(V)
