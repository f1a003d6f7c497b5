"""Single-particle orbitals: periodic tricubic B-splines and analytic plane waves.

Sec. "B-spline basis sets": each orbital is stored as a regular 3D B-spline, and one
evaluation touches the 4 x 4 x 4 = 64 coefficients around the point, whatever the size
of the underlying plane-wave basis. Here the grid is uniform with spacing D = L / n and
periodic; along each axis s = x / D, i = floor(s), t = s - i, and the four coefficients
i-1, i, i+1, i+2 (mod n) are weighted by the uniform cubic B-spline basis
    b0 = (1-t)^3/6, b1 = (3t^3 - 6t^2 + 4)/6, b2 = (-3t^3 + 3t^2 + 3t + 1)/6, b3 = t^3/6,
whose first and second derivatives (divided by D and D^2) give the gradient and the
Laplacian (the sum of the three second derivatives).

Sec. "Specialised bases" (homogeneous electron gas plane waves): the analytic plane-wave
evaluation below is used only by the tests (zero-variance check), never by a sweep that
is compared with the CUDA path.

Pins: cubic polynomial reproduction with exact derivatives away from the periodic
wrap; exact interpolation of the closed-form coefficient fit at every grid node; value,
gradient and Laplacian against the analytic plane-wave orbitals within the spline's
O((k D)^2) error; central finite differences of value and gradient.
"""
from __future__ import annotations

import numpy as np


def bspline_basis(t):
    """Weights of the four nodes i-1..i+2 and their first and second derivatives with
    respect to t (arrays of shape (4, ...))."""
    t = np.asarray(t, dtype=np.float64)
    t2, t3 = t * t, t * t * t
    b = np.stack([(1 - t) ** 3 / 6, (3 * t3 - 6 * t2 + 4) / 6,
                  (-3 * t3 + 3 * t2 + 3 * t + 1) / 6, t3 / 6])
    db = np.stack([-(1 - t) ** 2 / 2, (3 * t2 - 4 * t) / 2,
                   (-3 * t2 + 2 * t + 1) / 2, t2 / 2])
    d2b = np.stack([1 - t, 3 * t - 2, 1 - 3 * t, t])
    return b, db, d2b


class SplineOrbitals:
    """Tricubic B-spline orbitals from coefficients ``coef[nx][ny][nz][n_orb]`` on the
    periodic cube [0, L)^3."""

    def __init__(self, coef: np.ndarray, L: float):
        self.coef = np.asarray(coef, dtype=np.float64)
        self.L = float(L)
        self.n = np.array(self.coef.shape[:3])
        self.n_orb = self.coef.shape[3]

    def vgl(self, r):
        """Value (n_orb,), gradient (3, n_orb) and Laplacian (n_orb,) at one point."""
        r = np.mod(np.asarray(r, dtype=np.float64), self.L)
        delta = self.L / self.n
        s = r / delta
        i = np.floor(s).astype(np.int64)
        t = s - i
        w = [bspline_basis(t[d]) for d in range(3)]        # per axis: (b, db, d2b)
        idx = [np.mod(i[d] - 1 + np.arange(4), self.n[d]) for d in range(3)]
        c = self.coef[np.ix_(idx[0], idx[1], idx[2])]      # (4, 4, 4, n_orb)
        bx, dbx, d2bx = w[0]
        by, dby, d2by = w[1]
        bz, dbz, d2bz = w[2]
        e = lambda wx, wy, wz: np.einsum("a,b,c,abco->o", wx, wy, wz, c)
        val = e(bx, by, bz)
        grad = np.stack([e(dbx, by, bz) / delta[0], e(bx, dby, bz) / delta[1],
                         e(bx, by, dbz) / delta[2]])
        lap = (e(d2bx, by, bz) / delta[0] ** 2 + e(bx, d2by, bz) / delta[1] ** 2
               + e(bx, by, d2bz) / delta[2] ** 2)
        return val, grad, lap

    def values(self, r):
        return self.vgl(r)[0]


class PlaneWaveOrbitals:
    """Analytic orbitals sum_t a_t cos(k_t . r) or a_t sin(k_t . r), k_t = 2 pi n_t / L."""

    def __init__(self, nvec, kind, amp, L: float):
        self.k = 2.0 * np.pi * np.asarray(nvec, dtype=np.float64) / L    # (n_orb, T, 3)
        self.kind = np.asarray(kind)
        self.amp = np.asarray(amp, dtype=np.float64)
        self.L = float(L)
        self.n_orb = self.k.shape[0]

    def vgl(self, r):
        r = np.asarray(r, dtype=np.float64)
        ph = self.k @ r                                      # (n_orb, T)
        c, s = np.cos(ph), np.sin(ph)
        is_sin = self.kind == 1
        f = np.where(is_sin, s, c)                          # the function
        df = np.where(is_sin, c, -s)                        # d f / d(phase)
        val = (self.amp * f).sum(1)
        grad = np.einsum("ot,otd->do", self.amp * df, self.k)
        k2 = (self.k ** 2).sum(-1)
        lap = -(self.amp * k2 * f).sum(1)
        return val, grad, lap

    def values(self, r):
        return self.vgl(r)[0]
