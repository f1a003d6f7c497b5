"""One- and two-body Jastrow factor built from 1D cubic B-spline radial functors.

Sec. "Jastrow factor": J = sum_i u_1(r_i) + 1/2 sum_{i != j} u_2(r_i, r_j); the one-body
term sums an electron-ion functor u_{sigma I}(|r_i - R_I|) over ions and the two-body term
a spin-dependent functor u_{sigma sigma'}(|r_i - r_j|) with up-up = down-down. Each functor
is u(r) = sum_{m=0}^{M} p_m B3(r / (r_c / M) - m), where B3 is the cardinal cubic B-spline
supported on [-3, 1) (centred at -1), i.e. B3(x) = N(x + 3) with N the standard cubic
B-spline on [0, 4), and u = 0 for r >= r_c. Distances use the minimum-image convention
of the periodic cube.

Readings adopted where the paper is silent or inconsistent:
* the wavefunction is D_up D_dn e^{+J} (Eq. msdj);
* the cusp condition is p_0 = p_2 - (2 r_c / M) u'(0), which is what the stated basis
  gives (u'(0) = (p_2 - p_0) M / (2 r_c)); the printed factor 2M/r_c is inconsistent
  with the basis argument r / (r_c / M);
* p_M = 0, which makes u vanish with its first two derivatives at r_c.

Pins: partition of unity of the basis, the cusp derivative, smooth vanishing at r_c,
finite differences of u, and finite differences of J over particle coordinates.
"""
from __future__ import annotations

import numpy as np


def cubic_bspline_N(x):
    """Standard uniform cubic B-spline on [0, 4) and its first two derivatives."""
    x = np.asarray(x, dtype=np.float64)
    v = np.zeros_like(x)
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    m0 = (x >= 0) & (x < 1)
    m1 = (x >= 1) & (x < 2)
    m2 = (x >= 2) & (x < 3)
    m3 = (x >= 3) & (x < 4)
    a = x[m0]
    v[m0], d1[m0], d2[m0] = a ** 3 / 6, a ** 2 / 2, a
    a = x[m1]
    v[m1] = (-3 * a ** 3 + 12 * a ** 2 - 12 * a + 4) / 6
    d1[m1] = (-9 * a ** 2 + 24 * a - 12) / 6
    d2[m1] = (-18 * a + 24) / 6
    a = x[m2]
    v[m2] = (3 * a ** 3 - 24 * a ** 2 + 60 * a - 44) / 6
    d1[m2] = (9 * a ** 2 - 48 * a + 60) / 6
    d2[m2] = (18 * a - 48) / 6
    a = x[m3]
    v[m3], d1[m3], d2[m3] = (4 - a) ** 3 / 6, -(4 - a) ** 2 / 2, (4 - a)
    return v, d1, d2


def functor(r, p, rc):
    """u(r), u'(r), u''(r) of one radial functor with control points p_0..p_M."""
    r = np.asarray(r, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    M = p.shape[0] - 1
    scale = M / rc
    s = r * scale
    u = np.zeros_like(r)
    du = np.zeros_like(r)
    d2u = np.zeros_like(r)
    for m in range(M + 1):
        v, d1, d2 = cubic_bspline_N(s - m + 3.0)
        u += p[m] * v
        du += p[m] * d1 * scale
        d2u += p[m] * d2 * scale * scale
    inside = r < rc
    return np.where(inside, u, 0.0), np.where(inside, du, 0.0), np.where(inside, d2u, 0.0)


def cusp_p0(p, rc, cusp):
    """p_0 from the cusp condition u'(0) = cusp (adopted reading, see module docstring)."""
    M = len(p) - 1
    return p[2] - (2.0 * rc / M) * cusp


def min_image(d, L):
    return d - L * np.rint(d / L)


class Jastrow:
    """J(R) for electrons R (n_elec, 3) with the first n_up up-spin, ions (n_ion, 3)."""

    def __init__(self, L, n_up, ions, p_eI, p_same, p_opp, rc):
        self.L = float(L)
        self.n_up = int(n_up)
        self.ions = np.asarray(ions, dtype=np.float64).reshape(-1, 3)
        self.p_eI = np.asarray(p_eI, dtype=np.float64)
        self.p_same = np.asarray(p_same, dtype=np.float64)
        self.p_opp = np.asarray(p_opp, dtype=np.float64)
        self.rc = float(rc)
        self.active = self.p_same.size > 0 or self.p_eI.size > 0

    def _spin(self, n):
        return (np.arange(n) >= self.n_up).astype(np.int64)

    def value(self, R):
        """J(R) by a full sum over electron-ion pairs and electron pairs i < j."""
        if not self.active:
            return 0.0
        R = np.asarray(R, dtype=np.float64)
        n = R.shape[0]
        J = 0.0
        if self.p_eI.size and self.ions.shape[0]:
            d = min_image(R[:, None, :] - self.ions[None, :, :], self.L)
            J += functor(np.sqrt((d * d).sum(-1)), self.p_eI, self.rc)[0].sum()
        if self.p_same.size:
            iu, ju = np.triu_indices(n, 1)
            d = min_image(R[iu] - R[ju], self.L)
            r = np.sqrt((d * d).sum(-1))
            spin = self._spin(n)
            same = spin[iu] == spin[ju]
            J += functor(r[same], self.p_same, self.rc)[0].sum()
            J += functor(r[~same], self.p_opp, self.rc)[0].sum()
        return float(J)

    def grad_lap(self, R, i):
        """grad_i J (3,) and lap_i J for electron i: sums of u'(r) r_hat and
        u''(r) + 2 u'(r) / r over the pairs that contain electron i."""
        R = np.asarray(R, dtype=np.float64)
        g = np.zeros(3)
        lap = 0.0
        if not self.active:
            return g, lap
        n = R.shape[0]
        parts = []
        if self.p_eI.size and self.ions.shape[0]:
            parts.append((min_image(R[i] - self.ions, self.L), self.p_eI))
        if self.p_same.size:
            others = np.array([j for j in range(n) if j != i], dtype=np.int64)
            d = min_image(R[i] - R[others], self.L)
            spin = self._spin(n)
            same = spin[others] == spin[i]
            parts.append((d[same], self.p_same))
            parts.append((d[~same], self.p_opp))
        for d, p in parts:
            if d.shape[0] == 0:
                continue
            r = np.sqrt((d * d).sum(-1))
            _, du, d2u = functor(r, p, self.rc)
            g += ((du / r)[:, None] * d).sum(0)
            lap += (d2u + 2.0 * du / r).sum()
        return g, float(lap)
