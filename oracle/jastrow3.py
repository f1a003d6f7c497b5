"""Three-body electron-electron-ion Jastrow factor.

Sec. "Jastrow factor": the three-body correlation function (the form of Drummond, Towler
and Needs) is a polynomial in the two electron-ion distances a = r_iI, b = r_jI and the
electron-electron distance c = r_ij, cut off smoothly at half the cutoff radius h = r_c / 2
in both electron-ion distances:

    u(a, b, c) = sum_{l,m=0}^{M_eI} sum_{n=0}^{M_ee} gamma_lmn a^l b^m c^n
                 (a - h)^3 Theta(h - a) (b - h)^3 Theta(h - b),

    J3(R) = sum_I sum_{i<j} u_{s(i)s(j)}(r_iI, r_jI, r_ij),

with one coefficient set for same-spin and one for opposite-spin electron pairs and one ion
species. Readings adopted where the paper is unclear:
* the step functions are Theta(h - r): the printed Theta(r - h) contradicts the stated
  behaviour (the correlation vanishes once either electron-ion distance exceeds r_c / 2);
* gamma_lmn = gamma_mln (symmetric under exchange of the two electrons), the constraint
  that makes u independent of the order of the pair; non-symmetric sets are rejected;
* no further constraints on gamma (cusp conditions) are imposed: the coefficients are
  inputs;
* distances are minimum-image distances in the periodic cube, with r_c <= L / 2;
* Psi = D_up D_dn e^{+J} with J = J1 + J2 + J3.

For electron i the derivatives follow from u(a, b, c) with a-hat = (r_i - R_I) / a and
c-hat = (r_i - r_j) / c:
    grad_i u = u_a a-hat + u_c c-hat,
    lap_i u  = u_aa + 2 u_a / a + u_cc + 2 u_c / c + 2 u_ac (a-hat . c-hat).

This is test infrastructure (part of the FP64 oracle), a direct evaluation of the sums
above. Pins: closed-form single-term values, vanishing beyond h with continuous first and
second derivatives, finite differences of J3 over the electron coordinates, exchange and
translation invariance, and the spin-pair assignment.
"""
from __future__ import annotations

import numpy as np


def _min_image(d, L):
    return d - L * np.rint(d / L)


def _powers(x, n):
    """x^0 .. x^n along a new last axis."""
    x = np.asarray(x, dtype=np.float64)
    return x[..., None] ** np.arange(n + 1)


def u3_derivs(a, b, c, gamma, h):
    """u and its partial derivatives (u, u_a, u_c, u_aa, u_cc, u_ac) at arrays a, b, c
    (the first electron's distances a = r_iI and c = r_ij; b = r_jI held fixed)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    meI, mee = gamma.shape[0] - 1, gamma.shape[2] - 1
    a, b, c = (np.asarray(x, dtype=np.float64) for x in (a, b, c))
    inside = (a < h) & (b < h)
    pa, pb, pc = _powers(a, meI), _powers(b, meI), _powers(c, mee)
    la = np.arange(meI + 1, dtype=np.float64)
    ln = np.arange(mee + 1, dtype=np.float64)
    # derivative factors of the powers: d/dx x^l = l x^(l-1), d2/dx2 x^l = l (l-1) x^(l-2)
    dpa = np.concatenate([np.zeros_like(pa[..., :1]), pa[..., :-1] * la[1:]], -1)
    d2pa = np.concatenate([np.zeros_like(pa[..., :2]), pa[..., :-2] * (la[2:] * (la[2:] - 1))], -1)[..., : meI + 1]
    dpc = np.concatenate([np.zeros_like(pc[..., :1]), pc[..., :-1] * ln[1:]], -1)
    d2pc = np.concatenate([np.zeros_like(pc[..., :2]), pc[..., :-2] * (ln[2:] * (ln[2:] - 1))], -1)[..., : mee + 1]

    def poly(xa, xc):
        return np.einsum("...l,...m,...n,lmn->...", xa, pb, xc, gamma)

    P, Pa, Pc = poly(pa, pc), poly(dpa, pc), poly(pa, dpc)
    Paa, Pcc, Pac = poly(d2pa, pc), poly(pa, d2pc), poly(dpa, dpc)
    F, dF, d2F = (a - h) ** 3, 3.0 * (a - h) ** 2, 6.0 * (a - h)
    G = np.where(inside, (b - h) ** 3, 0.0)
    F = np.where(inside, F, 0.0)
    dF = np.where(inside, dF, 0.0)
    d2F = np.where(inside, d2F, 0.0)
    u = P * F * G
    ua = (Pa * F + P * dF) * G
    uc = Pc * F * G
    uaa = (Paa * F + 2.0 * Pa * dF + P * d2F) * G
    ucc = Pcc * F * G
    uac = (Pac * F + Pc * dF) * G
    return u, ua, uc, uaa, ucc, uac


class ThreeBodyJastrow:
    """J3(R) for electrons R (n_elec, 3) with the first n_up up-spin, ions (n_ion, 3)."""

    def __init__(self, L, n_up, ions, gamma_same, gamma_opp, rc):
        self.L = float(L)
        self.n_up = int(n_up)
        self.ions = np.asarray(ions, dtype=np.float64).reshape(-1, 3)
        self.g = [np.asarray(gamma_same, dtype=np.float64), np.asarray(gamma_opp, dtype=np.float64)]
        for g in self.g:
            if g.ndim != 3 or g.shape[0] != g.shape[1]:
                raise ValueError("gamma must have shape (M_eI + 1, M_eI + 1, M_ee + 1)")
            if not np.array_equal(g, g.transpose(1, 0, 2)):
                raise ValueError("gamma_lmn must equal gamma_mln")
        if self.g[0].shape != self.g[1].shape:
            raise ValueError("both coefficient sets must have the same orders")
        self.rc = float(rc)
        if not (0.0 < self.rc <= 0.5 * self.L):
            raise ValueError("r_c must lie in (0, L/2]")
        self.h = 0.5 * self.rc

    def _set(self, i, j):
        return self.g[0] if (i < self.n_up) == (j < self.n_up) else self.g[1]

    def value(self, R):
        R = np.asarray(R, dtype=np.float64)
        J = 0.0
        for I in range(self.ions.shape[0]):
            dI = _min_image(R - self.ions[I], self.L)
            rI = np.sqrt((dI * dI).sum(-1))
            inside = np.flatnonzero(rI < self.h)       # only these electrons have u != 0
            for x, i in enumerate(inside):
                for j in inside[x + 1:]:
                    d = _min_image(R[i] - R[j], self.L)
                    c = np.sqrt(d @ d)
                    J += float(u3_derivs(rI[i], rI[j], c, self._set(i, j), self.h)[0])
        return J

    def grad_lap(self, R, i):
        """grad_i J3 (3,) and lap_i J3 for electron i."""
        R = np.asarray(R, dtype=np.float64)
        g = np.zeros(3)
        lap = 0.0
        for I in range(self.ions.shape[0]):
            da = _min_image(R[i] - self.ions[I], self.L)
            a = np.sqrt(da @ da)
            if a >= self.h:
                continue
            dI = _min_image(R - self.ions[I], self.L)
            rI = np.sqrt((dI * dI).sum(-1))
            for j in np.flatnonzero(rI < self.h):     # only these electrons have u != 0
                if j == i:
                    continue
                b = rI[j]
                dc = _min_image(R[i] - R[j], self.L)
                c = np.sqrt(dc @ dc)
                u, ua, uc, uaa, ucc, uac = (float(x) for x in
                                            u3_derivs(a, b, c, self._set(i, j), self.h))
                ah, ch = da / a, dc / c
                g += ua * ah + uc * ch
                lap += uaa + 2.0 * ua / a + ucc + 2.0 * uc / c + 2.0 * uac * float(ah @ ch)
        return g, float(lap)


class JastrowSum:
    """J = sum of Jastrow terms, each with value(R) and grad_lap(R, i)."""

    def __init__(self, *terms):
        self.terms = [t for t in terms if t is not None]

    def value(self, R):
        return float(sum(t.value(R) for t in self.terms))

    def grad_lap(self, R, i):
        g, lap = np.zeros(3), 0.0
        for t in self.terms:
            gt, lt = t.grad_lap(R, i)
            g = g + gt
            lap += lt
        return g, float(lap)
