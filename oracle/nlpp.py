"""Non-local (semi-local) pseudopotential energy by angular quadrature.

Sec. "Hamiltonian": with semi-local pseudopotentials the electron-ion interaction carries,
besides its local part, channel projectors sum_{l m} |Y_lm> [v_l(r) - v_loc(r)] <Y_lm| that
vanish beyond a cutoff radius; their contribution to the local energy is evaluated
following Mitas, Shirley and Ceperley (J. Chem. Phys. 95, 3467 (1991)) with a 12-point
angular integration. For electron i at distance r = |r_i - R_I| < r_c from ion I (nearest
image), by the addition theorem of the spherical harmonics

    V_NL(i, I) = sum_l (2 l + 1) dv_l(r) (1/4pi) int dW' P_l(u . u') Psi(.., R_I + r u', ..) / Psi(R)

(u the unit vector from R_I to r_i, P_l the Legendre polynomials), and the angular integral
is replaced by a quadrature on the sphere of radius r around R_I:

    (1/4pi) int dW' f(u') ~ (1/12) sum_q f(O n_q),

n_q the 12 vertices of an icosahedron (exact for spherical harmonics of degree <= 5) and O a
random rotation drawn anew for each walker and measurement (the orientation's error then
averages out instead of biasing the run). Psi(..)/Psi(R) is the full Slater-Jastrow ratio of
moving electron i alone: a determinant ratio and exp(dJ).

Adopted readings (the paper states none of them; real pseudopotentials are not in the
container):
* channels l = 0..l_max with dv_l(r) = a_l exp(-(r / b_l)^2) for r < r_c, 0 beyond (a smooth,
  short-ranged stand-in for tabulated semi-local channels);
* the rotation of walker w at measurement t comes from Philox block (t, 0xD, w, 3), words
  0..2 -> u1, u2, u3, as the unit quaternion (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2,
  sqrt(u1) sin 2pi u3, sqrt(u1) cos 2pi u3) (Shoemake's uniform random rotation), turned into
  a rotation matrix; t is the walker set's sweep counter at the measurement;
* the quadrature point of electron i about ion I is the nearest image of R_I plus r O n_q,
  wrapped into the cell.

This is test infrastructure (part of the FP64 oracle). Each quadrature point's ratio is
taken by LU of the Slater matrix with the moved row replaced and the Jastrow factor is
recomputed in full, as in the oracle's moves.

Pins: the rule integrates P_l(u . n) to delta_l0 for l <= 5 under any rotation and not for
l = 6; with a constant orbital the energy is sum dv_0 over pairs; for one electron in a
plane-wave orbital the quadrature reproduces the closed form i^l j_l(k r) P_l(u . k^) of the
angular integral to the rule's degree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .philox import philox4x32_10, seed_key, to_unit
from .jastrow import min_image

_PHI = (1.0 + math.sqrt(5.0)) / 2.0


def icosahedron() -> np.ndarray:
    """The 12 unit vertices of an icosahedron: (0, +-1, +-phi), (+-1, +-phi, 0), (+-phi, 0, +-1)
    normalised."""
    v = []
    for a in (1.0, -1.0):
        for b in (_PHI, -_PHI):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def legendre(l: int, x):
    """P_l(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x
    if l == 0:
        return p0
    for n in range(1, l):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    return p1


def rotation(seed: int, t: int, walker_id: int) -> np.ndarray:
    """Uniform random rotation matrix of walker `walker_id` at measurement t."""
    w0, w1, w2, _ = philox4x32_10((t, 0xD, walker_id, 3), seed_key(seed))
    u1, u2, u3 = float(to_unit(w0)), float(to_unit(w1)), float(to_unit(w2))
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    # rotation of the unit quaternion w + x i + y j + z k
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class NonLocalPP:
    """Channels dv_l(r) = amp[l] exp(-(r / width[l])^2) for r < rcut, l = 0..len(amp)-1."""
    amp: np.ndarray
    width: np.ndarray
    rcut: float

    def dv(self, l: int, r: float) -> float:
        if not (r < self.rcut):
            return 0.0
        return float(self.amp[l] * math.exp(-(r / self.width[l]) ** 2))


def nonlocal_energy(wf, pp: NonLocalPP, R, seed: int, t: int, walker_id: int,
                    ratio_fn=None) -> float:
    """V_NL of configuration R (N_e, 3) for the Slater-Jastrow function `wf` (the oracle's
    SlaterJastrow) and ions wf.ions: the quadrature sum over every electron-ion pair within
    the cutoff. `ratio_fn(R, i, r_new)` overrides the wavefunction ratio (pins use closed
    forms)."""
    R = np.asarray(R, dtype=np.float64)
    L = wf.L
    O = rotation(seed, t, walker_id)
    pts = icosahedron() @ O.T                     # rotated quadrature directions O n_q
    if ratio_fn is None:
        ratio_fn = lambda RR, i, rn: slater_jastrow_ratio(wf, RR, i, rn)   # noqa: E731
    total = 0.0
    for i in range(R.shape[0]):
        for I in range(wf.ions.shape[0]):
            d = min_image(R[i] - wf.ions[I], L)
            r = float(np.sqrt(d @ d))
            if not (r < pp.rcut) or r == 0.0:
                continue
            u = d / r
            img = R[i] - d                        # nearest image of ion I
            for q in range(12):
                rn = np.mod(img + r * pts[q], L)
                ratio = ratio_fn(R, i, rn)
                cos_t = float(u @ pts[q])
                s = 0.0
                for l in range(len(pp.amp)):
                    s += (2 * l + 1) * pp.dv(l, r) * float(legendre(l, cos_t))
                total += s * ratio / 12.0
    return total


def slater_jastrow_ratio(wf, R, i, r_new) -> float:
    """Psi(R with r_i -> r_new) / Psi(R) by LU of both Slater matrices of the moved block and
    full recomputation of J."""
    spin, first, ns = wf.block(i)
    A = wf.slater_matrix(R, spin)
    s0, l0 = np.linalg.slogdet(A)
    A2 = A.copy()
    A2[i - first] = wf.orb.values(r_new)[:ns]
    s1, l1 = np.linalg.slogdet(A2)
    ratio = 0.0 if s1 == 0.0 else s1 * s0 * math.exp(l1 - l0)
    if wf.jas is not None:
        R2 = R.copy()
        R2[i] = r_new
        ratio *= math.exp(wf.jas.value(R2) - wf.jas.value(R))
    return ratio
