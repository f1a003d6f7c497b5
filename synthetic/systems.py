"""Synthetic Slater-Jastrow systems shaped like the paper's periodic solid-state workloads.

The paper's production inputs (DFT orbitals converted to B-splines, pseudopotentials,
NiO/TiO2/VO2 structures; Sec. "B-spline basis sets", Sec. "Applications") are not
available, so every system here is generated from a seed:

* a cubic periodic cell of side L (bohr) holding n_up + n_dn electrons;
* ions on an fcc or bcc lattice (or a seeded subset of one) with a small Gaussian jitter;
* orbitals that are seeded sums of 20 real plane waves a*cos(k.r) or a*sin(k.r) with
  k = 2*pi*n/L, |n| <= n_c and a ~ N(0, 1); one orbital set is shared by both spins,
  as the paper shares one B-spline table per node or GPU;
* the periodic tricubic B-spline coefficients of those orbitals on an n^3 grid, in the
  closed form that makes the spline interpolate every orbital exactly at the grid nodes;
* three 1D cubic B-spline Jastrow functors (electron-ion, same-spin and opposite-spin
  electron pairs) with M intervals to the cutoff L/2, p_1..p_{M-1} ~ U(-0.5, 0),
  p_M = 0 and p_0 = p_2 (zero cusp);
* initial electron positions uniform in the cell.

All randomness comes from numpy's PCG64 generator seeded with the system seed, so the
same seed always yields the same arrays on every machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """Sizes and physical parameters of one synthetic system (Hartree atomic units)."""
    name: str
    n_up: int
    n_dn: int
    L: float
    grid: int
    n_orb: int
    n_ion: int
    ion_lattice: str            # "fcc", "bcc", "fcc-subset" or "none"
    jastrow_M: int              # 0 disables the Jastrow factor
    n_walkers: int
    n_sweeps: int
    move: str = "metropolis"    # or "drift"
    step: float = 0.3           # sigma (Metropolis) or tau (drift)
    ion_Z: float = 4.0
    kappa: float = 1.0          # Yukawa screening (1/bohr)
    orbitals: str = "random"    # "random" (20 plane waves each) or "pw7" (k=0 and |k|=2pi/L)
    n_terms: int = 20
    with_potential: bool = True

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_dn


def n_c_for(n_orb: int) -> int:
    """Smallest integer n_c >= 3 whose ball |n| <= n_c holds at least 1.5 * n_orb lattice
    points, so that n_orb random plane-wave sums are linearly independent."""
    n_c = 3
    while _ball(n_c).shape[0] < 1.5 * n_orb:
        n_c += 1
    return n_c


def _ball(n_c: int) -> np.ndarray:
    r = np.arange(-n_c, n_c + 1)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    return g[(g * g).sum(1) <= n_c * n_c]


# The five workloads: plain plane-wave VMC, Slater-Jastrow VMC at 128, 512 and 1024
# electrons, and the three systems of the batched DMC-style workload.
PRESETS: Dict[str, SystemSpec] = {
    "pw14": SystemSpec("pw14", 7, 7, 10.0, 32, 7, 0, "none", 0, 32, 200,
                       step=0.5, orbitals="pw7", with_potential=False),
    "sj128": SystemSpec("sj128", 64, 64, 15.0, 48, 64, 32, "fcc", 8, 512, 100),
    "sj512": SystemSpec("sj512", 256, 256, 24.0, 64, 256, 128, "bcc", 8, 256, 50),
    "dmc64": SystemSpec("dmc64", 32, 32, 15.0 * (64 / 128) ** (1 / 3), 48, 32, 16,
                        "fcc-subset", 8, 768, 100, move="drift", step=0.01),
    "dmc192": SystemSpec("dmc192", 96, 96, 15.0 * (192 / 128) ** (1 / 3), 56, 96, 48,
                         "fcc-subset", 8, 512, 100, move="drift", step=0.01),
    "dmc384": SystemSpec("dmc384", 192, 192, 15.0 * (384 / 128) ** (1 / 3), 64, 192, 96,
                         "fcc-subset", 8, 256, 100, move="drift", step=0.01),
    "sj1024": SystemSpec("sj1024", 512, 512, 30.0, 96, 512, 256, "fcc", 10, 128, 20),
}


def spec_for(name: str, **overrides) -> SystemSpec:
    return dataclasses.replace(PRESETS[name], **overrides)


def small_spec(n_up: int, n_dn: int, grid: int = 16, n_ion: Optional[int] = None,
               jastrow_M: int = 8, move: str = "metropolis", step: float = 0.3,
               n_walkers: int = 4, n_sweeps: int = 2, L: Optional[float] = None,
               with_potential: bool = True, n_orb: Optional[int] = None) -> SystemSpec:
    """A small Slater-Jastrow system at the density of the 128-electron workload, for
    tests the oracle finishes in seconds."""
    ne = n_up + n_dn
    if L is None:
        L = 15.0 * (ne / 128.0) ** (1.0 / 3.0)
    if n_ion is None:
        n_ion = max(1, ne // 4)
    return SystemSpec(f"small{ne}", n_up, n_dn, float(L), grid,
                      n_orb if n_orb is not None else max(n_up, n_dn), n_ion,
                      "fcc-subset", jastrow_M, n_walkers, n_sweeps, move=move, step=step,
                      with_potential=with_potential)


# ----------------------------------------------------------------------------- ions
def _fcc(n: int) -> np.ndarray:
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (cells[:, None, :] + base[None]).reshape(-1, 3) / n


def _bcc(n: int) -> np.ndarray:
    base = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (cells[:, None, :] + base[None]).reshape(-1, 3) / n


def make_ions(spec: SystemSpec, rng: np.random.Generator) -> np.ndarray:
    """Ion positions (n_ion, 3) in [0, L)^3."""
    if spec.n_ion == 0:
        return np.zeros((0, 3))
    if spec.ion_lattice == "fcc":
        n = round((spec.n_ion / 4) ** (1 / 3))
        frac = _fcc(n)
    elif spec.ion_lattice == "bcc":
        n = round((spec.n_ion / 2) ** (1 / 3))
        frac = _bcc(n)
    else:
        n = 1
        while 4 * n ** 3 < spec.n_ion:
            n += 1
        frac = _fcc(n)[rng.permutation(4 * n ** 3)[: spec.n_ion]]
    assert frac.shape[0] == spec.n_ion, (spec.name, frac.shape)
    pos = frac * spec.L + rng.normal(0.0, 0.05 * spec.L / n, size=frac.shape)
    return np.mod(pos, spec.L)


# ------------------------------------------------------------------------- orbitals
def make_orbital_terms(spec: SystemSpec, rng: np.random.Generator):
    """Plane-wave recipe of every orbital: integer wave vectors n (n_orb, T, 3), kind
    (n_orb, T) with 0 = cos and 1 = sin, and amplitudes (n_orb, T)."""
    if spec.orbitals == "pw7":
        nvec = np.array([[0, 0, 0], [1, 0, 0], [1, 0, 0], [0, 1, 0], [0, 1, 0],
                         [0, 0, 1], [0, 0, 1]])[:, None, :]
        kind = np.array([0, 0, 1, 0, 1, 0, 1])[:, None]
        amp = np.ones((7, 1))
        return nvec[: spec.n_orb], kind[: spec.n_orb], amp[: spec.n_orb]
    ball = _ball(n_c_for(spec.n_orb))
    idx = rng.integers(0, ball.shape[0], size=(spec.n_orb, spec.n_terms))
    nvec = ball[idx]
    kind = rng.integers(0, 2, size=(spec.n_orb, spec.n_terms))
    kind[(nvec == 0).all(-1)] = 0          # n = 0 is always the constant (cos) term
    amp = rng.normal(0.0, 1.0, size=(spec.n_orb, spec.n_terms))
    return nvec, kind, amp


def spline_coefficients(nvec: np.ndarray, kind: np.ndarray, amp: np.ndarray,
                        grid: int, chunk: int = 8) -> np.ndarray:
    """Periodic tricubic B-spline coefficients [grid][grid][grid][n_orb] (float64).

    For a plane wave e^{i 2 pi n.g / grid} the coefficient sequence divided, per axis, by
    (4 + 2 cos(2 pi n_d / grid)) / 6 makes the uniform cubic B-spline reproduce the wave
    exactly at every grid node, because a node value of such a spline is
    (c_{g-1} + 4 c_g + c_{g+1}) / 6 along each axis. The sum over the (few) distinct wave
    vectors is done as three small separable discrete Fourier sums.
    """
    n_orb, _, _ = nvec.shape
    n_c = int(np.abs(nvec).max()) if nvec.size else 0
    nf = 2 * n_c + 1
    # spectrum S[o, nx, ny, nz] (complex) with cos -> a, sin -> -i a, divided by the
    # node-interpolation factor.
    fac1d = (4.0 + 2.0 * np.cos(2.0 * np.pi * np.arange(-n_c, n_c + 1) / grid)) / 6.0
    S = np.zeros((n_orb, nf, nf, nf), dtype=np.complex128)
    w = amp * np.where(kind == 0, 1.0 + 0j, -1j)
    f = fac1d[nvec[..., 0] + n_c] * fac1d[nvec[..., 1] + n_c] * fac1d[nvec[..., 2] + n_c]
    w = w / f
    o_idx = np.broadcast_to(np.arange(n_orb)[:, None], w.shape)
    np.add.at(S, (o_idx, nvec[..., 0] + n_c, nvec[..., 1] + n_c, nvec[..., 2] + n_c), w)
    g = np.arange(grid)
    E = np.exp(2j * np.pi * np.outer(np.arange(-n_c, n_c + 1), g) / grid)   # [nf, grid]
    T1 = np.tensordot(S, E, axes=([3], [0]))            # [o, nx, ny, gz]
    T2 = np.einsum("oxyz,yg->oxgz", T1, E)               # [o, nx, gy, gz]
    T2 = np.ascontiguousarray(np.transpose(T2, (1, 2, 3, 0)))   # [nx, gy, gz, o]
    out = np.empty((grid, grid, grid, n_orb))
    flat = T2.reshape(nf, -1)
    for g0 in range(0, grid, chunk):
        g1 = min(grid, g0 + chunk)
        out[g0:g1] = (E[:, g0:g1].T @ flat).real.reshape(g1 - g0, grid, grid, n_orb)
    return out


# -------------------------------------------------------------------------- Jastrow
def make_jastrow(spec: SystemSpec, rng: np.random.Generator) -> Dict[str, np.ndarray]:
    """Control points p_0..p_M of the three radial functors (e-ion, same-spin pair,
    opposite-spin pair): p_1..p_{M-1} ~ U(-0.5, 0), p_M = 0, p_0 = p_2 (zero cusp)."""
    out = {}
    M = spec.jastrow_M
    for key in ("eI", "same", "opp"):
        if M == 0 or (key == "eI" and spec.n_ion == 0):
            out[key] = np.zeros(0)
            continue
        p = np.zeros(M + 1)
        p[1:M] = rng.uniform(-0.5, 0.0, size=M - 1)
        p[M] = 0.0
        p[0] = p[2]
        out[key] = p
    return out


# ---------------------------------------------------------------------------- build
def build_inputs(spec: SystemSpec, seed: int = 0, n_walkers: Optional[int] = None,
                 with_coefficients: bool = True) -> dict:
    """All arrays of one system. Walker positions are (n_walkers, n_elec, 3) with the
    n_up up-spin electrons first."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, _name_key(spec.name)]))
    ions = make_ions(spec, rng)
    nvec, kind, amp = make_orbital_terms(spec, rng)
    jas = make_jastrow(spec, rng)
    nw = spec.n_walkers if n_walkers is None else n_walkers
    pos = rng.uniform(0.0, spec.L, size=(nw, spec.n_elec, 3))
    out = dict(spec=spec, seed=seed, ions=ions, nvec=nvec, kind=kind, amp=amp,
               jastrow=jas, pos=pos, rcut=spec.L / 2.0)
    if with_coefficients:
        out["coef"] = spline_coefficients(nvec, kind, amp, spec.grid)
    return out


def _name_key(name: str) -> int:
    return int.from_bytes(name.encode()[:8].ljust(8, b"\0"), "little")


def jastrow3_coefficients(m_ei: int, m_ee: int, rc: float, seed: int = 0):
    """Coefficient sets (same spin, opposite spin) of the three-body e-e-I polynomial, each
    [m_ei+1][m_ei+1][m_ee+1] and symmetric in its first two indices: gamma_lmn =
    x_lmn * 0.05 / h^(6 + l + m + n) with h = rc / 2 and x ~ N(0, 1) symmetrised, so that every
    term of the polynomial times the cutoff factors is of order 0.05 inside the sphere."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4A33]))
    h = 0.5 * rc
    l = np.arange(m_ei + 1)[:, None, None]
    m = np.arange(m_ei + 1)[None, :, None]
    n = np.arange(m_ee + 1)[None, None, :]
    scale = 0.05 / h ** (6 + l + m + n)
    out = []
    for _ in range(2):
        x = rng.normal(0.0, 1.0, size=(m_ei + 1, m_ei + 1, m_ee + 1))
        out.append(0.5 * (x + x.transpose(1, 0, 2)) * scale)
    return out[0], out[1]
