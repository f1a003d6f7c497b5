"""Pins of the oracle's tricubic B-spline orbitals (CPU)."""
import json
import os

import numpy as np
import pytest

from oracle.orbitals import PlaneWaveOrbitals, SplineOrbitals, bspline_basis
from synthetic import build_inputs, small_spec, spec_for, spline_coefficients

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def test_basis_closed_forms_and_partition_of_unity():
    b, db, _ = bspline_basis(0.0)
    assert np.allclose(b, GOLD["cubic_bspline_node_weights"]["value"], atol=1e-16)
    assert np.allclose(db, GOLD["cubic_bspline_node_first_derivatives"]["value"], atol=1e-16)
    t = np.linspace(0, 1, 101)
    b, db, d2b = bspline_basis(t)
    assert np.allclose(b.sum(0), 1, atol=1e-15)
    assert np.allclose(db.sum(0), 0, atol=1e-14)
    assert np.allclose(d2b.sum(0), 0, atol=1e-14)
    # continuity across the node: weights at t=1 equal the next cell's weights at t=0 shifted
    b1, db1, d2b1 = bspline_basis(1.0)
    b0, db0, d2b0 = bspline_basis(0.0)
    assert np.allclose(b1[1:], b0[:3], atol=1e-15)
    assert np.allclose(db1[1:], db0[:3], atol=1e-15)
    assert np.allclose(d2b1[1:], d2b0[:3], atol=1e-14)


# Marsden's identity for uniform cubic B-splines: coefficient sequences 1, g, g^2 - 1/3 and
# g^3 - g reproduce 1, s, s^2 and s^3 exactly (s in grid units).
_MARSDEN = [lambda g: np.ones_like(g), lambda g: g, lambda g: g * g - 1.0 / 3.0,
            lambda g: g ** 3 - g]


def _poly(c, s):
    return sum(c[k] * s ** k for k in range(4))


def _dpoly(c, s):
    return sum(k * c[k] * s ** (k - 1) for k in range(1, 4))


def _d2poly(c, s):
    return sum(k * (k - 1) * c[k] * s ** (k - 2) for k in range(2, 4))


def test_cubic_polynomial_reproduction_with_exact_derivatives():
    n = np.array([20, 24, 28])            # distinct axes catch a transposed axis
    L = 7.0
    delta = L / n
    rng = np.random.default_rng(0)
    n_orb = 3
    cx, cy, cz = (rng.normal(size=(n_orb, 4)) for _ in range(3))
    coef = np.zeros((n[0], n[1], n[2], n_orb))
    for o in range(n_orb):
        per_axis = []
        for ax, c in zip(range(3), (cx, cy, cz)):
            g = np.arange(n[ax], dtype=float)
            per_axis.append(sum(c[o, k] * _MARSDEN[k](g) for k in range(4)))
        coef[..., o] = np.einsum("a,b,c->abc", *per_axis)
    orb = SplineOrbitals(coef, L)
    for _ in range(25):
        s = np.array([rng.uniform(2, n[d] - 3) for d in range(3)])    # away from the wrap
        r = s * delta
        val, grad, lap = orb.vgl(r)
        for o in range(n_orb):
            px, py, pz = _poly(cx[o], s[0]), _poly(cy[o], s[1]), _poly(cz[o], s[2])
            dx, dy, dz = (_dpoly(cx[o], s[0]) / delta[0], _dpoly(cy[o], s[1]) / delta[1],
                          _dpoly(cz[o], s[2]) / delta[2])
            ddx, ddy, ddz = (_d2poly(cx[o], s[0]) / delta[0] ** 2,
                             _d2poly(cy[o], s[1]) / delta[1] ** 2,
                             _d2poly(cz[o], s[2]) / delta[2] ** 2)
            scale = 1 + abs(px * py * pz)
            assert abs(val[o] - px * py * pz) < 1e-11 * scale * 1e3
            assert np.allclose(grad[:, o], [dx * py * pz, px * dy * pz, px * py * dz],
                               rtol=1e-9, atol=1e-9 * scale)
            assert abs(lap[o] - (ddx * py * pz + px * ddy * pz + px * py * ddz)) < 1e-8 * scale


@pytest.mark.parametrize("name", ["pw14", "sj128"])
def test_closed_form_fit_interpolates_at_every_node(name):
    d = build_inputs(spec_for(name), n_walkers=1)
    spec = d["spec"]
    sp = SplineOrbitals(d["coef"], spec.L)
    pw = PlaneWaveOrbitals(d["nvec"], d["kind"], d["amp"], spec.L)
    rng = np.random.default_rng(1)
    for _ in range(20):
        g = rng.integers(0, spec.grid, size=3)
        r = g * spec.L / spec.grid
        assert np.allclose(sp.values(r), pw.values(r), rtol=0, atol=1e-11)


def test_spline_close_to_plane_waves_between_nodes():
    d = build_inputs(spec_for("pw14"), n_walkers=1)
    spec = d["spec"]
    sp = SplineOrbitals(d["coef"], spec.L)
    pw = PlaneWaveOrbitals(d["nvec"], d["kind"], d["amp"], spec.L)
    kd = 2 * np.pi / spec.L * spec.L / spec.grid
    rng = np.random.default_rng(2)
    for _ in range(20):
        r = rng.uniform(0, spec.L, 3)
        v1, g1, l1 = sp.vgl(r)
        v2, g2, l2 = pw.vgl(r)
        assert np.abs(v1 - v2).max() < 2 * kd ** 4
        assert np.abs(g1 - g2).max() < 2 * kd ** 3 * (2 * np.pi / spec.L)
        assert np.abs(l1 - l2).max() < 2 * kd ** 2 * (2 * np.pi / spec.L) ** 2


def test_gradient_and_laplacian_match_finite_differences():
    d = build_inputs(small_spec(5, 5, grid=12), n_walkers=1)
    sp = SplineOrbitals(d["coef"], d["spec"].L)
    rng = np.random.default_rng(3)
    h = 1e-4
    for _ in range(10):
        r = rng.uniform(0, d["spec"].L, 3)
        v, g, lap = sp.vgl(r)
        fd_lap = np.zeros_like(lap)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            vp, gp, _ = sp.vgl(r + e)
            vm, gm, _ = sp.vgl(r - e)
            assert np.allclose((vp - vm) / (2 * h), g[ax], rtol=1e-6, atol=1e-6)
            fd_lap += (gp[ax] - gm[ax]) / (2 * h)
        assert np.allclose(fd_lap, lap, rtol=1e-5, atol=1e-5)


def test_periodic_wrap():
    d = build_inputs(small_spec(4, 4, grid=10), n_walkers=1)
    L = d["spec"].L
    sp = SplineOrbitals(d["coef"], L)
    r = np.array([0.3, 1.7, 2.9])
    for shift in ([L, 0, 0], [0, -L, 0], [0, 0, 2 * L]):
        assert np.allclose(sp.vgl(r)[0], sp.vgl(r + np.array(shift))[0], atol=1e-13)


def test_separable_fit_matches_direct_plane_wave_sum():
    """The generator's separable Fourier sum agrees with a direct per-node evaluation of
    sum_t a_t trig(k_t . r_g) / prod_d factor_d."""
    spec = small_spec(3, 3, grid=6)
    d = build_inputs(spec, n_walkers=1)
    nvec, kind, amp = d["nvec"], d["kind"], d["amp"]
    n = spec.grid
    coef = spline_coefficients(nvec, kind, amp, n)
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    fac = lambda m: (4 + 2 * np.cos(2 * np.pi * m / n)) / 6
    for o in range(nvec.shape[0]):
        ref = np.zeros(g.shape[0])
        for t in range(nvec.shape[1]):
            ph = 2 * np.pi * (g @ nvec[o, t]) / n
            f = np.sin(ph) if kind[o, t] else np.cos(ph)
            ref += amp[o, t] * f / np.prod(fac(nvec[o, t]))
        assert np.allclose(coef[..., o].reshape(-1), ref, atol=1e-12)
