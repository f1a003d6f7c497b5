"""Pins of the oracle's three-body electron-electron-ion Jastrow factor (Sec. "Jastrow
factor": the polynomial in r_iI, r_jI and r_ij of Drummond et al., cut off at r_c / 2)."""
import math

import numpy as np
import pytest

from oracle.jastrow3 import JastrowSum, ThreeBodyJastrow, u3_derivs

L = 12.0
CENTER = np.array([6.0, 6.0, 6.0])


def _gamma(meI, mee, entries):
    g = np.zeros((meI + 1, meI + 1, mee + 1))
    for (l, m, n), v in entries.items():
        g[l, m, n] = v
        g[m, l, n] = v
    return g


def _one_ion(gamma_same, rc=4.0, gamma_opp=None):
    return ThreeBodyJastrow(L, 2, CENTER[None], gamma_same,
                            gamma_same if gamma_opp is None else gamma_opp, rc)


# two electrons at a = 1 and b = 1.5 from the ion, h = 2: (a - h)^3 (b - h)^3 = 1/8, c^2 = 3.25
R2 = np.array([CENTER + [1.0, 0.0, 0.0], CENTER + [0.0, 1.5, 0.0]])


@pytest.mark.parametrize("entries, expect", [
    ({(0, 0, 0): 1.0}, 0.125),
    ({(0, 0, 1): 1.0}, 0.125 * math.sqrt(3.25)),
    ({(1, 0, 0): 1.0}, 0.125 * (1.0 + 1.5)),                     # a + b
    ({(2, 0, 1): 1.0}, 0.125 * (1.0 + 2.25) * math.sqrt(3.25)),  # (a^2 + b^2) c
    ({(1, 1, 2): 1.0}, 0.125 * 1.5 * 3.25),                      # a b c^2
    ({(2, 1, 0): -2.0}, -2.0 * 0.125 * (1.0 ** 2 * 1.5 + 1.0 * 1.5 ** 2)),  # -2 (a^2 b + a b^2)
])
def test_single_terms_closed_form(entries, expect):
    g = _gamma(2, 2, entries)
    assert _one_ion(g).value(R2) == pytest.approx(expect, rel=1e-14)


def test_zero_beyond_half_cutoff():
    g = _gamma(2, 2, {(0, 0, 0): 1.0, (1, 0, 1): 0.3})
    j = _one_ion(g)
    far = np.array([CENTER + [2.0, 0.0, 0.0], CENTER + [0.0, 1.0, 0.0]])   # a = h exactly
    assert j.value(far) == 0.0
    # C2 at a = h: u ~ (h - a)^3, so u, u_a and u_aa vanish as a -> h
    d1 = u3_derivs(2.0 - 1e-3, 1.0, 2.2, g, 2.0)
    d2 = u3_derivs(2.0 - 5e-4, 1.0, 2.2, g, 2.0)
    assert d1[0] / d2[0] == pytest.approx(8.0, rel=1e-2)     # u    ~ (h - a)^3
    assert d1[1] / d2[1] == pytest.approx(4.0, rel=1e-2)     # u_a  ~ (h - a)^2
    assert d1[3] / d2[3] == pytest.approx(2.0, rel=1e-2)     # u_aa ~ (h - a)
    gr, lap = j.grad_lap(far, 0)
    assert np.all(gr == 0.0) and lap == 0.0


def _random_gamma(rng, meI=2, mee=3):
    g = rng.normal(0.0, 0.3, size=(meI + 1, meI + 1, mee + 1))
    return 0.5 * (g + g.transpose(1, 0, 2))


def _cluster(rng, n_e, n_ion, rc):
    ions = rng.uniform(0.0, L, size=(n_ion, 3))
    # electrons placed around the ions so that many triples fall inside r_c / 2
    R = ions[rng.integers(0, n_ion, size=n_e)] + rng.normal(0.0, 0.4 * rc, size=(n_e, 3))
    return np.mod(R, L), ions


def test_gradient_and_laplacian_by_finite_differences():
    rng = np.random.default_rng(11)
    rc = 5.0
    R, ions = _cluster(rng, 7, 3, rc)
    j = ThreeBodyJastrow(L, 4, ions, _random_gamma(rng), _random_gamma(rng), rc)
    assert j.value(R) != 0.0
    h = 1e-4
    for i in range(R.shape[0]):
        g, lap = j.grad_lap(R, i)
        gfd = np.zeros(3)
        lfd = 0.0
        v0 = j.value(R)
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, c] += h
            Rm[i, c] -= h
            vp, vm = j.value(Rp), j.value(Rm)
            gfd[c] = (vp - vm) / (2 * h)
            lfd += (vp - 2 * v0 + vm) / (h * h)
        assert np.allclose(g, gfd, rtol=1e-6, atol=1e-7), (i, g, gfd)
        assert lap == pytest.approx(lfd, rel=1e-4, abs=1e-4), (i, lap, lfd)


def test_exchange_translation_and_spin_assignment():
    rng = np.random.default_rng(12)
    rc = 5.0
    R, ions = _cluster(rng, 6, 2, rc)
    gs, go = _random_gamma(rng), _random_gamma(rng)
    j = ThreeBodyJastrow(L, 3, ions, gs, go, rc)
    v = j.value(R)
    # exchange of two same-spin electrons
    P = R[[1, 0, 2, 3, 4, 5]]
    assert j.value(P) == pytest.approx(v, rel=1e-13)
    # a common translation of electrons and ions, and a lattice translation of one electron
    s = np.array([0.7, -2.1, 5.3])
    jt = ThreeBodyJastrow(L, 3, np.mod(ions + s, L), gs, go, rc)
    assert jt.value(np.mod(R + s, L)) == pytest.approx(v, rel=1e-12)
    Q = R.copy()
    Q[4] += [L, -L, 2 * L]
    assert j.value(Q) == pytest.approx(v, rel=1e-12)
    # with no opposite-spin coefficients the down electrons do not interact with the up ones
    j0 = ThreeBodyJastrow(L, 3, ions, gs, np.zeros_like(go), rc)
    up = ThreeBodyJastrow(L, 3, ions, gs, np.zeros_like(go), rc).value(R[:3])
    dn = ThreeBodyJastrow(L, 0, ions, gs, np.zeros_like(go), rc).value(R[3:])
    assert j0.value(R) == pytest.approx(up + dn, rel=1e-13)


def test_rejects_unsymmetric_or_bad_cutoff():
    g = np.zeros((2, 2, 2))
    g[1, 0, 0] = 1.0
    with pytest.raises(ValueError):
        ThreeBodyJastrow(L, 1, CENTER[None], g, g, 4.0)
    with pytest.raises(ValueError):
        ThreeBodyJastrow(L, 1, CENTER[None], np.zeros((2, 2, 2)), np.zeros((2, 2, 2)), 0.6 * L)


def test_sum_adds_terms():
    rng = np.random.default_rng(13)
    R, ions = _cluster(rng, 5, 2, 5.0)
    a = ThreeBodyJastrow(L, 2, ions, _random_gamma(rng), _random_gamma(rng), 5.0)
    b = ThreeBodyJastrow(L, 2, ions, _random_gamma(rng), _random_gamma(rng), 4.0)
    s = JastrowSum(a, None, b)
    assert s.value(R) == pytest.approx(a.value(R) + b.value(R), rel=1e-14)
    g, lap = s.grad_lap(R, 3)
    assert np.allclose(g, a.grad_lap(R, 3)[0] + b.grad_lap(R, 3)[0], rtol=1e-14, atol=0)
