"""GPU parity of the non-local pseudopotential energy (Sec. "Hamiltonian": semi-local
channels, 12-point angular quadrature after Mitas et al.) against the FP64 oracle at the
GPU's own walker positions and measurement counter.

FP64: V_NL of every walker to 1e-10. Single precision: each quadrature ratio carries the
ratio error of the sweep's moves (1e-4 relative, or cond 2^-24), so V_NL is gated at
1e-4 of the sum of the magnitudes of its terms. E_L minus V_NL is the local energy of the
same state measured without the channels (and, in FP64, the oracle's).
"""
import math

import numpy as np
import pytest

from synthetic import build_inputs, small_spec, spec_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1802_06922_gb300 as q   # noqa: E402
from oracle.jastrow import functor, min_image   # noqa: E402
from oracle.nlpp import NonLocalPP, icosahedron, nonlocal_energy, rotation   # noqa: E402
from oracle.vmc import OracleSystem   # noqa: E402

AMP, WIDTH = np.array([1.5, -1.0]), np.array([1.0, 0.9])


def _fast_ratio(osys, R):
    """Psi ratio of a single-electron move from the FP64 inverses (determinant lemma) and the
    moved electron's Jastrow pair terms: exact, and fast enough for 512 electrons."""
    wf = osys.wf
    inv = {sp: np.linalg.inv(wf.slater_matrix(R, sp)) for sp in (0, 1)}
    jas = wf.jas

    def ratio(RR, i, rn):
        spin, first, ns = wf.block(i)
        det = float(wf.orb.values(rn)[:ns] @ inv[spin][:, i - first])
        dj = 0.0
        parts = []
        if jas.p_eI.size and jas.ions.shape[0]:
            parts.append((jas.ions, jas.p_eI))
        others = np.delete(np.arange(RR.shape[0]), i)
        same = (others < wf.n_up) == (i < wf.n_up)
        if jas.p_same.size:
            parts += [(RR[others[same]], jas.p_same), (RR[others[~same]], jas.p_opp)]
        for X, p in parts:
            if X.shape[0] == 0:
                continue
            dn = np.linalg.norm(min_image(rn - X, wf.L), axis=1)
            do = np.linalg.norm(min_image(RR[i] - X, wf.L), axis=1)
            dj += functor(dn, p, jas.rc)[0].sum() - functor(do, p, jas.rc)[0].sum()
        return det * math.exp(dj)
    return ratio


def _magnitude(wf, pp, R, seed, t, wid, ratio_fn):
    """Sum over the pairs inside the cutoff of sum_l (2l+1) |dv_l(r)| max_q |ratio_q|: the
    scale of V_NL's terms, which cancel in the sum."""
    pts = icosahedron() @ rotation(seed, t, wid).T
    tot = 0.0
    for i in range(R.shape[0]):
        for I in range(wf.ions.shape[0]):
            d = min_image(R[i] - wf.ions[I], wf.L)
            r = float(np.sqrt(d @ d))
            if not (r < pp.rcut):
                continue
            rat = max(abs(ratio_fn(R, i, np.mod(R[i] - d + r * p, wf.L))) for p in pts)
            tot += sum((2 * l + 1) * abs(pp.dv(l, r)) for l in range(len(pp.amp))) * rat
    return tot


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_nonlocal_energy_small_system(precision):
    inputs = build_inputs(small_spec(8, 7, grid=12), n_walkers=6)
    rcut = 2.5
    pp = NonLocalPP(AMP, WIDTH, rcut)
    coef = None
    if precision == "bf16":
        from parity_util import bf16_round
        coef = bf16_round(inputs["coef"])
        inputs = dict(inputs, coef=coef)
    s = q.system_from_inputs(inputs, precision=precision, delay_k=4)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(1)
    s.set_nonlocal(AMP, WIDTH, rcut)
    w.sweep(1)                                   # measured with the channels at t = 2
    e_gpu, _ = w.measure()
    vnl = w.nonlocal_energy()
    pos = w.positions()
    osys = OracleSystem(inputs, coef=coef)
    n_pairs = 0
    for k in range(6):
        ref = nonlocal_energy(osys.wf, pp, pos[k], seed=inputs["seed"], t=2, walker_id=k)
        e_ref = osys.wf.local_energy(pos[k])[0]
        mag = _magnitude(osys.wf, pp, pos[k], inputs["seed"], 2, k, _fast_ratio(osys, pos[k]))
        if precision == "fp64":
            assert abs(vnl[k] - ref) <= 1e-10 * max(1.0, abs(ref)), (k, vnl[k], ref)
            assert abs(e_gpu[k] - vnl[k] - e_ref) <= 1e-10 * max(1.0, abs(e_ref))
        else:
            assert abs(vnl[k] - ref) <= 1e-4 * mag + 1e-12, (k, vnl[k], ref)
        n_pairs += int(ref != 0.0)
    assert n_pairs >= 3, "too few electron-ion pairs inside the cutoff to test anything"
    # the channels add V_NL and nothing else: the same state measured without them gives
    # E_L - V_NL (up to the rounding of the double-precision add)
    s.set_nonlocal([], [], 1.0)
    e_local, _ = w.measure()
    assert np.all(w.nonlocal_energy() == 0.0)
    assert np.allclose(e_gpu - vnl, e_local, rtol=1e-13, atol=1e-13)
    w.close()
    s.close()


def test_nonlocal_energy_full_size_sampled():
    """The 512-electron workload with the channels, in the bench's launch configuration
    (FP32, k = 32): V_NL of sampled walkers against the oracle's quadrature with FP64 ratios."""
    spec = spec_for("sj512")
    inputs = build_inputs(spec)
    rcut = 1.6
    s = q.system_from_inputs(inputs, precision="fp32", delay_k=32, reinv_period=128,
                             logdet_period=1024)
    s.set_nonlocal(AMP, WIDTH, rcut)
    w = q.Walkers(s, inputs["pos"])
    w.sweep(2)
    vnl = w.nonlocal_energy()
    pos = w.positions()
    osys = OracleSystem(inputs)
    pp = NonLocalPP(AMP, WIDTH, rcut)
    for k in (0, 200):
        ratio = _fast_ratio(osys, pos[k])
        ref = nonlocal_energy(osys.wf, pp, pos[k], seed=inputs["seed"], t=2, walker_id=k,
                              ratio_fn=ratio)
        mag = _magnitude(osys.wf, pp, pos[k], inputs["seed"], 2, k, ratio)
        print(f"walker {k}: V_NL {vnl[k]:.6f} oracle {ref:.6f} scale {mag:.3f}")
        assert abs(vnl[k] - ref) <= 1e-4 * mag + 1e-12, (k, vnl[k], ref)
        assert ref != 0.0
    w.close()
    s.close()
