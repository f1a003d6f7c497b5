"""Helpers shared by the GPU parity tests: run the oracle on the same seeded inputs and
compare per-move traces."""
from __future__ import annotations

import numpy as np

from oracle.vmc import OracleSystem, run_vmc

FIELDS = ("ratio", "dJ", "gx", "gy", "gz", "u", "A", "accepted")


def bf16_round(x: np.ndarray) -> np.ndarray:
    """double -> float32 (nearest) -> bfloat16 (nearest even), returned as float64: the
    rounding the library applies when it stores a BF16 coefficient table."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# Per-move gate of the single-precision ratios (reading 13): the relative error (floor
# 1e-3 on |R|) of every move is at most max(1e-4, RATIO_C cond 2^-24), cond the larger
# 2-norm condition number of the moved spin block's Slater matrix before and after the
# move (oracle, FP64). Each rounding of the stored A^-1 to single precision (at walker
# creation or re-inversion, and at every flush of a delayed window or rank-1 update) can
# move a ratio by about cond 2^-24, and so can the single-precision orbital row; every
# tested configuration has at most 15 flushes between re-inversions, hence RATIO_C = 16.
RATIO_C = 16.0
RATIO_FLOOR = 1e-3


def ratio_gate(gpu_ratio, ref_ratio, cond, c=RATIO_C, floor=RATIO_FLOOR):
    """(relative errors, per-move bounds) of GPU ratios against the oracle's."""
    err = rel_err(gpu_ratio, ref_ratio, floor)
    bound = np.maximum(1e-4, c * np.asarray(cond) * 2.0 ** -24)
    return err, bound


def assert_ratio_gate(gpu_ratio, ref_ratio, cond, label=""):
    err, bound = ratio_gate(gpu_ratio, ref_ratio, cond)
    q = err / bound
    worst = np.unravel_index(np.argmax(q), q.shape)
    print(f"{label}: ratio rel err median {np.median(err):.2e} p90 {np.quantile(err, 0.9):.2e} "
          f"max {err.max():.2e}; worst err/bound {q.max():.3f} (cond {np.asarray(cond)[worst]:.3g})")
    assert q.max() <= 1.0, (f"{label}: move {worst} ratio error {err[worst]:.3e} above its "
                            f"bound {bound[worst]:.3e} (cond {np.asarray(cond)[worst]:.3g})")


def oracle_vmc(inputs, walker_ids, n_sweeps, forced=None, coef=None, electrons=None,
               conds=None):
    """Oracle trace [n_w][sweeps*n_e][8] and energies [n_w][sweeps][3]."""
    sysm = OracleSystem(inputs, coef=coef)
    pos = inputs["pos"][walker_ids]
    if electrons is None:
        return run_vmc(sysm, pos, walker_ids, n_sweeps, forced=forced, conds=conds)
    walkers = [sysm.walker(R, wid) for R, wid in zip(pos, walker_ids)]
    tr = []
    for w in walkers:
        rows = []
        sysm.sweep(w, 0, trace=rows, electrons=electrons)
        tr.append(np.array(rows))
    return walkers, np.array(tr), None


def rel_err(a, b, floor):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(b), floor)


def assert_trace_close(gpu, ref, rtol, ratio_floor=1e-3, exact_decisions=True):
    """Compare traces [n_w][moves][8]."""
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    assert np.array_equal(gpu[..., 5], ref[..., 5]), "acceptance variates differ"
    if exact_decisions:
        bad = np.argwhere(gpu[..., 7] != ref[..., 7])
        assert bad.size == 0, f"decisions differ at {bad[:5]}"
    r = rel_err(gpu[..., 0], ref[..., 0], ratio_floor)
    assert r.max() <= rtol, f"ratio max rel err {r.max():.3e}"
    d = np.abs(gpu[..., 1] - ref[..., 1]) / np.maximum(np.abs(ref[..., 1]), 1.0)
    assert d.max() <= rtol, f"dJ max err {d.max():.3e}"
    g = np.linalg.norm(gpu[..., 2:5] - ref[..., 2:5], axis=-1) / np.maximum(
        np.linalg.norm(ref[..., 2:5], axis=-1), 1.0)
    assert g.max() <= rtol * 10, f"grad max rel err {g.max():.3e}"
    a = np.abs(gpu[..., 6] - ref[..., 6])
    assert a.max() <= rtol * 10, f"A max err {a.max():.3e}"


# Gate of ln|Psi| in the single-precision forms (reading 18): LOGPSI_ABS + LOGPSI_PER_E * N_e
# absolute, right after a log-determinant anchor. What remains there is set by single
# precision itself: the orbital rows of A in FP32 move ln|det A| by about tr(A^-1 dA)
# (measured 1e-5 at 40 electrons, 3-7e-5 at 512, ~2e-4 at 1024, against ln|det| of the
# FP64 orbitals), and J, a sum of ~10^5 pair terms, is evaluated from FP32 distances
# (~1e-5). Between anchors the FP64 sum of the moves' ln|R| adds the ratios' own errors.
LOGPSI_ABS = 2e-5
LOGPSI_PER_E = 3e-7


def logpsi_tol(n_e: int) -> float:
    return LOGPSI_ABS + LOGPSI_PER_E * n_e


def logpsi_errors(gpu_lp, ref_lp):
    """|ln|Psi|_GPU - ln|Psi|_oracle| (absolute; ln|Psi| is a sum of ~10^5 terms whose
    magnitude, not the result's, sets the scale of single-precision errors)."""
    return np.abs(np.asarray(gpu_lp) - np.asarray(ref_lp))


def assert_logpsi(gpu_lp, ref_lp, n_e, label="", extra=0.0):
    err = logpsi_errors(gpu_lp, ref_lp)
    tol = logpsi_tol(n_e) + extra
    print(f"{label}: ln|Psi| error max {err.max():.2e} (gate {tol:.2e})")
    assert err.max() <= tol, (label, float(err.max()), tol)


# Single-precision local energy, per walker: max(1e-5 Ha per electron, 2^-24 cond K), where
# K = sum_i [ sum_j |lap phi_j(r_i) Ainv[j][i]| + 2 |grad_i ln D| sum_j |grad phi_j(r_i)| |Ainv[j][i]| ]
# is the sum of the magnitudes of the kinetic energy's determinant terms and cond the larger
# 2-norm condition number of the two Slater matrices: to first order the dot products add
# about 2^-24 of K, and an inverse carried to a relative error of about cond 2^-24 adds
# cond 2^-24 of K.
EL_PER_E = 1e-5


def el_gate(wf, R) -> float:
    R = np.asarray(R, dtype=np.float64)
    kmag, cond = 0.0, 1.0
    inv = {}
    for sp in (0, 1):
        ns = wf.n_up if sp == 0 else wf.n_dn
        if ns:
            A = wf.slater_matrix(R, sp)
            inv[sp] = np.linalg.inv(A)
            cond = max(cond, float(np.linalg.cond(A)))
    for i in range(R.shape[0]):
        spin, first, ns = wf.block(i)
        _, grad, lap = wf.orb.vgl(R[i])
        col = inv[spin][:, i - first]
        g = grad[:, :ns] @ col
        kmag += float(np.abs(lap[:ns] * col).sum() + 2.0 * np.linalg.norm(g) * np.abs(grad[:, :ns] * col).sum())
    return max(EL_PER_E * R.shape[0], 2.0 ** -24 * cond * kmag)
