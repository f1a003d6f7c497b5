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


def oracle_vmc(inputs, walker_ids, n_sweeps, forced=None, coef=None, electrons=None):
    """Oracle trace [n_w][sweeps*n_e][8] and energies [n_w][sweeps][3]."""
    sysm = OracleSystem(inputs, coef=coef)
    pos = inputs["pos"][walker_ids]
    if electrons is None:
        return run_vmc(sysm, pos, walker_ids, n_sweeps, forced=forced)
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
