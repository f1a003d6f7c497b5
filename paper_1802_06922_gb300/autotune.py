"""Choice of the launch parameters of a sweep by measurement.

A larger delay rank k makes each move's window work (the d, z and x of the delayed update)
longer and each flush rarer; a smaller proposal batch (moves whose proposals and orbital
rows one launch pair forms) keeps those rows in L2 until the sweep reads them but adds
launches. The best pair depends on the system size, the walker count and the GPU, so
`tune_launch` times a few sweeps for every candidate pair on the caller's own inputs and keeps
the fastest (`tune_delay` does the same for k alone). Timing uses the library's per-kernel
device-time profiling (`qmc_profile_read`); the classes whose cost depends on neither
parameter (re-inversion, local energy) are left out of the ranking. Neither parameter
changes the Markov chain.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional, Tuple

from .qmcgb import KERNEL_CLASSES, Walkers, system_from_inputs

# kernel classes whose device time changes with the delay rank or the proposal batch
_K_DEPENDENT = ("propose", "vgl", "sweep", "flush")


def _time_sweeps(inputs, pos, precision, k, chunk, reinv_period, reinv_on_accepted,
                 warm_sweeps, timed_sweeps) -> float:
    idx = [KERNEL_CLASSES.index(c) for c in _K_DEPENDENT]
    s = system_from_inputs(inputs, precision=precision, delay_k=int(k), prop_chunk=int(chunk),
                           reinv_period=reinv_period, reinv_on_accepted=reinv_on_accepted)
    w = Walkers(s, pos)
    try:
        w.sweep(warm_sweeps)
        w.profile(True)
        w.sweep(timed_sweeps)
        ms, _ = w.profile_read()
        return float(sum(ms[i] for i in idx)) / timed_sweeps
    finally:
        w.close()
        s.close()


def tune_delay(inputs: dict, positions=None, candidates: Iterable[int] = (8, 16, 32),
               precision: str = "fp32", reinv_period: int = 0, reinv_on_accepted: bool = False,
               warm_sweeps: int = 2, timed_sweeps: int = 1) -> Tuple[int, Dict[int, float]]:
    """Returns (best k, {k: device ms per sweep of the k-dependent kernels}) with whole-block
    proposal batches.

    `inputs` is a ``synthetic.build_inputs``-style dictionary; `positions` (host array
    [n_walkers][n_elec][3]) defaults to ``inputs["pos"]``.
    """
    pos = inputs["pos"] if positions is None else positions
    times = {int(k): _time_sweeps(inputs, pos, precision, k, 0, reinv_period, reinv_on_accepted,
                                  warm_sweeps, timed_sweeps) for k in candidates}
    best = min(times, key=times.get)
    return best, times


def tune_launch(inputs: dict, positions=None, delays: Iterable[int] = (8, 16, 32),
                chunks: Optional[Iterable[int]] = None, precision: str = "fp32",
                reinv_period: int = 0, reinv_on_accepted: bool = False, warm_sweeps: int = 2,
                timed_sweeps: int = 1) -> Tuple[Tuple[int, int], Dict[Tuple[int, int], float]]:
    """Returns ((best k, best proposal batch), {(k, batch): device ms per sweep of the
    classes that depend on them}). Batches default to 2k, 4k and the whole spin block (0);
    a batch is always a multiple of k so that no window is cut short."""
    pos = inputs["pos"] if positions is None else positions
    times: Dict[Tuple[int, int], float] = {}
    for k in delays:
        cands = [2 * k, 4 * k, 0] if chunks is None else [c for c in chunks if c == 0 or c % k == 0]
        for c in dict.fromkeys(cands):
            times[(int(k), int(c))] = _time_sweeps(inputs, pos, precision, k, c, reinv_period,
                                                   reinv_on_accepted, warm_sweeps, timed_sweeps)
    best = min(times, key=times.get)
    return best, times
