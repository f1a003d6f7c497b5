"""Choice of the delay rank k of the delayed inverse update by measurement.

A larger k makes each move's window work (the d, z and x of the delayed update) longer and
each flush rarer, so the best k depends on the system size, the walker count and the GPU.
`tune_delay` times a few sweeps for every candidate on the caller's own inputs and keeps the
fastest. Timing uses the library's per-kernel device-time profiling (`qmc_profile_read`);
the classes whose cost does not depend on k (re-inversion, local energy) are left out of the
ranking.
"""
from __future__ import annotations

from typing import Iterable, Tuple, Dict

from .qmcgb import KERNEL_CLASSES, Walkers, system_from_inputs

# kernel classes whose device time changes with the delay rank
_K_DEPENDENT = ("propose", "vgl", "sweep", "flush")


def tune_delay(inputs: dict, positions=None, candidates: Iterable[int] = (8, 16, 32),
               precision: str = "fp32", reinv_period: int = 0, reinv_on_accepted: bool = False,
               warm_sweeps: int = 2, timed_sweeps: int = 1) -> Tuple[int, Dict[int, float]]:
    """Returns (best k, {k: device ms per sweep of the k-dependent kernels}).

    `inputs` is a ``synthetic.build_inputs``-style dictionary; `positions` (host array
    [n_walkers][n_elec][3]) defaults to ``inputs["pos"]``.
    """
    pos = inputs["pos"] if positions is None else positions
    idx = [KERNEL_CLASSES.index(c) for c in _K_DEPENDENT]
    times: Dict[int, float] = {}
    for k in candidates:
        s = system_from_inputs(inputs, precision=precision, delay_k=int(k),
                               reinv_period=reinv_period, reinv_on_accepted=reinv_on_accepted)
        w = Walkers(s, pos)
        try:
            w.sweep(warm_sweeps)
            w.profile(True)
            w.sweep(timed_sweeps)
            ms, _ = w.profile_read()
            times[int(k)] = float(sum(ms[i] for i in idx)) / timed_sweeps
        finally:
            w.close()
            s.close()
    best = min(times, key=times.get)
    return best, times
