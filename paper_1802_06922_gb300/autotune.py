"""Choice of the launch parameters of a sweep by measurement.

A larger delay rank k makes each move's window work (the d, z and x of the delayed update)
longer and each flush rarer; a smaller proposal batch (moves whose proposals and orbital
rows one launch pair forms) keeps those rows in L2 until the sweep reads them but adds
launches. The best pair depends on the system size, the walker count and the GPU, so
`tune_launch` times whole sweeps for every candidate pair on the caller's own inputs and
keeps the fastest (`tune_delay` does the same for k alone). A sweep is timed as it runs in
production, one CUDA-graph replay, by CUDA events on the launching stream, after warm-up
sweeps that capture its graphs. Neither parameter changes the Markov chain.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional, Tuple

from .qmcgb import Walkers, system_from_inputs


def _time_sweeps(inputs, pos, precision, k, chunk, reinv_period, reinv_on_accepted,
                 warm_sweeps, timed_sweeps) -> float:
    import torch
    s = system_from_inputs(inputs, precision=precision, delay_k=int(k), prop_chunk=int(chunk),
                           reinv_period=reinv_period, reinv_on_accepted=reinv_on_accepted)
    w = Walkers(s, pos)
    stream = torch.cuda.current_stream()
    try:
        w.sweep(warm_sweeps, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w.sweep(timed_sweeps, stream)
        e1.record(stream)
        e1.synchronize()
        w.check(stream)
        return e0.elapsed_time(e1) / timed_sweeps
    finally:
        w.close()
        s.close()


def tune_delay(inputs: dict, positions=None, candidates: Iterable[int] = (8, 16, 32),
               precision: str = "fp32", reinv_period: int = 0, reinv_on_accepted: bool = False,
               warm_sweeps: int = 3, timed_sweeps: int = 2) -> Tuple[int, Dict[int, float]]:
    """Returns (best k, {k: device ms per sweep}) with whole-block proposal batches.

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
                reinv_period: int = 0, reinv_on_accepted: bool = False, warm_sweeps: int = 3,
                timed_sweeps: int = 2) -> Tuple[Tuple[int, int], Dict[Tuple[int, int], float]]:
    """Returns ((best k, best proposal batch), {(k, batch): device ms per sweep}). Batches
    default to 2k, 4k and the whole spin block (0); a batch is always a multiple of k so
    that no window is cut short."""
    pos = inputs["pos"] if positions is None else positions
    times: Dict[Tuple[int, int], float] = {}
    for k in delays:
        cands = [2 * k, 4 * k, 0] if chunks is None else [c for c in chunks if c == 0 or c % k == 0]
        for c in dict.fromkeys(cands):
            times[(int(k), int(c))] = _time_sweeps(inputs, pos, precision, k, c, reinv_period,
                                                   reinv_on_accepted, warm_sweeps, timed_sweeps)
    best = min(times, key=times.get)
    return best, times
