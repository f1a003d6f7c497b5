"""Timing harness of the oracle on the host cores (the bench's CPU-baseline leg and its
reference arm). TEST INFRASTRUCTURE: it only times the oracle as it stands.

Workers are started with the ``spawn`` method, one process per core, each single-threaded
(BLAS threads pinned to 1 through the environment inherited from the parent); each worker
builds the system once and then times particle-by-particle moves of its walkers.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

_STATE = {}


def _init(preset: str, seed: int):
    from synthetic import build_inputs, spec_for
    from oracle.vmc import OracleSystem
    inputs = build_inputs(spec_for(preset), seed=seed, n_walkers=None)
    _STATE["sys"] = OracleSystem(inputs)
    _STATE["pos"] = inputs["pos"]


def _moves(task):
    walker, e0, n_moves, sweep = task
    sysm = _STATE["sys"]
    w = sysm.walker(_STATE["pos"][walker % len(_STATE["pos"])], walker)
    ne = sysm.spec.n_elec
    t0 = time.perf_counter()
    sysm.sweep(w, sweep, electrons=[(e0 + i) % ne for i in range(n_moves)])
    return n_moves, time.perf_counter() - t0


class OraclePool:
    """A pool of single-threaded oracle processes for one preset."""

    def __init__(self, preset: str, cores: int, seed: int = 0):
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(cores, initializer=_init, initargs=(preset, seed))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.cores = cores
        # make sure every worker finished building the system before anything is timed
        seen, t0 = set(), time.perf_counter()
        while len(seen) < cores and time.perf_counter() - t0 < 600:
            seen.update(self.pool.map(_pid, range(cores * 2), chunksize=1))

    def run(self, walkers, e0: int, n_moves: int, sweep: int = 0):
        """Time n_moves moves of each walker; returns (moves, wall seconds)."""
        tasks = [(w, e0, n_moves, sweep) for w in walkers]
        t0 = time.perf_counter()
        res = self.pool.map(_moves, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        return sum(r[0] for r in res), wall

    def close(self):
        self.pool.terminate()
        self.pool.join()


def _pid(_):
    time.sleep(0.02)
    return os.getpid()
