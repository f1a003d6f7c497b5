"""Branching DMC step with a variable walker count.

Sec. "Projector Monte Carlo" and "Diffusion Monte Carlo": after the drift-diffusion
sweep (fixed-node rule: a move that changes the sign of Psi is rejected) each walker's
weight is multiplied by the branching Green's function of Eq. pmc:g_growth,
    w <- w exp(-1/2 (E_L(R_old) + E_L(R_new) - 2 E_T) tau)        (Eq. pmc:walker_weight),
averages are weighted (Eq. pmc:weighted_average), and the walker is replaced by
M = INT(w + xi) copies with xi uniform in (0, 1); M = 0 removes it.

Adopted readings (the paper leaves them open, so no value of the paper can pin them; the
tests pin the invariants any population control must keep: an exact fixed point when E_T
equals a constant E_L at the target population, a negative feedback that returns an
off-target population to the target, and unique walker IDs under branching):
* copies are renormalised to weight 1;
* the first copy keeps the parent's walker ID and every further copy takes the next
  value of a per-system counter, copies being appended in parent order;
* the population is capped at ``capacity`` walkers (copies beyond it are dropped);
* E_T <- E_w - ln(N_w / N_target) / (10 tau), E_w being this step's weighted mean E_L
  (population control by trial-energy feedback, Sec. "Diffusion Monte Carlo").

Pins: with E_L constant (plane-wave determinant without Jastrow or potential) every
weight equals exp(-tau (E - E_T)) exactly; the invariants above.
"""
from __future__ import annotations

import copy
import math
from typing import List

import numpy as np

from .philox import branch_draw


class DMCPopulation:
    def __init__(self, system, positions, walker_ids, E_T: float, capacity: int):
        self.sys = system
        self.walkers = [system.walker(R, wid) for R, wid in zip(positions, walker_ids)]
        self.E_L = np.array([system.measure(w)[0] for w in self.walkers])
        self.n_target = len(self.walkers)
        self.next_id = int(max(walker_ids)) + 1 if len(walker_ids) else 0
        self.E_T = float(E_T)
        self.capacity = int(capacity)

    def step(self, t: int, trace=None):
        """One DMC step t. Returns (sum of weights, weighted mean E_L, walkers after)."""
        tau = self.sys.step
        w_new, e_new = [], []
        for k, w in enumerate(self.walkers):
            rows = [] if trace is not None else None
            self.sys.sweep(w, t, fixed_node=True, trace=rows)
            if trace is not None:
                trace.append((w.wid, np.array(rows)))
            e = self.sys.measure(w)[0]
            weight = math.exp(-0.5 * (self.E_L[k] + e - 2.0 * self.E_T) * tau)
            w_new.append(weight)
            e_new.append(e)
        w_new = np.array(w_new)
        e_new = np.array(e_new)
        sum_w = float(w_new.sum())
        e_mean = float((w_new * e_new).sum() / sum_w)
        walkers, energies = [], []
        for k, w in enumerate(self.walkers):
            m = int(math.floor(w_new[k] + branch_draw(self.sys.seed, t, w.wid)))
            for c in range(m):
                if len(walkers) >= self.capacity:
                    break
                child = w if c == 0 else copy.deepcopy(w)
                if c > 0:
                    child.wid = self.next_id
                    self.next_id += 1
                walkers.append(child)
                energies.append(e_new[k])
        self.walkers = walkers
        self.E_L = np.array(energies)
        n = max(len(walkers), 1)
        self.E_T = e_mean - math.log(n / self.n_target) / (10.0 * tau)
        return sum_w, e_mean, w_new
