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

Two refinements of the full DMC driver (Sec. "Diffusion Monte Carlo", last paragraphs,
and Sec. "Projector Monte Carlo"), which the paper names but does not spell out; both are
restated from the cited methods, the specific choices being adopted readings:
* effective time step (Umrigar, Nightingale and Runge, J. Chem. Phys. 99, 2865 (1993)):
  the branching factor of a walker uses tau_eff = tau * sum(accepted |dr|^2) / sum(|dr|^2)
  over the moves of its sweep (dr the proposed displacement), which accounts for the
  diffusion lost to rejected moves; tau_eff = tau when every move is accepted. (The nodal
  drift rescaling of the same paper is ``vmc.drift_displacement``.)
* stochastic reconfiguration at a fixed walker count (Assaraf, Caffarel and Khelif, Phys.
  Rev. E 61, 4566 (2000)): instead of M = INT(w + xi) independent copies, the N walkers are
  resampled with one comb of N teeth at (k + xi) W / N, k = 0..N-1, over their cumulative
  weights (W the total weight, xi one uniform draw per step, ``philox.comb_draw``); walker
  i receives as many copies as teeth fall in its interval, so N is kept exactly, every
  walker's expected copy count is N w_i / W and each count is its floor or ceiling; the
  copies carry weight one, and the step's mean weight W / N enters the estimators (the
  weighted mean E_L of the step uses the weights before resampling, as with branching).

Pins: with E_L constant (plane-wave determinant without Jastrow or potential) every
weight equals exp(-tau (E - E_T)) exactly; the invariants above; tau_eff = tau when every
move is accepted and 0 when none is; the reconfiguration keeps N and the total weight,
gives every walker the floor or the ceiling of N w_i / W copies and is unbiased.
"""
from __future__ import annotations

import copy
import math
from typing import List

import numpy as np

from .philox import branch_draw, comb_draw


def comb_counts(weights, xi: float):
    """Copy counts of a stochastic reconfiguration: a comb of N = len(weights) teeth at
    (k + xi) W / N, k = 0..N-1, over the cumulative weights (summed left to right); walker i
    gets the number of teeth in [C_{i-1}, C_i)."""
    w = np.asarray(weights, dtype=np.float64)
    n = w.size
    W = float(w.sum())

    def teeth_below(c):      # #{k in [0, N): (k + xi) W / N < c}
        return min(n, max(0, math.ceil(c * n / W - xi)))

    counts = np.zeros(n, dtype=np.int64)
    prev, cum = 0, 0.0
    for i in range(n):
        cum += w[i]
        t = teeth_below(cum) if i < n - 1 else n
        counts[i] = t - prev
        prev = t
    return counts


class DMCPopulation:
    def __init__(self, system, positions, walker_ids, E_T: float, capacity: int,
                 tau_eff: bool = False, reconfigure: bool = False):
        self.sys = system
        self.walkers = [system.walker(R, wid) for R, wid in zip(positions, walker_ids)]
        self.E_L = np.array([system.measure(w)[0] for w in self.walkers])
        self.n_target = len(self.walkers)
        self.next_id = int(max(walker_ids)) + 1 if len(walker_ids) else 0
        self.E_T = float(E_T)
        self.capacity = int(capacity)
        self.tau_eff = bool(tau_eff)
        self.reconfigure = bool(reconfigure)
        self.last_tau_eff = None

    def step(self, t: int, trace=None):
        """One DMC step t. Returns (sum of weights, weighted mean E_L, walkers after)."""
        tau = self.sys.step
        w_new, e_new, taus = [], [], []
        for k, w in enumerate(self.walkers):
            rows = [] if trace is not None else None
            r2 = [0.0, 0.0]
            self.sys.sweep(w, t, fixed_node=True, trace=rows, r2=r2)
            if trace is not None:
                trace.append((w.wid, np.array(rows)))
            e = self.sys.measure(w)[0]
            te = tau
            if self.tau_eff:
                te = tau * r2[1] / r2[0] if r2[0] > 0.0 else 0.0
            taus.append(te)
            weight = math.exp(-0.5 * (self.E_L[k] + e - 2.0 * self.E_T) * te)
            w_new.append(weight)
            e_new.append(e)
        w_new = np.array(w_new)
        e_new = np.array(e_new)
        self.last_tau_eff = np.array(taus)
        sum_w = float(w_new.sum())
        e_mean = float((w_new * e_new).sum() / sum_w)
        walkers, energies = [], []
        counts = comb_counts(w_new, comb_draw(self.sys.seed, t)) if self.reconfigure else None
        for k, w in enumerate(self.walkers):
            if counts is not None:
                m = int(counts[k])
            else:
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
