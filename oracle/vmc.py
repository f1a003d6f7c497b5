"""Particle-by-particle VMC (and the drift-diffusion sweep used by DMC), move by move.

Sec. "Variational Monte Carlo" / "Trial Moves": electrons are visited one at a time; the
trial position of electron i is drawn from T(r -> r') (the particle-by-particle form of
Eq. trans_prob_alle) and accepted with A = min(1, |Psi(R')|^2 / |Psi(R)|^2 * T(R'->R) /
T(R->R')) (Eq. accept_reject). Sec. "Diffusion Monte Carlo": a DMC step moves every
electron by the drift-diffusion step of Eq. pmc:driftdiffusion_step and, under the fixed
node approximation, rejects any move that changes the sign of Psi.

Steps of one sweep t of one walker (the order is the paper's; the specific choices are
adopted readings):
 1. for e = 0 .. N_e - 1 (up block first): draw xi, u (``philox.move_draws``);
 2. Metropolis: r' = r_e + sigma xi.  Drift: r' = r_e + tau grad_e ln|Psi(R)| + sqrt(tau) xi
    (displacement tau * F/2 and variance tau: the standard Fokker-Planck form of
    Eq. pmc:driftdiffusion_step with lambda = 1/2); every component wrapped into [0, L);
 3. A' = A with row e replaced by phi(r'); R_det = det A' / det A from two LU
    factorisations (an exact zero pivot gives R_det = 0 and a rejection);
 4. dJ = J(R') - J(R), J(R') summed over all pairs;
 5. drift only: T(R'->R) / T(R->R') from the Gaussian densities, with grad ln|Psi(R')|
    from a fresh inverse of A';
 6. A = min(1, R_det^2 exp(2 dJ) T-ratio); DMC rejects when R_det < 0; accept iff u < A.
After the sweep: E_L and ln|Psi| of the final configuration.

Every move is recorded: R_det, dJ, grad_e ln|Psi(R')| (3), u, A, accepted.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from .jastrow import Jastrow, min_image
from .orbitals import PlaneWaveOrbitals, SplineOrbitals
from .philox import move_draws
from .wavefunction import SlaterJastrow

TRACE_FIELDS = ("ratio", "dJ", "gx", "gy", "gz", "u", "A", "accepted")


def drift_displacement(v, tau: float, a: float = 0.0):
    """Drift part of a drift-diffusion step for an electron whose drift velocity is
    v = grad_e ln|Psi| (3,).

    a = 0: the plain short-time step tau v (Eq. pmc:driftdiffusion_step, reading 1).
    a > 0: the drift rescaled near nodes of Psi following Umrigar, Nightingale and Runge
    (J. Chem. Phys. 99, 2865 (1993)), which Sec. "Projector Monte Carlo" and Sec. "Diffusion
    Monte Carlo" name without formulas: v is replaced by
        vbar = v (-1 + sqrt(1 + 2 a |v|^2 tau)) / (a |v|^2 tau),
    which tends to v where |v|^2 tau << 1 (far from a node) and keeps the displacement
    vbar tau below sqrt(2 tau / a) where |v| diverges (next to a node)."""
    v = np.asarray(v, dtype=np.float64)
    if a <= 0.0:
        return tau * v
    v2 = float(v @ v)
    x = 2.0 * a * v2 * tau
    if x < 1e-12:
        return tau * v
    # (-1 + sqrt(1 + x)) / (x / 2) written without the cancellation of -1 + sqrt(1 + x)
    return tau * v * 2.0 / (1.0 + np.sqrt(1.0 + x))


@dataclasses.dataclass
class Walker:
    R: np.ndarray              # (N_e, 3)
    wid: int
    A: list                    # Slater matrices per spin (N_s, N_s)
    logdet: list               # ln|det A| per spin
    sign: list                 # sign of det A per spin
    J: float


class OracleSystem:
    """The wavefunction and move parameters of one system built by ``synthetic``."""

    def __init__(self, inputs: dict, orbitals: str = "spline", coef=None, drift_a: float = 0.0):
        spec = inputs["spec"]
        self.spec = spec
        self.L = spec.L
        self.seed = int(inputs["seed"])
        if orbitals == "spline":
            orb = SplineOrbitals(inputs["coef"] if coef is None else coef, spec.L)
        else:
            orb = PlaneWaveOrbitals(inputs["nvec"], inputs["kind"], inputs["amp"], spec.L)
        jas = None
        if spec.jastrow_M > 0:
            j = inputs["jastrow"]
            jas = Jastrow(spec.L, spec.n_up, inputs["ions"], j["eI"], j["same"], j["opp"],
                          inputs["rcut"])
        self.wf = SlaterJastrow(orb, spec.n_up, spec.n_dn, jas, inputs["ions"], spec.ion_Z,
                                spec.kappa, spec.L, spec.with_potential)
        self.move = spec.move
        self.step = spec.step
        self.drift_a = float(drift_a)   # > 0: nodal drift rescaling (see drift_displacement)

    def walker(self, R, wid) -> Walker:
        R = np.mod(np.array(R, dtype=np.float64), self.L)
        A, ld, sg = [], [], []
        for spin in (0, 1):
            ns = self.spec.n_up if spin == 0 else self.spec.n_dn
            Am = self.wf.slater_matrix(R, spin) if ns else np.zeros((0, 0))
            s, l = np.linalg.slogdet(Am) if ns else (1.0, 0.0)
            A.append(Am)
            ld.append(float(l))
            sg.append(float(s))
        J = self.wf.jas.value(R) if self.wf.jas is not None else 0.0
        return Walker(R, int(wid), A, ld, sg, J)

    def log_psi(self, w: Walker) -> float:
        return float(w.logdet[0] + w.logdet[1] + w.J)

    # --------------------------------------------------------------------- sweep
    def sweep(self, w: Walker, t: int, fixed_node: bool = False,
              forced: Optional[np.ndarray] = None, trace: Optional[list] = None,
              electrons=None, conds: Optional[list] = None,
              r2: Optional[list] = None) -> None:
        """One sweep t of walker w, in place. ``forced`` (N_e bools) replaces the
        acceptance decisions (lockstep replay); ``trace`` collects one row per move;
        ``conds`` (a diagnostic for the tests' error bounds, no effect on the chain)
        collects max(cond_2(A), cond_2(A')) of the moved spin block per move; ``r2``, a
        two-element list, accumulates the squared proposed displacements |r' - r|^2 of all
        moves and of the accepted ones (the effective time step of a DMC step)."""
        wf, L = self.wf, self.L
        ne = w.R.shape[0]
        drift = self.move == "drift"
        tau = sigma = self.step
        for e in (range(ne) if electrons is None else electrons):
            xi, u = move_draws(self.seed, t, e, w.wid)
            spin, first, ns = wf.block(e)
            row = e - first
            r_old = w.R[e].copy()
            if drift:
                g_old = wf.grad_log_psi(w.R, e, np.linalg.inv(w.A[spin]))
                r_new = r_old + drift_displacement(g_old, tau, self.drift_a) + np.sqrt(tau) * xi
            else:
                r_new = r_old + sigma * xi
            r_new = np.mod(r_new, L)
            A_new = w.A[spin].copy()
            A_new[row] = wf.orb.values(r_new)[:ns]
            s_new, ld_new = np.linalg.slogdet(A_new)
            R_new = w.R.copy()
            R_new[e] = r_new
            if s_new == 0.0:
                ratio = 0.0
                g_new = np.zeros(3)
            else:
                ratio = s_new * w.sign[spin] * np.exp(ld_new - w.logdet[spin])
                g_new = wf.grad_log_psi(R_new, e, np.linalg.inv(A_new))
            if conds is not None:
                conds.append(max(np.linalg.cond(w.A[spin]), np.linalg.cond(A_new)))
            J_new = wf.jas.value(R_new) if wf.jas is not None else 0.0
            dJ = J_new - w.J
            t_ratio = 1.0
            d = min_image(r_new - r_old, L)
            if drift:
                fwd = d - drift_displacement(g_old, tau, self.drift_a)
                rev = -d - drift_displacement(g_new, tau, self.drift_a)
                t_ratio = np.exp((fwd @ fwd - rev @ rev) / (2.0 * tau))
            acc_prob = min(1.0, ratio * ratio * np.exp(2.0 * dJ) * t_ratio) if ratio != 0 else 0.0
            accept = bool(u < acc_prob)
            if fixed_node and ratio < 0.0:
                accept = False
            if forced is not None:
                accept = bool(forced[e])
            if trace is not None:
                trace.append((ratio, dJ, g_new[0], g_new[1], g_new[2], u, acc_prob,
                              float(accept)))
            if r2 is not None:
                r2[0] += float(d @ d)
                if accept:
                    r2[1] += float(d @ d)
            if accept:
                w.R[e] = r_new
                w.A[spin] = A_new
                w.logdet[spin] = float(ld_new)
                w.sign[spin] = float(s_new)
                w.J = J_new

    def measure(self, w: Walker):
        """(E_L, kinetic energy, ln|Psi|) of the walker's current configuration."""
        e, kin = self.wf.local_energy(w.R)
        return e, kin, self.log_psi(w)


def run_vmc(system: OracleSystem, positions, walker_ids, n_sweeps: int, first_sweep: int = 0,
            forced=None, conds: Optional[np.ndarray] = None):
    """Run n_sweeps of every walker. Returns (walkers, trace [n_w][sweeps*N_e][8],
    energies [n_w][sweeps][3] = (E_L, kinetic, ln|Psi|)). ``conds``, if given, is filled
    with the per-move condition numbers of ``OracleSystem.sweep`` ([n_w][sweeps*N_e])."""
    walkers = [system.walker(R, wid) for R, wid in zip(positions, walker_ids)]
    ne = system.spec.n_elec
    tr = np.zeros((len(walkers), n_sweeps * ne, len(TRACE_FIELDS)))
    en = np.zeros((len(walkers), n_sweeps, 3))
    for k, w in enumerate(walkers):
        for s in range(n_sweeps):
            rows: List = []
            cl = [] if conds is not None else None
            fb = None if forced is None else forced[k][s * ne:(s + 1) * ne]
            system.sweep(w, first_sweep + s, fixed_node=False, forced=fb, trace=rows, conds=cl)
            tr[k, s * ne:(s + 1) * ne] = np.array(rows)
            if conds is not None:
                conds[k, s * ne:(s + 1) * ne] = cl
            en[k, s] = system.measure(w)
    return walkers, tr, en
