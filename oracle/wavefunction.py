"""Slater-Jastrow trial wavefunction, its log-derivatives and the local energy.

Eq. msdj with one determinant pair: Psi = D_up D_dn e^{J}. The Slater matrix of a spin
block has one row per electron, A[e][j] = phi_j(r_e) for orbitals j = 0..N_s-1 (the
convention stated in Sec. "Backflow"). Determinants are taken by LU with partial
pivoting (numpy.linalg.slogdet, LAPACK getrf) and inverses by numpy.linalg.inv.

Local energy (Sec. "Quantum Monte Carlo"; E_L = Psi^-1 H Psi, Sec. "Hamiltonian"):
    T_L = -1/2 sum_i [ lap_i ln Psi + |grad_i ln Psi|^2 ]
with grad_i ln D = sum_j grad phi_j(r_i) Ainv[j][i] and
lap_i ln D = sum_j lap phi_j(r_i) Ainv[j][i] - |grad_i ln D|^2; the potential is the
short-range Yukawa stand-in of ``hamiltonian.py``.

Pins: the determinant ratio against the Leibniz permutation expansion on tiny matrices;
grad and lap of ln|Psi| against central finite differences of ln|Psi|; the zero-variance
kinetic energy sum_j |k_j|^2 / 2 of a plane-wave determinant.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import yukawa_potential


class SlaterJastrow:
    def __init__(self, orbitals, n_up, n_dn, jastrow=None, ions=None, ion_Z=0.0,
                 kappa=1.0, L=None, with_potential=True):
        self.orb = orbitals
        self.n_up, self.n_dn = int(n_up), int(n_dn)
        self.jas = jastrow
        self.ions = np.zeros((0, 3)) if ions is None else np.asarray(ions, float)
        self.Z = float(ion_Z)
        self.kappa = float(kappa)
        self.L = float(orbitals.L if L is None else L)
        self.with_potential = with_potential

    # ---------------------------------------------------------------- spin blocks
    def block(self, e):
        """(spin, first electron of the block, N_s) of electron e."""
        if e < self.n_up:
            return 0, 0, self.n_up
        return 1, self.n_up, self.n_dn

    def slater_matrix(self, R, spin):
        first, ns = (0, self.n_up) if spin == 0 else (self.n_up, self.n_dn)
        return np.array([self.orb.values(R[first + i])[:ns] for i in range(ns)])

    # ---------------------------------------------------------------- ln |Psi|
    def log_psi(self, R):
        """(ln|Psi|, sign of Psi)."""
        logv, sign = 0.0, 1.0
        for spin in (0, 1):
            ns = self.n_up if spin == 0 else self.n_dn
            if ns == 0:
                continue
            s, ld = np.linalg.slogdet(self.slater_matrix(R, spin))
            logv += ld
            sign *= s
        if self.jas is not None:
            logv += self.jas.value(R)
        return float(logv), float(sign)

    def grad_lap_log_det(self, R, i, Ainv=None):
        """grad_i ln|D| (3,) and lap_i ln|D| for electron i, from a fresh inverse."""
        spin, first, ns = self.block(i)
        if Ainv is None:
            Ainv = np.linalg.inv(self.slater_matrix(R, spin))
        _, grad, lap = self.orb.vgl(R[i])
        col = Ainv[:, i - first]
        g = grad[:, :ns] @ col
        return g, float(lap[:ns] @ col - g @ g)

    def grad_log_psi(self, R, i, Ainv=None):
        g, _ = self.grad_lap_log_det(R, i, Ainv)
        if self.jas is not None:
            g = g + self.jas.grad_lap(R, i)[0]
        return g

    def local_energy(self, R):
        """(E_L, kinetic part) of configuration R."""
        R = np.asarray(R, dtype=np.float64)
        inv = {}
        for spin in (0, 1):
            ns = self.n_up if spin == 0 else self.n_dn
            if ns:
                inv[spin] = np.linalg.inv(self.slater_matrix(R, spin))
        kin = 0.0
        for i in range(R.shape[0]):
            spin, _, _ = self.block(i)
            g, lap = self.grad_lap_log_det(R, i, inv[spin])
            if self.jas is not None:
                gj, lj = self.jas.grad_lap(R, i)
                g = g + gj
                lap = lap + lj
            kin += -0.5 * (lap + g @ g)
        pot = 0.0
        if self.with_potential:
            pot = yukawa_potential(R, self.ions, self.Z, self.kappa, self.L)
        return float(kin + pot), float(kin)
