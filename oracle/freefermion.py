"""Closed form for the Trotterised XX chain (TEST INFRASTRUCTURE ONLY).

At Delta = 0 the XXZ hopping S+S- + S-S+ (times 1/2) maps by Jordan-Wigner to
free fermions hopping with amplitude 1/2 between neighbours; a two-site gate
exp(-i tau h) is then exactly the single-particle 2x2 propagator
exp(-i tau sigma_x / 2) on rows (s, s+1).  The Trotterised evolution of a
product state stays Gaussian, so occupations and bond entropies follow from
the evolved orbitals alone.
"""
from __future__ import annotations

import numpy as np


def propagator(tau: float) -> np.ndarray:
    c, s = np.cos(0.5 * tau), np.sin(0.5 * tau)
    return np.array([[c, -1j * s], [-1j * s, c]])


class FreeFermions:
    def __init__(self, occupations):
        occ = list(occupations)
        self.L = len(occ)
        sites = [i for i, x in enumerate(occ) if x]
        self.phi = np.zeros((self.L, len(sites)), dtype=np.complex128)
        for a, i in enumerate(sites):
            self.phi[i, a] = 1.0

    def apply(self, s: int, tau: float) -> None:
        self.phi[s:s + 2, :] = propagator(tau) @ self.phi[s:s + 2, :]

    def densities(self) -> np.ndarray:
        return np.sum(np.abs(self.phi) ** 2, axis=1)

    def entropy(self, b: int) -> float:
        """Entropy of sites 0..b-1 from the correlation matrix restricted there."""
        C = self.phi @ self.phi.conj().T
        nu = np.linalg.eigvalsh(C[:b, :b])
        nu = np.clip(nu, 0.0, 1.0)
        s = 0.0
        for v in nu:
            for p in (v, 1.0 - v):
                if p > 1e-300:
                    s -= p * np.log(p)
        return float(s)
