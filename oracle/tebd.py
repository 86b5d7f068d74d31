"""TEBD schedules and model drivers for the oracle (TEST INFRASTRUCTURE ONLY).

The paper cites TEBD (Sec. I) without giving its schedule; the reading used
here is second-order Strang splitting per time step, with no merging of
adjacent half steps: odd bonds (0-based left sites 0, 2, 4, ...) for dt/2,
even bonds (1, 3, 5, ...) for dt, odd bonds again for dt/2.
"""
from __future__ import annotations

import numpy as np

from . import gates
from .u1mps import U1MPS


def strang_layers(L: int):
    odd = list(range(0, L - 1, 2))
    even = list(range(1, L - 1, 2))
    return [(odd, 0.5), (even, 1.0), (odd, 0.5)]


def xxz_gates(L: int, delta: float, dt: float):
    """Gate blocks per (left site, dt factor) of the XXZ chain (uniform bonds)."""
    half = gates.xxz_gate(delta, 0.5 * dt)
    full = gates.xxz_gate(delta, dt)
    return lambda s, f: half if f == 0.5 else full


def bh_gates(L: int, d: int, J: float, U: float, dt: float):
    cache = {}

    def get(s, f):
        key = (gates.bh_weights(L, s), f)
        if key not in cache:
            cache[key] = gates.bh_gate(L, s, d, J, U, f * dt)
        return cache[key]
    return get


def run_tebd(state: U1MPS, gate_of, n_steps: int, chi: int, cutoff: float, observe=None):
    """Evolve in place; returns the list of per-update info dicts."""
    infos = []
    for step in range(n_steps):
        for sites, f in strang_layers(state.L):
            for s in sites:
                infos.append(state.apply_gate2(s, gate_of(s, f), chi, cutoff))
        if observe is not None:
            observe(step, state)
    return infos


def run_brickwork(state: U1MPS, layers, angles, chi: int, cutoff: float):
    """Apply beam splitters layer by layer; angles are consumed in gate order."""
    infos = []
    k = 0
    for sites in layers:
        for s in sites:
            th, ph = angles[k]
            k += 1
            infos.append(state.apply_gate2(s, gates.beam_splitter_gate(th, ph, state.d), chi, cutoff))
    return infos


def interferometer(M: int, layers, angles) -> np.ndarray:
    """M x M mode matrix of the brickwork: product of embedded 2x2 u's in gate order."""
    U = np.eye(M, dtype=np.complex128)
    k = 0
    for sites in layers:
        for s in sites:
            th, ph = angles[k]
            k += 1
            E = np.eye(M, dtype=np.complex128)
            E[s:s + 2, s:s + 2] = gates.beam_splitter_u(th, ph)
            U = E @ U
    return U
