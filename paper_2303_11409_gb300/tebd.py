"""TEBD drivers on the GPU library: one launch set per Trotter layer.

Second-order Strang splitting per time step (odd bonds dt/2, even bonds dt,
odd bonds dt/2; left sites 0, 2, 4, ... are the odd bonds).  All bonds of a
layer touch disjoint tensors and go to the library as one mps_apply_layer call
(independent two-site updates processed in parallel, arXiv:2303.11409 Sec. II).
"""
from __future__ import annotations

import numpy as np

from . import models
from ._binding import MPS


def strang_layers(L: int):
    odd = list(range(0, L - 1, 2))
    even = list(range(1, L - 1, 2))
    return [(odd, 0.5), (even, 1.0), (odd, 0.5)]


class GateTable:
    """Flattened gate blocks per (left site, dt factor), built once per workload."""

    def __init__(self, model: str, L: int, d: int, dt: float, **p):
        self.model, self.L, self.d, self.dt, self.p = model, L, d, dt, p
        self._cache = {}

    def __call__(self, s: int, f: float) -> np.ndarray:
        if self.model == "xxz":
            key = f
        else:
            key = (models.bose_hubbard_weights(self.L, s), f)
        g = self._cache.get(key)
        if g is None:
            tau = f * self.dt
            if self.model == "xxz":
                blocks = models.xxz_gate(self.p["delta"], tau, self.p.get("J", 1.0))
            elif self.model == "clock":
                wl, wr = models.bose_hubbard_weights(self.L, s)
                blocks = models.clock_gate(self.d, self.p.get("J", 1.0), self.p["f"], tau, wl, wr)
            elif self.model == "bh":
                wl, wr = models.bose_hubbard_weights(self.L, s)
                blocks = models.bose_hubbard_gate(self.d, self.p.get("J", 1.0), self.p["U"], tau, wl, wr)
            else:
                raise ValueError(self.model)
            if self.p.get("zn") and self.model != "clock":   # a U(1) model on a Z_n handle (d < n)
                blocks = models.cyclic_blocks(blocks, self.d, int(self.p["zn"]))
            g = models.flatten(blocks)
            self._cache[key] = g
        return g


def trotter_step(psi: MPS, gates: GateTable, chi: int, cutoff: float) -> list[np.ndarray]:
    errs = []
    for sites, f in strang_layers(psi.L):
        errs.append(psi.apply_layer(sites, [gates(s, f) for s in sites], chi, cutoff))
    return errs


def brickwork(psi: MPS, layers, angles, chi: int, cutoff: float):
    k = 0
    errs = []
    for sites in layers:
        gs = []
        for _ in sites:
            th, ph = angles[k]
            k += 1
            gs.append(models.flatten(models.beam_splitter_gate(th, ph, psi.d)))
        errs.append(psi.apply_layer(sites, gs, chi, cutoff))
    return errs
