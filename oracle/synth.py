"""Synthetic U(1) states for the oracle (TEST INFRASTRUCTURE ONLY).

A state with every inner bond at a given saturated sector structure and random
block entries: the sector dimensions spread chi over the charges of a bond in
proportion to the Hilbert-space bound of each charge (Sec. II: a sector of
bond k can be no larger than the number of configurations on either side).
Random numbers come from the shared seeded generators in `workloads`.
"""
from __future__ import annotations

import numpy as np

from .u1mps import U1MPS, bond_charge_range, hilbert_dim


def saturated_dims(L: int, d: int, N: int, b: int, chi: int) -> dict:
    lo, hi = bond_charge_range(L, d, N, b)
    h = {c: hilbert_dim(L, d, N, b, c) for c in range(lo, hi + 1)}
    h = {c: v for c, v in h.items() if v > 0}
    tot = sum(h.values())
    if tot <= chi:
        return h
    dims = {}
    for c, v in h.items():
        k = min(v, int(chi * v / tot))
        if k > 0:
            dims[c] = k
    if not dims:
        dims[max(h, key=h.get)] = 1
    return dims


def random_state(L: int, d: int, N: int, chi: int, seed: int, occ=None) -> U1MPS:
    """Every inner bond at saturated_dims(.., chi); random blocks and positive lambdas.

    The result is a valid U(1) block structure but not canonical; the two-site
    update is still well defined on it and costs what it costs at saturation.
    """
    import workloads as W
    rng = np.random.default_rng(seed)
    if occ is None:
        occ = W.random_occupations(L, d, N, rng)
    st = U1MPS.product(d, occ)
    for b in range(1, L):
        dims = saturated_dims(L, d, N, b, chi)
        st.bond[b] = dict(sorted(dims.items()))
        lam = W.random_positive(sum(dims.values()), rng)
        lam /= np.linalg.norm(lam)
        st.lam[b] = {}
        off = 0
        for c, D in st.bond[b].items():
            st.lam[b][c] = np.sort(lam[off:off + D])[::-1].copy()
            off += D
    for s in range(L):
        blocks = {}
        for l, Dl in st.bond[s].items():
            for m, Dm in st.bond[s + 1].items():
                if 0 <= l - m <= d - 1:
                    blocks[(l, m)] = W.random_complex((Dl, Dm), rng) / np.sqrt(max(Dl, Dm))
        st.B[s] = blocks
    return st
