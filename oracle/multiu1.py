"""Float64 CPU oracle of the two-site TEBD update with several U(1) charges (tuple charges).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import it; the library never does, and this module
imports nothing from the library.

Sec. I names "more general Abelian" symmetries beside U(1); this is the U(1) x ... x U(1)
case.  Every physical index i carries a charge vector q_i (distinct vectors), a bond
carries the vector sum of the charges to its right, and the Kronecker deltas of Sec. II
become vector equalities: block (l, m) of a site exists iff l - m = q_i for some i.  A
two-site gate conserving every charge is block diagonal in the pair's total Q = q_i + q_j;
block Q acts on the pairs (i, j) with q_i + q_j = Q, i ascending (rows outputs).

The update is the one of u1mps.py with vector charges: Theta(c) for each candidate middle
charge c has as rows the left sectors l with l - c a physical charge and as columns the
right sectors r with c - r a physical charge, both in ascending (lexicographic) charge
order; one SVD per Theta(c); the global truncation, tie rule and noise floor of
u1mps.select_kept with charges compared lexicographically; the inverse-free reassembly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .u1mps import NOISE_REL, SectorPlan, select_kept


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def pair_blocks(q):
    """Two-site charge blocks: sorted totals Q, and for each the pairs (i, j), i ascending."""
    d = len(q)
    tot = {}
    for i in range(d):
        for j in range(d):
            tot.setdefault(_add(q[i], q[j]), []).append((i, j))
    keys = sorted(tot)
    return keys, {Q: sorted(tot[Q]) for Q in keys}


def phys_index(q, l, m) -> int:
    """The physical index i with q_i = l - m (the vector Kronecker delta of Sec. II), or -1."""
    dq = _sub(l, m)
    for i, x in enumerate(q):
        if x == dq:
            return i
    return -1


def plan_update(left: dict, mid: dict, right: dict, q) -> SectorPlan:
    """The sector structure of a two-site update with charge vectors q_i, by looping over charges.

    triples: (l, m, r) with l - m and m - r physical charges, lexicographic; sectors: every middle
    charge c = l - q_i that some right r reaches with c - r a physical charge; rows of Theta(c):
    the left l with l - c a physical charge, columns: the right r with c - r one, ascending.
    """
    triples = [(l, m, r) for l in sorted(left) for m in sorted(mid) if phys_index(q, l, m) >= 0
               for r in sorted(right) if phys_index(q, m, r) >= 0]
    cands = set()
    for l in left:
        for r in right:
            for x in q:
                c = _sub(l, x)
                if phys_index(q, c, r) >= 0:
                    cands.add(c)
    sectors = sorted(cands)
    rows = {c: [l for l in sorted(left) if phys_index(q, l, c) >= 0] for c in sectors}
    cols = {c: [r for r in sorted(right) if phys_index(q, c, r) >= 0] for c in sectors}
    return SectorPlan(triples, sectors, rows, cols)


@dataclass
class MultiU1MPS:
    """Right-canonical MPS with tuple charges: bond[b] charge -> dim, lam[b], B[s][(l, m)]."""
    L: int
    q: list
    N: tuple
    bond: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    B: list = field(default_factory=list)

    @classmethod
    def product(cls, q, occupations) -> "MultiU1MPS":
        q = [tuple(int(v) for v in x) for x in q]
        if len(set(q)) != len(q):
            raise ValueError("physical charges must be distinct")
        occ = [int(x) for x in occupations]
        L = len(occ)
        zero = tuple(0 for _ in q[0])
        c = [zero] * (L + 1)
        for b in range(L - 1, -1, -1):
            c[b] = _add(c[b + 1], q[occ[b]])
        st = cls(L, q, c[0])
        st.bond = [{c[b]: 1} for b in range(L + 1)]
        st.lam = [{c[b]: np.ones(1)} for b in range(L + 1)]
        st.B = [{(c[s], c[s + 1]): np.ones((1, 1), dtype=np.complex128)} for s in range(L)]
        return st

    def phys(self, l, m):
        return phys_index(self.q, l, m)

    def apply_gate2(self, s: int, G: dict, chi: int, cutoff: float) -> dict:
        """G[Q]: the gate block of total charge Q over pair_blocks(q)[1][Q]."""
        left, mid, right = self.bond[s], self.bond[s + 1], self.bond[s + 2]
        BL, BR = self.B[s], self.B[s + 1]
        _, pairs = pair_blocks(self.q)
        plan = plan_update(left, mid, right, self.q)
        sectors, rows, cols = plan.sectors, plan.rows, plan.cols
        theta = {}
        for c in sectors:
            T = np.zeros((sum(left[l] for l in rows[c]), sum(right[r] for r in cols[c])), dtype=np.complex128)
            ro = 0
            for l in rows[c]:
                co = 0
                ip = self.phys(l, c)
                for r in cols[c]:
                    Q = _sub(l, r)
                    idx = [p[0] for p in pairs[Q]]
                    blk = T[ro:ro + left[l], co:co + right[r]]
                    for m in sorted(mid):
                        i, j = self.phys(l, m), self.phys(m, r)
                        if i < 0 or j < 0:
                            continue
                        g = G[Q][idx.index(ip), idx.index(i)]
                        if g != 0:
                            blk += g * (BL[(l, m)] @ BR[(m, r)])
                    co += right[r]
                ro += left[l]
            theta[c] = T
        svals, vecs = {}, {}
        for c in sectors:
            lam_rows = np.concatenate([self.lam[s][l] for l in rows[c]])
            M = lam_rows[:, None] * theta[c]
            _, S, Yh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
            S = np.where(S <= NOISE_REL * math.sqrt(float(np.sum(S * S))), 0.0, S)
            svals[c], vecs[c] = S, Yh
        kept, info = select_kept(svals, chi, cutoff)
        nk = info["kept_norm"]
        new_mid, new_lam, nBL, nBR = {}, {}, {}, {}
        for c in sectors:
            k = kept[c]
            if k == 0:
                continue
            new_mid[c] = k
            new_lam[c] = svals[c][:k] / nk
            Yh = vecs[c][:k, :]
            lp = (theta[c] @ Yh.conj().T) / nk
            ro = 0
            for l in rows[c]:
                nBL[(l, c)] = lp[ro:ro + left[l], :].copy()
                ro += left[l]
            co = 0
            for r in cols[c]:
                nBR[(c, r)] = Yh[:, co:co + right[r]].copy()
                co += right[r]
        self.bond[s + 1], self.lam[s + 1], self.B[s], self.B[s + 1] = new_mid, new_lam, nBL, nBR
        info["kept"] = {c: k for c, k in kept.items() if k}
        return info

    def expect_local(self, s: int, diag_op) -> float:
        val = 0.0
        for (l, m), blk in self.B[s].items():
            w = self.lam[s][l] ** 2
            val += float(diag_op[self.phys(l, m)]) * float(np.sum(w[:, None] * np.abs(blk) ** 2))
        return val

    def entropy(self, b: int) -> float:
        p = np.concatenate([v ** 2 for v in self.lam[b].values()])
        p = p[p > 0]
        return float(-np.sum(p * np.log(p)))

    def amplitude(self, config) -> complex:
        cfg = [int(x) for x in config]
        zero = tuple(0 for _ in self.q[0])
        c = [zero] * (self.L + 1)
        for b in range(self.L - 1, -1, -1):
            c[b] = _add(c[b + 1], self.q[cfg[b]])
        if c[0] != self.N:
            return 0j
        v = np.ones((1, 1), dtype=np.complex128)
        for s in range(self.L):
            blk = self.B[s].get((c[s], c[s + 1]))
            if blk is None:
                return 0j
            v = v @ blk
        return complex(v[0, 0])

    def check_structure(self) -> None:
        for s in range(self.L):
            for (l, m), blk in self.B[s].items():
                assert self.phys(l, m) >= 0, (s, l, m)
                assert blk.shape == (self.bond[s][l], self.bond[s + 1][m])


# ---------------------------------------------------------------------------
# Two-species hard-core bosons: q = (n_up, n_down), index i = 2 n_up + n_down
# ---------------------------------------------------------------------------
TWO_SPECIES_Q = [(0, 0), (0, 1), (1, 0), (1, 1)]


def two_species_h(J: float, U: float, w_left: float, w_right: float) -> np.ndarray:
    """16 x 16 matrix <i' j'|h|i j> (index 4 i + j) of -J sum_s (b1s^dag b2s + h.c.) + U (w1 n1u n1d + w2 n2u n2d)."""
    H = np.zeros((16, 16))
    for i in range(4):
        for j in range(4):
            ui, di = TWO_SPECIES_Q[i]
            uj, dj = TWO_SPECIES_Q[j]
            H[4 * i + j, 4 * i + j] = U * (w_left * ui * di + w_right * uj * dj)
            for sp in (0, 1):                  # species 0 = up, 1 = down
                a, b = list(TWO_SPECIES_Q[i]), list(TWO_SPECIES_Q[j])
                if a[sp] == 0 and b[sp] == 1:  # b1^dag b2: the particle hops left
                    a2, b2 = a.copy(), b.copy()
                    a2[sp], b2[sp] = 1, 0
                    i2, j2 = TWO_SPECIES_Q.index(tuple(a2)), TWO_SPECIES_Q.index(tuple(b2))
                    H[4 * i2 + j2, 4 * i + j] += -J
                    H[4 * i + j, 4 * i2 + j2] += -J
    return H


def gate_blocks_from_matrix(G: np.ndarray, q) -> dict:
    """Charge blocks of a two-site matrix (index i d + j) that conserves every charge."""
    d = len(q)
    keys, pairs = pair_blocks(q)
    out = {}
    for Q in keys:
        pl = pairs[Q]
        out[Q] = np.array([[G[a * d + b, c * d + e] for (c, e) in pl] for (a, b) in pl], dtype=np.complex128)
    return out


def two_species_gate(J: float, U: float, w_left: float, w_right: float, tau: float) -> dict:
    h = two_species_h(J, U, w_left, w_right)
    w, v = np.linalg.eigh(h)
    G = (v * np.exp(-1j * w * tau)) @ v.conj().T
    return gate_blocks_from_matrix(G, TWO_SPECIES_Q)
