"""Float64 CPU oracle of the Z_n-symmetric MPS and its block-sparse two-site update.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it; the library never does, and it imports nothing from the library.

arXiv:2303.11409, Sec. II builds the block-sparse MPS for U(1); Sec. I and the outlook
name more general Abelian symmetries.  This is the same construction for the cyclic
group Z_n with local dimension d <= n, the physical index i = 0..d-1 carrying charge
i (mod n):
  * bond b carries the right-charge c^[b] = (sum_{j >= b} i_j) mod n, c^[L] = 0;
  * block (l, m) of site s exists iff i = (l - m) mod n is a physical index (i < d); for
    d = n every pair (l, m) of charges occurs;
  * the two-site gate is block diagonal in the total charge q = (i + j) mod n; block q
    acts on the pairs (i, (q - i) mod n) with both entries below d, i ascending (rows
    outputs, columns inputs); for d < n one block can join pairs whose plain sums i + j
    differ by n;
  * Theta of an update splits by its middle charge c: rows are the left sectors l with
    i' = (l - c) mod n < d, columns the right sectors r with j' = (c - r) mod n < d
    (all of them for d = n), and
      Theta'(c)[l, r] = sum_m G_q[i', i] B^[s][l, m] B^[s+1][m, r],
      q = (l - r) mod n,  i = (l - m) mod n,
    one SVD per c, the global top-chi truncation, the inverse-free reassembly and the
    renormalisation exactly as in the U(1) oracle (same readings, same tie rule).
Charge sectors are listed in ascending order of their residue.  A U(1)-conserving model
also conserves the particle number mod n, so for d < n the same evolution runs in the
coarser Z_n blocks: each Theta(c) is a direct sum of the U(1) blocks of charges c + kn.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .u1mps import NOISE_REL, SectorPlan, select_kept


def zn_blocks_of(n: int, q: int, d: int | None = None) -> list[tuple[int, int]]:
    """Basis of the two-site gate block of total charge q: the pairs (i, (q - i) mod n) with
    both entries below d (default n), i ascending."""
    d = n if d is None else d
    return [(i, (q - i) % n) for i in range(d) if (q - i) % n < d]


def zn_charges(n: int, d: int | None = None) -> list[int]:
    """The total charges q whose gate block is not empty, ascending (all of 0..n-1 for d = n)."""
    return [q for q in range(n) if zn_blocks_of(n, q, d)]


def gate_blocks_from_dense(G: np.ndarray, n: int, d: int) -> dict:
    """The Z_n blocks of a two-site operator given as a d^2 x d^2 matrix on |i j>."""
    out = {}
    for q in zn_charges(n, d):
        idx = [i * d + j for i, j in zn_blocks_of(n, q, d)]
        out[q] = np.ascontiguousarray(G[np.ix_(idx, idx)], dtype=np.complex128)
    return out


def gate_blocks_from_u1(u1_blocks, n: int, d: int) -> dict:
    """The Z_n blocks of a U(1)-conserving gate given by its U(1) blocks (block t over the pairs
    (i, t - i), i ascending): a U(1) gate conserves the particle number mod n too, so block q
    joins the U(1) blocks of totals t = q, q + n, ..., with zeros between different totals."""
    out = {}
    for q in zn_charges(n, d):
        pairs = zn_blocks_of(n, q, d)
        G = np.zeros((len(pairs), len(pairs)), dtype=np.complex128)
        for a, (i, j) in enumerate(pairs):
            for b, (k, l) in enumerate(pairs):
                if i + j == k + l:
                    base = max(0, i + j - d + 1)       # first left index of U(1) block i + j
                    G[a, b] = u1_blocks[i + j][i - base, k - base]
        out[q] = G
    return out


def plan_update(left: dict, mid: dict, right: dict, n: int, d: int | None = None) -> SectorPlan:
    """The sector structure of a Z_n two-site update, by looping over charges: the triples
    (l, m, r) with (l - m) mod n and (m - r) mod n below d (every triple for d = n), the
    residues c with a row and a column, and for each the left sectors l with (l - c) mod n < d
    as rows and the right sectors r with (c - r) mod n < d as columns, ascending."""
    d = n if d is None else d
    triples = [(l, m, r) for l in sorted(left) for m in sorted(mid) if (l - m) % n < d
               for r in sorted(right) if (m - r) % n < d]
    rows, cols, sectors = {}, {}, []
    for c in range(n):
        rl = [l for l in sorted(left) if (l - c) % n < d]
        cl = [r for r in sorted(right) if (c - r) % n < d]
        if rl and cl:
            sectors.append(c)
            rows[c], cols[c] = rl, cl
    return SectorPlan(triples, sectors, rows, cols)


@dataclass
class ZnMPS:
    """Z_n-symmetric MPS in right-canonical block form (d = n).

    bond[b]: charge -> dimension; lam[b]: charge -> Schmidt values (descending);
    B[s]: (l, m) -> complex128 block of shape (bond[s][l], bond[s+1][m]).
    """
    L: int
    n: int
    Q: int
    bond: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    B: list = field(default_factory=list)
    d_local: int = 0          # local dimension d <= n (0: d = n)

    @property
    def d(self) -> int:
        return self.d_local or self.n

    @classmethod
    def product(cls, n: int, occupations, d: int | None = None) -> "ZnMPS":
        d = n if d is None else int(d)
        if not 2 <= d <= n:
            raise ValueError("local dimension outside [2, n]")
        occ = [int(x) for x in occupations]
        if any(not 0 <= x <= d - 1 for x in occ):
            raise ValueError("occupation outside [0, d-1]")
        L = len(occ)
        c = [sum(occ[b:]) % n for b in range(L + 1)]
        st = cls(L, n, c[0], d_local=d)
        st.bond = [{c[b]: 1} for b in range(L + 1)]
        st.lam = [{c[b]: np.ones(1)} for b in range(L + 1)]
        st.B = [{(c[s], c[s + 1]): np.ones((1, 1), dtype=np.complex128)} for s in range(L)]
        return st

    def apply_gate2(self, s: int, G, chi: int, cutoff: float) -> dict:
        """G[q] (q in zn_charges(n, d)): the gate on total charge q over zn_blocks_of(n, q, d)."""
        n, d = self.n, self.d
        left, mid, right = self.bond[s], self.bond[s + 1], self.bond[s + 2]
        BL, BR = self.B[s], self.B[s + 1]
        plan = plan_update(left, mid, right, n, d)
        # position of the left index i inside gate block q (i itself for d = n)
        pos = {q: {i: k for k, (i, _) in enumerate(zn_blocks_of(n, q, d))} for q in zn_charges(n, d)}
        theta = {}
        # loop over the middle charges and build Theta'(c) block by block
        for c in plan.sectors:
            rows, cols = plan.rows[c], plan.cols[c]
            T = np.zeros((sum(left[l] for l in rows), sum(right[r] for r in cols)), dtype=np.complex128)
            ro = 0
            for l in rows:
                co = 0
                for r in cols:
                    q = (l - r) % n
                    ip = (l - c) % n
                    block = T[ro:ro + left[l], co:co + right[r]]
                    for m in sorted(mid):
                        if (l, m) in BL and (m, r) in BR:
                            i = (l - m) % n
                            g = G[q][pos[q][ip], pos[q][i]]
                            if g != 0:
                                block += g * (BL[(l, m)] @ BR[(m, r)])
                    co += right[r]
                ro += left[l]
            theta[c] = T
        svals, vecs = {}, {}
        for c in plan.sectors:
            lam_rows = np.concatenate([self.lam[s][l] for l in plan.rows[c]])
            M = lam_rows[:, None] * theta[c]
            _, S, Yh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
            S = np.where(S <= NOISE_REL * math.sqrt(float(np.sum(S * S))), 0.0, S)
            svals[c], vecs[c] = S, Yh
        kept, info = select_kept(svals, chi, cutoff)
        norm_kept = info["kept_norm"]
        new_mid, new_lam, new_BL, new_BR = {}, {}, {}, {}
        for c in plan.sectors:
            k = kept[c]
            if k == 0:
                continue
            new_mid[c] = k
            new_lam[c] = svals[c][:k] / norm_kept
            Yh = vecs[c][:k, :]
            left_part = (theta[c] @ Yh.conj().T) / norm_kept
            ro = 0
            for l in plan.rows[c]:
                new_BL[(l, c)] = left_part[ro:ro + left[l], :].copy()
                ro += left[l]
            co = 0
            for r in plan.cols[c]:
                new_BR[(c, r)] = Yh[:, co:co + right[r]].copy()
                co += right[r]
        self.bond[s + 1] = new_mid
        self.lam[s + 1] = new_lam
        self.B[s] = new_BL
        self.B[s + 1] = new_BR
        info["kept"] = {c: k for c, k in kept.items() if k}
        return info

    # -- observables ---------------------------------------------------------
    def expect_local(self, s: int, diag_op) -> float:
        """<O_s> for an operator diagonal in the physical index: sum lambda^2 |B|^2 O(i)."""
        op = np.asarray(diag_op, dtype=np.float64)
        tot = 0.0
        for (l, m), blk in self.B[s].items():
            w = self.lam[s][l] ** 2
            tot += float(np.sum(w[:, None] * np.abs(blk) ** 2)) * op[(l - m) % self.n]
        return tot

    def amplitude(self, config) -> complex:
        """<i_1 ... i_L | psi>: one block per site along the charges the config fixes."""
        cfg = [int(x) for x in config]
        c = [sum(cfg[b:]) % self.n for b in range(self.L + 1)]
        if c[0] != self.Q:
            return 0.0
        v = np.ones((1,), dtype=np.complex128)
        for s in range(self.L):
            blk = self.B[s].get((c[s], c[s + 1]))
            if blk is None:
                return 0.0
            v = v @ blk
        return complex(v[0])

    def entropy(self, b: int) -> float:
        p = np.concatenate([v ** 2 for v in self.lam[b].values()])
        p = p[p > 0]
        return float(-np.sum(p * np.log(p)))
