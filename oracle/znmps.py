"""Float64 CPU oracle of the Z_n-symmetric MPS and its block-sparse two-site update.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it; the library never does, and it imports nothing from the library.

arXiv:2303.11409, Sec. II builds the block-sparse MPS for U(1); Sec. I and the outlook
name more general Abelian symmetries.  This is the same construction for the cyclic
group Z_n with local dimension d = n, the physical index i carrying charge i (mod n):
  * bond b carries the right-charge c^[b] = (sum_{j >= b} i_j) mod n, c^[L] = 0;
  * block (l, m) of site s carries the physical index i = (l - m) mod n; since d = n,
    every pair (l, m) of charges occurs;
  * the two-site gate is block diagonal in the total charge q = (i + j) mod n; block q
    acts on the pairs (i, (q - i) mod n), i = 0..n-1 ascending (rows outputs, columns
    inputs);
  * Theta of an update splits by its middle charge c: rows are all left sectors l (with
    i' = (l - c) mod n), columns all right sectors r (with j' = (c - r) mod n), and
      Theta'(c)[l, r] = sum_m G_q[i', i] B^[s][l, m] B^[s+1][m, r],
      q = (l - r) mod n,  i = (l - m) mod n,
    one SVD per c, the global top-chi truncation, the inverse-free reassembly and the
    renormalisation exactly as in the U(1) oracle (same readings, same tie rule).
Charge sectors are listed in ascending order of their residue.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .u1mps import NOISE_REL, SectorPlan, select_kept


def zn_blocks_of(n: int, q: int) -> list[tuple[int, int]]:
    """Basis of the two-site gate block of total charge q: (i, (q - i) mod n), i ascending."""
    return [(i, (q - i) % n) for i in range(n)]


def plan_update(left: dict, mid: dict, right: dict, n: int) -> SectorPlan:
    """The sector structure of a Z_n two-site update (d = n): every (l, m, r) is a triple (each
    residue difference is a physical index), every residue c = 0..n-1 a middle charge, and
    Theta(c) has all left sectors as rows and all right sectors as columns, ascending."""
    triples = [(l, m, r) for l in sorted(left) for m in sorted(mid) for r in sorted(right)]
    sectors = list(range(n))
    rows = {c: sorted(left) for c in sectors}
    cols = {c: sorted(right) for c in sectors}
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

    @property
    def d(self) -> int:
        return self.n

    @classmethod
    def product(cls, n: int, occupations) -> "ZnMPS":
        occ = [int(x) for x in occupations]
        if any(not 0 <= x <= n - 1 for x in occ):
            raise ValueError("occupation outside [0, n-1]")
        L = len(occ)
        c = [sum(occ[b:]) % n for b in range(L + 1)]
        st = cls(L, n, c[0])
        st.bond = [{c[b]: 1} for b in range(L + 1)]
        st.lam = [{c[b]: np.ones(1)} for b in range(L + 1)]
        st.B = [{(c[s], c[s + 1]): np.ones((1, 1), dtype=np.complex128)} for s in range(L)]
        return st

    def apply_gate2(self, s: int, G, chi: int, cutoff: float) -> dict:
        """G[q] (q = 0..n-1): the gate on total charge q over zn_blocks_of(n, q)."""
        n = self.n
        left, mid, right = self.bond[s], self.bond[s + 1], self.bond[s + 2]
        BL, BR = self.B[s], self.B[s + 1]
        plan = plan_update(left, mid, right, n)
        rows = plan.rows[0]
        cols = plan.cols[0]
        m_rows = sum(left[l] for l in rows)
        n_cols = sum(right[r] for r in cols)
        theta = {}
        # loop over the middle charges and build Theta'(c) block by block
        for c in range(n):
            T = np.zeros((m_rows, n_cols), dtype=np.complex128)
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
                            g = G[q][ip, i]
                            if g != 0:
                                block += g * (BL[(l, m)] @ BR[(m, r)])
                    co += right[r]
                ro += left[l]
            theta[c] = T
        lam_rows = np.concatenate([self.lam[s][l] for l in rows])
        svals, vecs = {}, {}
        for c in range(n):
            M = lam_rows[:, None] * theta[c]
            _, S, Yh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
            S = np.where(S <= NOISE_REL * math.sqrt(float(np.sum(S * S))), 0.0, S)
            svals[c], vecs[c] = S, Yh
        kept, info = select_kept(svals, chi, cutoff)
        norm_kept = info["kept_norm"]
        new_mid, new_lam, new_BL, new_BR = {}, {}, {}, {}
        for c in range(n):
            k = kept[c]
            if k == 0:
                continue
            new_mid[c] = k
            new_lam[c] = svals[c][:k] / norm_kept
            Yh = vecs[c][:k, :]
            left_part = (theta[c] @ Yh.conj().T) / norm_kept
            ro = 0
            for l in rows:
                new_BL[(l, c)] = left_part[ro:ro + left[l], :].copy()
                ro += left[l]
            co = 0
            for r in cols:
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
