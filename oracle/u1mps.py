"""Float64 CPU oracle of the U(1)-symmetric MPS and its block-sparse two-site update.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import it; the library itself never
does, and this module imports nothing from the library.

What it follows (arXiv:2303.11409, Sec. II):
  * the canonical MPS  c_{i1..iM} = sum Gamma^[1] lambda^[1] ... Gamma^[M]
    (the amplitude formula of Sec. II), stored here as the right-canonical
    product B^[k] = Gamma^[k] lambda^[k] together with the lambda's;
  * the U(1) form: every bond index carries a right-charge
    c^[k] = sum_{j>k} i_j, the Kronecker deltas force c^[k-1] - c^[k] = i_k,
    with c^[0] = N and c^[M] = 0 (Sec. II, U(1) amplitude formula), so a site
    tensor is a block matrix whose block (l, m) exists only for
    0 <= l - m <= d - 1 and carries no explicit physical index;
  * the two-site update: Theta is split by its middle charge into blocks
    Theta(c) of at most chi x chi each, and each is decomposed by its own SVD
    (Sec. II: one SVD per charge block of Theta);
  * the CPU algorithm "loops over allowed charge values to construct Theta(c)"
    (Sec. II, CPU/GPU implementation paragraph): update() does exactly that.

Readings where the paper is silent (the CUDA path follows the same ones):
  * sites are 0-based s = 0..L-1, bond b sits left of site b (b = 0..L), so site
    s joins bond s (left) and bond s+1 (right);
  * the state is kept right-canonical (B = Gamma lambda); the update is the
    inverse-free form: Theta' = G . B^[s] B^[s+1], M = diag(lambda^[s]) Theta',
    M = X S Y^dag, new B^[s+1] = Y^dag_kept, new B^[s] = Theta' Y_kept / |S_kept|;
  * truncation is global over all middle charges: keep the largest
    min(chi, #{sigma > cutoff * |sigma|_2}) values (strict '>'), ordered by
    (sigma descending, charge ascending, in-sector index ascending); values
    within TIE_REL * sigma_max of the chi-th value count as ties and are taken
    by (charge, index) order;
  * lambda on the new bond is renormalised to unit 2-norm after every update;
  * a sector's singular values at or below NOISE_REL * |M(c)|_F (32 eps) are
    rounding noise and count as exact zeros, so a zero cutoff keeps exactly the
    numerically nonzero spectrum.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

TIE_REL = 1e-11
NOISE_REL = 32.0 * np.finfo(np.float64).eps


# ---------------------------------------------------------------------------
# Charge bookkeeping (Sec. II, U(1) amplitude formula and its Kronecker deltas)
# ---------------------------------------------------------------------------

def gate_basis(n: int, d: int) -> list[int]:
    """Left-site occupations i of the two-site block of total charge n.

    The block's basis is (i, n - i) with 0 <= i, n - i <= d - 1, i ascending.
    """
    return list(range(max(0, n - d + 1), min(d - 1, n) + 1))


def bond_charge_range(L: int, d: int, N: int, b: int) -> tuple[int, int]:
    """Charges a bond b can carry: c = sum of occupations right of bond b.

    Sites 0..b-1 hold N - c with at most d-1 each, sites b..L-1 hold c.
    """
    lo = max(0, N - (d - 1) * b)
    hi = min(N, (d - 1) * (L - b))
    return lo, hi


def count_configs(n_sites: int, d: int, q: int) -> int:
    """Number of occupation strings of n_sites sites (0..d-1 each) summing to q."""
    if q < 0 or q > n_sites * (d - 1):
        return 0
    if n_sites == 0:
        return 1
    # inclusion-exclusion over sites exceeding d-1
    tot = 0
    for j in range(n_sites + 1):
        rem = q - j * d
        if rem < 0:
            break
        tot += (-1) ** j * math.comb(n_sites, j) * math.comb(rem + n_sites - 1, n_sites - 1)
    return tot


def hilbert_dim(L: int, d: int, N: int, b: int, c: int) -> int:
    """Largest possible dimension of charge sector c on bond b (Schmidt rank bound)."""
    return min(count_configs(b, d, N - c), count_configs(L - b, d, c))


@dataclass
class SectorPlan:
    """The sector structure of one two-site update at sites (s, s+1).

    triples: every (l, m, r) with l on bond s, m on bond s+1, r on bond s+2,
             0 <= l-m <= d-1 and 0 <= m-r <= d-1 (ascending lexicographic).
    sectors: the candidate new middle charges c', ascending; for each, the row
             charges (l ascending, 0 <= l-c' <= d-1) and column charges
             (r ascending, 0 <= c'-r <= d-1) that make up Theta(c').
    """
    triples: list[tuple[int, int, int]]
    sectors: list[int]
    rows: dict[int, list[int]]
    cols: dict[int, list[int]]


def plan_update(left: dict, mid: dict, right: dict, d: int) -> SectorPlan:
    """Enumerate the charge sectors of a two-site update by looping over charges."""
    triples = []
    for l in sorted(left):
        for m in sorted(mid):
            if not 0 <= l - m <= d - 1:
                continue
            for r in sorted(right):
                if 0 <= m - r <= d - 1:
                    triples.append((l, m, r))
    cands = set()
    for l in left:
        for r in right:
            if 0 <= l - r <= 2 * (d - 1):
                for c in range(max(r, l - d + 1), min(l, r + d - 1) + 1):
                    cands.add(c)
    sectors = sorted(cands)
    rows = {c: [l for l in sorted(left) if 0 <= l - c <= d - 1] for c in sectors}
    cols = {c: [r for r in sorted(right) if 0 <= c - r <= d - 1] for c in sectors}
    return SectorPlan(triples, sectors, rows, cols)


# ---------------------------------------------------------------------------
# Global truncation (Sec. II: bond dimension at most chi; tie-break is a reading)
# ---------------------------------------------------------------------------

def select_kept(sigmas: dict, chi: int, cutoff: float, tie_rel: float = TIE_REL):
    """Kept count per sector under the global top-chi rule.

    sigmas: charge -> singular values of that sector, descending.
    Returns (kept: dict charge -> count, info: dict).
    """
    if chi < 1:
        raise ValueError("chi must be >= 1")
    labels = []
    for c in sorted(sigmas):
        for idx, v in enumerate(sigmas[c]):
            labels.append((float(v), c, idx))
    total2 = sum(v * v for v, _, _ in labels)
    if total2 <= 0.0:
        raise FloatingPointError("all singular values vanish")
    total = math.sqrt(total2)
    thr = cutoff * total
    cand = [t for t in labels if t[0] > thr]
    info = dict(norm=total, threshold=thr, n_candidates=len(cand), band=0)
    if len(cand) <= chi:
        chosen = cand
    else:
        vals = sorted((t[0] for t in cand), reverse=True)
        v = vals[chi - 1]
        smax = vals[0]
        delta = tie_rel * smax
        above = [t for t in cand if t[0] > v + delta]
        band = [t for t in cand if t[0] <= v + delta and t[0] >= v - delta]
        band.sort(key=lambda t: (t[1], t[2]))
        chosen = above + band[: chi - len(above)]
        info["band"] = len(band)
    kept = {c: 0 for c in sigmas}
    for _, c, _ in chosen:
        kept[c] += 1
    # the kept set of a sector is a prefix of its descending list
    for c in sigmas:
        k = kept[c]
        chosen_idx = sorted(t[2] for t in chosen if t[1] == c)
        assert chosen_idx == list(range(k)), "kept set is not a prefix"
    kept2 = sum(float(np.sum(np.asarray(sigmas[c][: kept[c]]) ** 2)) for c in sigmas)
    disc2 = sum(float(np.sum(np.asarray(sigmas[c][kept[c]:]) ** 2)) for c in sigmas)
    info["kept_norm"] = math.sqrt(kept2)
    info["trunc_err"] = disc2 / total2
    return kept, info


# ---------------------------------------------------------------------------
# The state
# ---------------------------------------------------------------------------

@dataclass
class U1MPS:
    """U(1)-symmetric MPS in right-canonical block form.

    bond[b]: charge -> dimension, for bonds b = 0..L
    lam[b]:  charge -> Schmidt values (float64, descending)
    B[s]:    (l, m) -> complex128 block of shape (bond[s][l], bond[s+1][m])
    """
    L: int
    d: int
    N: int
    bond: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    B: list = field(default_factory=list)

    @classmethod
    def product(cls, d: int, occupations) -> "U1MPS":
        occ = [int(x) for x in occupations]
        L = len(occ)
        if any(not 0 <= x <= d - 1 for x in occ):
            raise ValueError("occupation outside [0, d-1]")
        c = [sum(occ[b:]) for b in range(L + 1)]
        st = cls(L, d, c[0])
        st.bond = [{c[b]: 1} for b in range(L + 1)]
        st.lam = [{c[b]: np.ones(1)} for b in range(L + 1)]
        st.B = [{(c[s], c[s + 1]): np.ones((1, 1), dtype=np.complex128)} for s in range(L)]
        return st

    def copy(self) -> "U1MPS":
        return U1MPS(self.L, self.d, self.N,
                     [dict(b) for b in self.bond],
                     [{c: v.copy() for c, v in lb.items()} for lb in self.lam],
                     [{k: v.copy() for k, v in bs.items()} for bs in self.B])

    # -- the two-site update -------------------------------------------------
    def apply_gate2(self, s: int, G, chi: int, cutoff: float) -> dict:
        """Apply a two-site gate to sites (s, s+1), truncate globally, reassemble.

        G[n] (n = 0..2(d-1)) is the gate restricted to total charge n, a square
        complex matrix over the basis gate_basis(n, d): rows are outputs
        (i', n-i'), columns inputs (i, n-i).
        """
        d = self.d
        if not 0 <= s < self.L - 1:
            raise IndexError("gate site out of range")
        left, mid, right = self.bond[s], self.bond[s + 1], self.bond[s + 2]
        lam_left = self.lam[s]
        BL, BR = self.B[s], self.B[s + 1]
        plan = plan_update(left, mid, right, d)

        theta = {}
        # Loop over the allowed middle charges and build Theta'(c) block by block.
        for c in plan.sectors:
            rows, cols = plan.rows[c], plan.cols[c]
            m_rows = sum(left[l] for l in rows)
            n_cols = sum(right[r] for r in cols)
            T = np.zeros((m_rows, n_cols), dtype=np.complex128)
            ro = 0
            for l in rows:
                co = 0
                for r in cols:
                    n = l - r
                    base = max(0, n - d + 1)
                    block = T[ro:ro + left[l], co:co + right[r]]
                    for m in sorted(mid):
                        i, j = l - m, m - r
                        if 0 <= i <= d - 1 and 0 <= j <= d - 1:
                            g = G[n][(l - c) - base, i - base]
                            if g != 0:
                                block += g * (BL[(l, m)] @ BR[(m, r)])
                    co += right[r]
                ro += left[l]
            theta[c] = T

        # Per-sector SVD of M(c) = diag(lambda^[s]) Theta'(c).
        svals, vecs = {}, {}
        for c in plan.sectors:
            lam_rows = np.concatenate([lam_left[l] for l in plan.rows[c]])
            M = lam_rows[:, None] * theta[c]
            _, S, Yh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
            # rounding-level singular values are zero (noise floor 32 eps |M|_F)
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
        info["sectors"] = {c: (sum(left[l] for l in plan.rows[c]), sum(right[r] for r in plan.cols[c]))
                           for c in plan.sectors}
        info["sigmas"] = svals
        return info

    # -- observables ---------------------------------------------------------
    def expect_local(self, s: int, diag_op) -> float:
        """<O_s> from the local canonical formula: sum lambda^2 |B|^2 O(l - m)."""
        val = 0.0
        for (l, m), blk in self.B[s].items():
            w = self.lam[s][l] ** 2
            val += float(diag_op[l - m]) * float(np.sum(w[:, None] * np.abs(blk) ** 2))
        return val

    def expect_transfer(self, s: int, diag_op) -> float:
        """<psi|O_s|psi> / <psi|psi> by a full left-to-right transfer contraction."""
        num = self._transfer(s, diag_op)
        den = self._transfer(-1, None)
        return num / den

    def _transfer(self, s, diag_op) -> float:
        E = {self.N: np.ones((1, 1), dtype=np.complex128)}
        for t in range(self.L):
            En = {}
            for (l, m), blk in self.B[t].items():
                if l not in E:
                    continue
                w = 1.0 if t != s else float(diag_op[l - m])
                contrib = w * (blk.conj().T @ E[l] @ blk)
                En[m] = En[m] + contrib if m in En else contrib
            E = En
        return float(E[0][0, 0].real)

    def norm2(self) -> float:
        return self._transfer(-1, None)

    def entropy(self, b: int) -> float:
        """Bond entropy -sum lambda^2 ln lambda^2 over all sectors of bond b."""
        p = np.concatenate([v ** 2 for v in self.lam[b].values()])
        p = p[p > 0]
        return float(-np.sum(p * np.log(p)))

    def amplitude(self, config) -> complex:
        """<i_1..i_L|psi> as the product of the one block per site the charges pick."""
        cfg = [int(x) for x in config]
        if len(cfg) != self.L or sum(cfg) != self.N:
            return 0j
        c = [sum(cfg[b:]) for b in range(self.L + 1)]
        v = np.ones((1, 1), dtype=np.complex128)
        for s in range(self.L):
            blk = self.B[s].get((c[s], c[s + 1]))
            if blk is None:
                return 0j
            v = v @ blk
        return complex(v[0, 0])

    def to_dense(self) -> np.ndarray:
        """Full state vector, shape (d,)*L, by contracting site by site (small L only)."""
        d = self.d
        # rows: occupation prefixes; track per right charge of the current bond
        cur = {self.N: ([()], np.ones((1, 1), dtype=np.complex128))}
        for s in range(self.L):
            nxt = {}
            for (l, m), blk in self.B[s].items():
                if l not in cur:
                    continue
                prefs, mat = cur[l]
                i = l - m
                newp = [p + (i,) for p in prefs]
                newm = mat @ blk
                if m in nxt:
                    nxt[m] = (nxt[m][0] + newp, np.vstack([nxt[m][1], newm]))
                else:
                    nxt[m] = (newp, newm)
            cur = nxt
        psi = np.zeros((d,) * self.L, dtype=np.complex128)
        prefs, mat = cur[0]
        for p, v in zip(prefs, mat[:, 0]):
            psi[p] = v
        return psi

    # -- structure checks ----------------------------------------------------
    def check_structure(self) -> None:
        """Assert the charge rule of every bond and block (Sec. II Kronecker deltas)."""
        L, d, N = self.L, self.d, self.N
        assert self.bond[0] == {N: 1} and self.bond[L] == {0: 1}
        for b in range(L + 1):
            lo, hi = bond_charge_range(L, d, N, b)
            for c, D in self.bond[b].items():
                assert lo <= c <= hi, (b, c)
                assert D >= 1
                assert self.lam[b][c].shape == (D,)
        for s in range(L):
            for (l, m), blk in self.B[s].items():
                assert 0 <= l - m <= d - 1, (s, l, m)
                assert blk.shape == (self.bond[s][l], self.bond[s + 1][m])

    def site_nnz(self, s: int) -> int:
        return sum(blk.size for blk in self.B[s].values())

    def bond_dim(self, b: int) -> int:
        return sum(self.bond[b].values())
