"""Float64 CPU oracle of two-site DMRG on the U(1) block-sparse MPS.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import it; the library never does, and this
module imports nothing from the library.

The paper (Sec. I) names DMRG as the ground-state method whose MPS the U(1)
machinery of Sec. II serves.  The variational two-site step is the same block
structure as the TEBD update: the two-site wave function of sites (s, s+1) is
the set of matrices Psi(c) over the middle charge c, laid out exactly as the
Theta(c) blocks of the TEBD update (rows: left-bond sectors l = c .. c+d-1,
physical index i = l - c; columns: right-bond sectors r = c-d+1 .. c, physical
index j = c - r).  One step replaces Psi by the lowest eigenvector of the
effective Hamiltonian, splits it per middle charge by an SVD (Sec. II: one SVD
per charge block), truncates globally with the TEBD rule and moves on.

Readings (the paper gives no DMRG schedule; the CUDA path follows the same):
  * H = sum_k h_{k,k+1} over the L-1 bonds, each h_k given by its charge blocks
    in the two-site gate layout (block n over (i, n - i), i ascending);
  * each bond term is split into charge-shifting operator pairs
    h = sum_t O_t (x) P_t, O_t raising the left site's occupation by delta_t and
    P_t lowering the right site's by delta_t (an SVD of h's matrix elements
    grouped by delta; terms below 1e-14 of the largest are dropped);
  * a sweep is a right-moving pass over s = 0 .. L-2 followed by a left-moving
    pass over s = L-2 .. 0 (2(L-1) local steps); the state starts right-canonical
    (B = Gamma lambda, any state the TEBD update produces, e.g. a product state);
  * right-moving: Psi(c) = U S V^dag, site s <- U_kept (left-canonical),
    site s+1 <- S_kept V_kept^dag / |S_kept|; left-moving: site s+1 <- V_kept^dag
    (right-canonical), site s <- Psi(c) V_kept / |S_kept|; the bond's lambda is
    S_kept / |S_kept| (the TEBD truncation and noise floor, u1mps.select_kept);
  * the local ground state: the lowest eigenvector of H_eff (dense eigh for
    dim <= DENSE_MAX, else ARPACK's Lanczos with tol 1e-13 from the current Psi);
  * two-site TDVP (tdvp_step): the same steps with the ground-state solve replaced by
    exp(-i dt/2 H_eff) of the pair, and after every split but the turn the new centre site
    evolved backward by exp(+i dt/2 H_eff^(1)) (its one-site effective Hamiltonian); a step
    of length dt is a right-moving then a left-moving pass of dt/2 each; exponentials by dense
    expm, or scipy's expm_multiply for large dimensions;
  * after the last sweep the state is brought back to the TEBD storage form
    (right-canonical B with every lambda the Schmidt values) by one inverse-free
    left-to-right pass: B'(l, m) = W(l) B(l, m), M(m) = diag(lambda_l) B'(., m)
    stacked over l, M = U S V^dag, lambda(m) = S, B(l, m) <- B'(l, m) V and
    W(m) = V^dag for the next site (values at or below the noise floor dropped).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse.linalg as spla

from .u1mps import NOISE_REL, U1MPS, gate_basis, plan_update, select_kept

DENSE_MAX = 600
SPLIT_REL = 1e-14


# ---------------------------------------------------------------------------
# Bond terms as charge-shifting operator pairs
# ---------------------------------------------------------------------------

def bond_matrix(h_blocks, d: int) -> np.ndarray:
    """The d^2 x d^2 matrix <i' j'|h|i j> (index i*d + j) of a bond term given by charge blocks."""
    H = np.zeros((d * d, d * d), dtype=np.complex128)
    for n, blk in enumerate(h_blocks):
        basis = gate_basis(n, d)
        for a, i2 in enumerate(basis):
            for b, i in enumerate(basis):
                H[i2 * d + (n - i2), i * d + (n - i)] = blk[a][b]
    return H


def split_bond_term(h_blocks, d: int):
    """h = sum_t O_t (x) P_t with O_t[i', i] != 0 only for i' - i = delta_t.

    Returns [(delta_t, O_t, P_t)].  For each delta the elements <i' j'|h|i j> with
    i' - i = delta (hence j' - j = -delta) form a matrix over (i', i) x (j', j),
    whose SVD gives the pairs.
    """
    H = bond_matrix(h_blocks, d)
    hmax = float(np.max(np.abs(H))) if H.size else 0.0
    terms = []
    for delta in range(-(d - 1), d):
        rows = [(i2, i) for i in range(d) for i2 in range(d) if i2 - i == delta]
        cols = [(j2, j) for j in range(d) for j2 in range(d) if j2 - j == -delta]
        X = np.zeros((len(rows), len(cols)), dtype=np.complex128)
        for a, (i2, i) in enumerate(rows):
            for b, (j2, j) in enumerate(cols):
                X[a, b] = H[i2 * d + j2, i * d + j]
        if not np.any(X):
            continue
        u, s, vh = np.linalg.svd(X)
        for t in range(len(s)):
            if s[t] <= SPLIT_REL * max(hmax, 1e-300):
                continue
            O = np.zeros((d, d), dtype=np.complex128)
            P = np.zeros((d, d), dtype=np.complex128)
            for a, (i2, i) in enumerate(rows):
                O[i2, i] = u[a, t] * s[t]
            for b, (j2, j) in enumerate(cols):
                P[j2, j] = vh[t, b]
            terms.append((delta, O, P))
    return terms


# ---------------------------------------------------------------------------
# Two-site DMRG
# ---------------------------------------------------------------------------

def _sub(mat, roff, coff, l, r, left, right):
    return mat[roff[l]:roff[l] + left[l], coff[r]:coff[r] + right[r]]


class DMRG:
    """Two-site DMRG on a U1MPS (modified in place)."""

    def __init__(self, state: U1MPS, h_bonds):
        if len(h_bonds) != state.L - 1:
            raise ValueError("one bond term per bond (L - 1)")
        self.st = state
        self.d = state.d
        self.h = [[np.asarray(b, dtype=np.complex128) for b in hb] for hb in h_bonds]
        self.terms = [split_bond_term(hb, state.d) for hb in h_bonds]
        L = state.L
        # left environments at bond b: EH[b][l] (D_l x D_l), ET[b][t][l] (D_l x D_{l+delta_t})
        # for the terms of bond b-1; right environments at bond b: RH[b][r] with
        # RH[b][r][b', b] = <b|H_right|b'>, RT[b][t][r] (D_{r+delta_t} x D_r) for the terms of bond b
        self.EH = [None] * (L + 1)
        self.ET = [None] * (L + 1)
        self.RH = [None] * (L + 1)
        self.RT = [None] * (L + 1)
        N = state.N
        self.EH[0] = {N: np.zeros((1, 1), dtype=np.complex128)}
        self.ET[0] = []
        self.RH[L] = {0: np.zeros((1, 1), dtype=np.complex128)}
        self.RT[L] = []
        for s in range(L - 1, 1, -1):
            self._right_env(s)
        self.energies = []

    # -- environments --------------------------------------------------------
    def _left_env(self, s: int) -> None:
        """Environment at bond s+1 from the one at bond s and the left-canonical site s."""
        st, d = self.st, self.d
        A = st.B[s]
        EH, ET = self.EH[s], self.ET[s]
        cross = self.terms[s - 1] if s >= 1 else []
        newH = {}
        for (l, m), a in A.items():
            if l not in EH:
                continue
            v = a.conj().T @ EH[l] @ a
            for t, (delta, _O, P) in enumerate(cross):
                l2 = l + delta
                if (l2, m) in A and l in ET[t]:
                    i, i2 = l - m, l2 - m
                    if P[i, i2] != 0:
                        v = v + P[i, i2] * (a.conj().T @ ET[t][l] @ A[(l2, m)])
            newH[m] = newH[m] + v if m in newH else v
        for m, Dm in st.bond[s + 1].items():
            if m not in newH:
                newH[m] = np.zeros((Dm, Dm), dtype=np.complex128)
        newT = []
        for delta, O, _P in self.terms[s] if s <= st.L - 2 else []:
            blocks = {}
            for (l, m), a in A.items():
                m2 = m + delta
                if (l, m2) not in A:
                    continue
                i, i2 = l - m, l - m2
                if O[i, i2] == 0:
                    continue
                v = O[i, i2] * (a.conj().T @ A[(l, m2)])
                blocks[m] = blocks[m] + v if m in blocks else v
            newT.append(blocks)
        self.EH[s + 1], self.ET[s + 1] = newH, newT

    def _right_env(self, s: int) -> None:
        """Environment at bond s from the one at bond s+1 and the right-canonical site s."""
        st = self.st
        B = st.B[s]
        RH, RT = self.RH[s + 1], self.RT[s + 1]
        cross = self.terms[s] if s <= st.L - 2 else []
        newH = {}
        for (m, r), b in B.items():
            if r not in RH:
                continue
            v = b @ RH[r] @ b.conj().T
            for t, (delta, O, _P) in enumerate(cross):
                r2 = r + delta
                if (m, r2) in B and r in RT[t]:
                    j, j2 = m - r, m - r2
                    if O[j, j2] != 0:
                        v = v + O[j, j2] * (B[(m, r2)] @ RT[t][r] @ b.conj().T)
            newH[m] = newH[m] + v if m in newH else v
        for m, Dm in st.bond[s].items():
            if m not in newH:
                newH[m] = np.zeros((Dm, Dm), dtype=np.complex128)
        newT = []
        for delta, _O, P in self.terms[s - 1] if s >= 1 else []:
            blocks = {}
            for (m, r), b in B.items():
                m2 = m + delta
                if (m2, r) not in B:
                    continue
                j, j2 = m - r, m2 - r
                if P[j, j2] == 0:
                    continue
                v = P[j, j2] * (B[(m2, r)] @ b.conj().T)
                blocks[m] = blocks[m] + v if m in blocks else v
            newT.append(blocks)
        self.RH[s], self.RT[s] = newH, newT

    # -- the two-site wave function and H_eff --------------------------------
    def _layout(self, s: int):
        st, d = self.st, self.d
        left, mid, right = st.bond[s], st.bond[s + 1], st.bond[s + 2]
        plan = plan_update(left, mid, right, d)
        lay = []
        off = 0
        for c in plan.sectors:
            rows, cols = plan.rows[c], plan.cols[c]
            roff, coff = {}, {}
            m_ = 0
            for l in rows:
                roff[l] = m_
                m_ += left[l]
            n_ = 0
            for r in cols:
                coff[r] = n_
                n_ += right[r]
            lay.append(dict(c=c, rows=rows, cols=cols, roff=roff, coff=coff, m=m_, n=n_, off=off))
            off += m_ * n_
        return lay, off

    def _theta(self, s: int, lay):
        """Psi(c)[l, r] = B^[s][l, c] B^[s+1][c, r] (the identity-gate Theta)."""
        st = self.st
        left, right = st.bond[s], st.bond[s + 2]
        out = {}
        for e in lay:
            c = e["c"]
            T = np.zeros((e["m"], e["n"]), dtype=np.complex128)
            for l in e["rows"]:
                for r in e["cols"]:
                    if (l, c) in st.B[s] and (c, r) in st.B[s + 1]:
                        _sub(T, e["roff"], e["coff"], l, r, left, right)[...] = st.B[s][(l, c)] @ st.B[s + 1][(c, r)]
            out[c] = T
        return out

    def _apply(self, s: int, lay, X: dict) -> dict:
        """H_eff Psi for the two-site centre (s, s+1)."""
        st, d = self.st, self.d
        left, right = st.bond[s], st.bond[s + 2]
        EH, ET, RH, RT = self.EH[s], self.ET[s], self.RH[s + 2], self.RT[s + 2]
        lcross = self.terms[s - 1] if s >= 1 else []
        rcross = self.terms[s + 1] if s + 1 <= st.L - 2 else []
        hc = self.h[s]
        byc = {e["c"]: e for e in lay}
        Y = {}
        for e in lay:
            c, roff, coff = e["c"], e["roff"], e["coff"]
            Yc = np.zeros((e["m"], e["n"]), dtype=np.complex128)
            Xc = X[c]
            for l in e["rows"]:
                i = l - c
                for r in e["cols"]:
                    j = c - r
                    y = _sub(Yc, roff, coff, l, r, left, right)
                    x = _sub(Xc, roff, coff, l, r, left, right)
                    # the left block's Hamiltonian and the right block's
                    y += EH[l] @ x
                    y += x @ RH[r]
                    # the bond term between the left block and site s
                    for t, (delta, _O, P) in enumerate(lcross):
                        l2, i2 = l + delta, i + delta
                        if l2 in roff and l in ET[t] and P[i, i2] != 0:
                            y += P[i, i2] * (ET[t][l] @ _sub(Xc, roff, coff, l2, r, left, right))
                    # the bond term between site s+1 and the right block
                    for t, (delta, O, _P) in enumerate(rcross):
                        r2, j2 = r + delta, j - delta
                        if r2 in coff and r in RT[t] and O[j, j2] != 0:
                            y += O[j, j2] * (_sub(Xc, roff, coff, l, r2, left, right) @ RT[t][r])
                    # the centre bond term mixes the middle charges of the pair (l, r)
                    n = l - r
                    basis = gate_basis(n, d)
                    for b, i2 in enumerate(basis):
                        c2 = l - i2
                        if c2 not in byc:
                            continue
                        e2 = byc[c2]
                        if l not in e2["roff"] or r not in e2["coff"]:
                            continue
                        g = hc[n][i - basis[0], b]
                        if g != 0:
                            y += g * _sub(X[c2], e2["roff"], e2["coff"], l, r, left, right)
            Y[c] = Yc
        return Y

    @staticmethod
    def _flat(lay, X):
        return np.concatenate([X[e["c"]].reshape(-1) for e in lay]) if lay else np.zeros(0, complex)

    @staticmethod
    def _unflat(lay, v):
        return {e["c"]: v[e["off"]:e["off"] + e["m"] * e["n"]].reshape(e["m"], e["n"]).copy() for e in lay}

    def local_ground_state(self, s: int, lay, dim, X0):
        """Lowest eigenpair of H_eff (dense eigh for small dim, else ARPACK Lanczos)."""
        if dim <= DENSE_MAX:
            H = np.zeros((dim, dim), dtype=np.complex128)
            for k in range(dim):
                e = np.zeros(dim, dtype=np.complex128)
                e[k] = 1.0
                H[:, k] = self._flat(lay, self._apply(s, lay, self._unflat(lay, e)))
            H = 0.5 * (H + H.conj().T)
            w, v = scipy.linalg.eigh(H)
            return float(w[0]), v[:, 0]
        op = spla.LinearOperator((dim, dim), dtype=np.complex128,
                                 matvec=lambda v: self._flat(lay, self._apply(s, lay, self._unflat(lay, v))))
        v0 = self._flat(lay, X0)
        if not np.any(v0):
            v0 = None
        w, v = spla.eigsh(op, k=1, which="SA", v0=v0, tol=1e-13, ncv=min(dim - 1, 40), maxiter=100000)
        return float(w[0]), v[:, 0]

    # -- one local step --------------------------------------------------------
    def step(self, s: int, chi: int, cutoff: float, right_moving: bool, local=None) -> dict:
        """One two-site step; `local(s, lay, dim, X0)` -> (value, new vector) replaces the
        ground-state solve (TDVP passes its forward exponential)."""
        st = self.st
        left, right = st.bond[s], st.bond[s + 2]
        lay, dim = self._layout(s)
        X0 = self._theta(s, lay)
        E, v = (local or self.local_ground_state)(s, lay, dim, X0)
        Psi = self._unflat(lay, v)
        svals, us, vhs = {}, {}, {}
        for e in lay:
            U, S, Vh = scipy.linalg.svd(Psi[e["c"]], full_matrices=False, lapack_driver="gesvd")
            S = np.where(S <= NOISE_REL * math.sqrt(float(np.sum(S * S))), 0.0, S)
            svals[e["c"]], us[e["c"]], vhs[e["c"]] = S, U, Vh
        kept, info = select_kept(svals, chi, cutoff)
        nk = info["kept_norm"]
        new_mid, new_lam, BL, BR = {}, {}, {}, {}
        for e in lay:
            c, k = e["c"], kept[e["c"]]
            if k == 0:
                continue
            new_mid[c] = k
            new_lam[c] = svals[c][:k] / nk
            U, S, Vh = us[c][:, :k], svals[c][:k], vhs[c][:k, :]
            if right_moving:
                lpart, rpart = U, (S[:, None] * Vh) / nk
            else:
                lpart, rpart = (Psi[c] @ Vh.conj().T) / nk, Vh
            for l in e["rows"]:
                BL[(l, c)] = lpart[e["roff"][l]:e["roff"][l] + left[l], :].copy()
            for r in e["cols"]:
                BR[(c, r)] = rpart[:, e["coff"][r]:e["coff"][r] + right[r]].copy()
        st.bond[s + 1], st.lam[s + 1], st.B[s], st.B[s + 1] = new_mid, new_lam, BL, BR
        if right_moving:
            self._left_env(s)
        else:
            self._right_env(s + 1)
        if E is not None:
            self.energies.append(E)
        return dict(energy=E, dim=dim, kept=dict(new_mid), trunc_err=info["trunc_err"], sigmas=svals)

    # -- TDVP -------------------------------------------------------------------
    def _apply1(self, j: int, C: dict) -> dict:
        """One-site H_eff on the blocks C[(l, m)] of site j (left environment at bond j,
        right environment at bond j+1)."""
        st, d = self.st, self.d
        EH, ET, RH, RT = self.EH[j], self.ET[j], self.RH[j + 1], self.RT[j + 1]
        lcross = self.terms[j - 1] if j >= 1 else []
        rcross = self.terms[j] if j <= st.L - 2 else []
        out = {}
        for (l, m), x in C.items():
            i = l - m
            y = EH[l] @ x + x @ RH[m]
            for t, (delta, _O, P) in enumerate(lcross):
                i2 = i + delta
                if 0 <= i2 < d and (l + delta, m) in C and l in ET[t] and P[i, i2] != 0:
                    y = y + P[i, i2] * (ET[t][l] @ C[(l + delta, m)])
            for t, (delta, O, _P) in enumerate(rcross):
                i3 = i - delta
                if 0 <= i3 < d and (l, m + delta) in C and m in RT[t] and O[i, i3] != 0:
                    y = y + O[i, i3] * (C[(l, m + delta)] @ RT[t][m])
            out[(l, m)] = y
        return out

    @staticmethod
    def _expm_apply(apply, v0: np.ndarray, t: complex) -> np.ndarray:
        """exp(t H) v0 for the Hermitian H that `apply` multiplies by (dense expm for small
        dimensions, else scipy's expm_multiply)."""
        dim = v0.size
        if dim <= DENSE_MAX:
            H = np.zeros((dim, dim), dtype=np.complex128)
            for k in range(dim):
                e = np.zeros(dim, dtype=np.complex128)
                e[k] = 1.0
                H[:, k] = apply(e)
            H = 0.5 * (H + H.conj().T)
            return scipy.linalg.expm(t * H) @ v0
        op = spla.LinearOperator((dim, dim), dtype=np.complex128, matvec=lambda v: t * apply(v),
                                 rmatvec=lambda v: np.conj(t) * apply(v))
        return spla.expm_multiply(op, v0, traceA=0.0)

    def _backward(self, j: int, tau: float) -> None:
        """Site j (the centre) <- exp(+i tau H_eff^(1)) site j."""
        keys = sorted(self.st.B[j])
        shapes = [self.st.B[j][k].shape for k in keys]
        sizes = [a * b for a, b in shapes]
        offs = np.cumsum([0] + sizes)

        def unflat(v):
            return {k: v[offs[n]:offs[n + 1]].reshape(shapes[n]) for n, k in enumerate(keys)}

        def flat(C):
            return np.concatenate([C[k].reshape(-1) for k in keys])

        v = self._expm_apply(lambda x: flat(self._apply1(j, unflat(x))), flat(self.st.B[j]), 1j * tau)
        self.st.B[j] = {k: b.copy() for k, b in unflat(v).items()}

    def tdvp_step(self, dt: float, chi: int, cutoff: float) -> list:
        """One second-order two-site TDVP step of length dt: a right-moving and a left-moving
        pass of dt/2 each; every pair is evolved forward by exp(-i dt/2 H_eff^(2)), split, and
        the new centre site evolved backward by exp(+i dt/2 H_eff^(1)) except at the turn."""
        L = self.st.L
        half = 0.5 * dt

        def forward(s, lay, dim, X0):
            v0 = self._flat(lay, X0)
            return None, self._expm_apply(lambda x: self._flat(lay, self._apply(s, lay, self._unflat(lay, x))),
                                          v0, -1j * half)
        out = []
        for s in range(0, L - 1):
            out.append(self.step(s, chi, cutoff, True, local=forward))
            if s < L - 2:
                self._backward(s + 1, half)
        for s in range(L - 2, -1, -1):
            out.append(self.step(s, chi, cutoff, False, local=forward))
            if s > 0:
                self._backward(s, half)
        return out

    def sweep(self, chi: int, cutoff: float) -> list:
        L = self.st.L
        out = []
        for s in range(0, L - 1):
            out.append(self.step(s, chi, cutoff, True))
        for s in range(L - 2, -1, -1):
            out.append(self.step(s, chi, cutoff, False))
        return out

    def canonicalize(self) -> None:
        """Back to right-canonical B with Schmidt lambdas (inverse-free left-to-right pass)."""
        st, d = self.st, self.d
        N = st.N
        W = {N: np.ones((1, 1), dtype=np.complex128)}
        st.lam[0] = {N: np.ones(1)}
        for s in range(st.L):
            Bp = {(l, m): W[l] @ blk for (l, m), blk in st.B[s].items() if l in W}
            if s == st.L - 1:
                st.B[s] = Bp
                break
            left = {l: W[l].shape[0] for l in W}
            svals, vhs, rows_of = {}, {}, {}
            for m in sorted(st.bond[s + 1]):
                rows = [l for l in sorted(left) if (l, m) in Bp]
                if not rows:
                    continue
                M = np.vstack([st.lam[s][l][:, None] * Bp[(l, m)] for l in rows])
                _, S, Vh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
                S = np.where(S <= NOISE_REL * math.sqrt(float(np.sum(S * S))), 0.0, S)
                svals[m], vhs[m], rows_of[m] = S, Vh, rows
            kept, info = select_kept(svals, 1 << 30, 0.0)
            nk = info["kept_norm"]
            newB, newW, bond, lam = {}, {}, {}, {}
            for m in sorted(svals):
                k = kept[m]
                if k == 0:
                    continue
                Vh = vhs[m][:k, :]
                for l in rows_of[m]:
                    newB[(l, m)] = Bp[(l, m)] @ Vh.conj().T
                newW[m] = Vh
                bond[m] = k
                lam[m] = svals[m][:k] / nk
            st.B[s], st.bond[s + 1], st.lam[s + 1] = newB, bond, lam
            W = newW
        st.lam[st.L] = {0: np.ones(1)}


def run_tdvp(state: U1MPS, h_bonds, n_steps: int, dt: float, chi: int, cutoff: float):
    """n_steps second-order two-site TDVP steps of length dt, then the canonical form."""
    dm = DMRG(state, h_bonds)
    infos = []
    for _ in range(n_steps):
        infos += dm.tdvp_step(dt, chi, cutoff)
    dm.canonicalize()
    return infos


def run_dmrg(state: U1MPS, h_bonds, n_sweeps: int, chi: int, cutoff: float):
    """n_sweeps two-site sweeps, then the canonical form; returns (energies, per-step infos)."""
    dm = DMRG(state, h_bonds)
    infos = []
    for _ in range(n_sweeps):
        infos += dm.sweep(chi, cutoff)
    dm.canonicalize()
    return dm.energies, infos


# ---------------------------------------------------------------------------
# Models
# ---------------------------------------------------------------------------

def xxz_bonds(L: int, delta: float, J: float = 1.0):
    from .gates import xxz_h_blocks
    hb = xxz_h_blocks(delta, J)
    return [hb for _ in range(L - 1)]


def bh_bonds(L: int, d: int, J: float, U: float):
    from .gates import bh_h_blocks, bh_weights
    return [bh_h_blocks(d, J, U, *bh_weights(L, s)) for s in range(L - 1)]
