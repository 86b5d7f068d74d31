"""Pins of the two-site DMRG oracle (oracle/dmrg.py) against what the physics fixes.

- The operator split h = sum_t O_t (x) P_t of a bond term equals the two-site
  Hamiltonian built independently from ladder operators (oracle/dense.py), and each
  O_t shifts the charge by a single delta_t.
- Untruncated DMRG ground energies equal exact diagonalisation in the charge sector
  (XXZ L=10, Bose-Hubbard L=6 with chain-end weights), and the final state is an
  eigenvector of the dense Hamiltonian.
- The XX chain (Delta = 0) is free fermions: the ground energy is the sum of the N
  lowest single-particle levels -cos(k pi / (L + 1)) (hopping 1/2).
- U = 0 bosons with n_max >= N: N times the lowest level -2J cos(pi / (L + 1)).
- The canonical form after the sweeps: right-canonical blocks, Schmidt lambdas equal
  the dense state's, unit norm; energies never rise over a sweep beyond rounding.
- Planted mistakes (a dropped boundary term, a transposed operator) fail the ED pin.
"""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, dense, dmrg, gates


def _chain_h(L, two_site):
    d = int(round(np.sqrt(two_site(0).shape[0])))
    H = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for k in range(L - 1):
        H += np.kron(np.kron(np.eye(d ** k), two_site(k)), np.eye(d ** (L - k - 2)))
    return H


def _sector(L, d, N):
    cfgs = list(itertools.product(range(d), repeat=L))
    return np.array([k for k, c in enumerate(cfgs) if sum(c) == N])


def _ed(L, d, N, two_site):
    H = _chain_h(L, two_site)
    idx = _sector(L, d, N)
    return np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0], H


@pytest.mark.parametrize("which", ["xxz", "bh", "bh_edge"])
def test_split_equals_ladder_operator_hamiltonian(which):
    if which == "xxz":
        d, hb, ref = 2, gates.xxz_h_blocks(0.7), dense.xxz_two_site(0.7)
    else:
        d = 5
        wl, wr = (1.0, 0.5) if which == "bh_edge" else (0.5, 0.5)
        hb, ref = gates.bh_h_blocks(d, 1.3, 2.1, wl, wr), dense.bh_two_site(d, 1.3, 2.1, wl, wr)
    terms = dmrg.split_bond_term(hb, d)
    S = sum(np.kron(O, P) for _, O, P in terms)
    assert np.max(np.abs(S - ref)) <= 1e-13
    for delta, O, P in terms:
        i2, i = np.nonzero(O)
        assert np.all(i2 - i == delta)
        j2, j = np.nonzero(P)
        assert np.all(j2 - j == -delta)


def test_xxz_L10_ground_energy_equals_exact_diagonalisation():
    L, delta = 10, 0.5
    st = U1MPS.product(2, W.neel_occupations(L))
    E, _ = dmrg.run_dmrg(st, dmrg.xxz_bonds(L, delta), 3, 32, 1e-12)
    e0, H = _ed(L, 2, L // 2, lambda k: dense.xxz_two_site(delta))
    assert abs(E[-1] - e0) <= 1e-10 * abs(e0)
    psi = st.to_dense().reshape(-1)
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-12
    assert np.linalg.norm(H @ psi - e0 * psi) <= 1e-8
    # lambdas are the Schmidt values of the dense state
    full = st.to_dense()
    for b in range(1, L):
        sv = np.sort(dense.schmidt_values(full, b))[::-1]
        lam = np.sort(np.concatenate(list(st.lam[b].values())))[::-1]
        assert np.max(np.abs(sv[:len(lam)] - lam)) <= 1e-10
        assert np.all(sv[len(lam):] <= 1e-10)


def test_bose_hubbard_L6_ground_energy_equals_exact_diagonalisation():
    L, d, J, U = 6, 5, 1.0, 2.0
    st = U1MPS.product(d, W.mott_occupations(L))
    E, _ = dmrg.run_dmrg(st, dmrg.bh_bonds(L, d, J, U), 3, 64, 1e-12)
    e0, H = _ed(L, d, L, lambda k: dense.bh_two_site(d, J, U, *gates.bh_weights(L, k)))
    assert abs(E[-1] - e0) <= 1e-10 * abs(e0)
    psi = st.to_dense().reshape(-1)
    assert np.linalg.norm(H @ psi - e0 * psi) <= 1e-8
    st.check_structure()


def test_xx_chain_free_fermion_ground_energy():
    L, N = 12, 6
    st = U1MPS.product(2, W.neel_occupations(L))
    E, _ = dmrg.run_dmrg(st, dmrg.xxz_bonds(L, 0.0), 3, 64, 1e-12)
    levels = np.sort(-np.cos(np.arange(1, L + 1) * np.pi / (L + 1)))
    assert abs(E[-1] - np.sum(levels[:N])) <= 1e-10


def test_free_bosons_ground_energy():
    L, d, N = 6, 5, 3
    occ = [1, 0, 1, 0, 1, 0]
    st = U1MPS.product(d, occ)
    E, _ = dmrg.run_dmrg(st, dmrg.bh_bonds(L, d, 1.0, 0.0), 3, 64, 1e-12)
    assert abs(E[-1] - N * (-2.0 * np.cos(np.pi / (L + 1)))) <= 1e-10


def test_canonical_form_and_monotone_energy_with_truncation():
    L, d = 12, 5
    st = U1MPS.product(d, W.mott_occupations(L))
    E, infos = dmrg.run_dmrg(st, dmrg.bh_bonds(L, d, 1.0, 2.0), 2, 16, 1e-10)
    # the variational energy does not rise from one local step to the next by more than
    # the truncation of the step before can (chi = 16 truncates here): dropping a weight
    # eps of |psi|^2 moves <H> by at most about 2 |H| eps
    for k in range(1, len(E)):
        assert E[k] <= E[k - 1] + 4.0 * abs(E[k - 1]) * infos[k - 1]["trunc_err"] + 1e-12, k
    assert E[-1] < E[L - 2]               # the second sweep improves on the first pass
    st.check_structure()
    for b in range(L + 1):
        assert abs(sum(float(v @ v) for v in st.lam[b].values()) - 1.0) <= 1e-12
    for s in range(L):
        # right-canonical: sum_r B(m, r) B(m, r)^dag = 1 per left sector
        acc = {}
        for (l, m), blk in st.B[s].items():
            acc[l] = acc.get(l, 0) + blk @ blk.conj().T
        for l, a in acc.items():
            assert np.max(np.abs(a - np.eye(a.shape[0]))) <= 1e-11
        # Vidal: diag(lambda_s) B has orthogonal columns of norm lambda_{s+1}
        cols = {}
        for (l, m), blk in st.B[s].items():
            cols.setdefault(m, []).append(st.lam[s][l][:, None] * blk)
        for m, parts in cols.items():
            M = np.vstack(parts)
            G = M.conj().T @ M
            assert np.max(np.abs(G - np.diag(st.lam[s + 1][m] ** 2))) <= 1e-11


def test_planted_mistakes_fail_the_ed_pin():
    L, delta = 8, 0.5
    e0, _ = _ed(L, 2, L // 2, lambda k: dense.xxz_two_site(delta))
    good = dmrg.run_dmrg(U1MPS.product(2, W.neel_occupations(L)), dmrg.xxz_bonds(L, delta), 2, 16, 1e-12)[0][-1]
    assert abs(good - e0) <= 1e-10 * abs(e0)

    # the boundary coupling between the left block and the centre dropped
    class NoLeft(dmrg.DMRG):
        def _apply(self, s, lay, X):
            keep = self.terms[s - 1] if s >= 1 else None
            if s >= 1:
                self.terms[s - 1] = []
            try:
                return super()._apply(s, lay, X)
            finally:
                if s >= 1:
                    self.terms[s - 1] = keep
    dm = NoLeft(U1MPS.product(2, W.neel_occupations(L)), dmrg.xxz_bonds(L, delta))
    for _ in range(2):
        dm.sweep(16, 1e-12)
    assert abs(dm.energies[-1] - e0) > 1e-3

    # the right boundary coupling taken from the centre bond instead of bond s+1 (an
    # off-by-one bond index; Bose-Hubbard bonds differ by their chain-end weights)
    Lb, d, J, U = 6, 3, 1.0, 2.0
    eb, _ = _ed(Lb, d, Lb, lambda k: dense.bh_two_site(d, J, U, *gates.bh_weights(Lb, k)))

    class OffByOne(dmrg.DMRG):
        def _apply(self, s, lay, X):
            if s + 1 > self.st.L - 2:
                return super()._apply(s, lay, X)
            keep = self.terms[s + 1]
            self.terms[s + 1] = self.terms[s]
            try:
                return super()._apply(s, lay, X)
            finally:
                self.terms[s + 1] = keep
    good = dmrg.run_dmrg(U1MPS.product(d, W.mott_occupations(Lb)), dmrg.bh_bonds(Lb, d, J, U), 2, 32, 1e-12)[0][-1]
    assert abs(good - eb) <= 1e-10 * abs(eb)
    dm = OffByOne(U1MPS.product(d, W.mott_occupations(Lb)), dmrg.bh_bonds(Lb, d, J, U))
    for _ in range(2):
        dm.sweep(32, 1e-12)
    assert abs(dm.energies[-1] - eb) > 1e-6
