"""Structural invariants the paper states for the U(1) MPS (Sec. II), checked on the oracle."""
import numpy as np

import workloads as W
from oracle import U1MPS, bond_charge_range, count_configs, dense, hilbert_dim, tebd
from tests.helpers import evolve_xxz_both


def _bh_state(L=8, d=4, steps=6, chi=40, cutoff=1e-10):
    st = U1MPS.product(d, W.mott_occupations(L))
    infos = tebd.run_tebd(st, tebd.bh_gates(L, d, 1.0, 2.0, 0.05), steps, chi, cutoff)
    return st, infos


def test_charge_rule_and_boundaries():
    st, infos = _bh_state()
    st.check_structure()
    assert st.bond[0] == {st.N: 1} and st.bond[st.L] == {0: 1}
    for b in range(st.L + 1):
        lo, hi = bond_charge_range(st.L, st.d, st.N, b)
        assert all(lo <= c <= hi for c in st.bond[b])


def test_theta_blocks_at_most_chi_by_chi():
    """Each Theta(c) has at most chi_{s} rows and chi_{s+2} columns (Sec. II)."""
    L, d = 8, 4
    st = U1MPS.product(d, W.mott_occupations(L))
    g = tebd.bh_gates(L, d, 1.0, 2.0, 0.05)
    for _ in range(5):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                left, right = st.bond_dim(s), st.bond_dim(s + 2)
                info = st.apply_gate2(s, g(s, f), 30, 1e-10)
                for c, (m, n) in info["sectors"].items():
                    assert m <= left and n <= right


def test_memory_reduced_by_local_dimension():
    """Stored entries of a site are at most chi_left * chi_right, a 1/d share of the dense d*chi^2."""
    st, _ = _bh_state()
    for s in range(st.L):
        assert st.site_nnz(s) <= st.bond_dim(s) * st.bond_dim(s + 1)


def test_norm_and_canonical_form_untruncated():
    L = 8
    st, psi, _ = evolve_xxz_both(L, 0.7, 0.1, 6, 1000, 0.0, W.neel_occupations(L))
    assert abs(st.norm2() - 1.0) < 1e-13
    for b in range(L + 1):
        assert abs(sum(np.sum(v ** 2) for v in st.lam[b].values()) - 1.0) < 1e-13
    for s in range(L):
        for l, Dl in st.bond[s].items():
            acc = np.zeros((Dl, Dl), dtype=complex)
            for (ll, m), blk in st.B[s].items():
                if ll == l:
                    acc += blk @ blk.conj().T
            assert np.max(np.abs(acc - np.eye(Dl))) < 1e-12


def test_right_charge_is_right_particle_number():
    """c^[k] counts particles right of bond k: <N_right(k)> = sum_c c |lambda_c|^2."""
    L = 8
    st, psi, _ = evolve_xxz_both(L, 0.5, 0.1, 5, 1000, 0.0, W.neel_occupations(L))
    for b in range(L + 1):
        from_lam = sum(c * np.sum(v ** 2) for c, v in st.lam[b].items())
        dense_val = sum(dense.density(psi, s) for s in range(b, L))
        assert abs(from_lam - dense_val) < 1e-12


def test_local_and_transfer_expectations_agree():
    st, _ = _bh_state(chi=1000, cutoff=0.0)
    for s in range(st.L):
        op = np.arange(st.d)
        assert abs(st.expect_local(s, op) - st.expect_transfer(s, op)) < 1e-12


def test_hilbert_bounds():
    assert count_configs(4, 2, 2) == 6
    assert count_configs(3, 3, 3) == 7   # compositions of 3 into 3 parts <= 2
    L, d, N = 16, 2, 8
    assert sum(hilbert_dim(L, d, N, 8, c) for c in range(N + 1)) == 256
    st, _ = _bh_state(L=6, d=3, steps=10, chi=10_000, cutoff=0.0)
    for b in range(st.L + 1):
        for c, D in st.bond[b].items():
            assert D <= hilbert_dim(st.L, st.d, st.N, b, c)


def test_layer_order_is_irrelevant():
    """Updates of one layer touch disjoint tensors: any order gives bit-identical states."""
    L, d = 8, 3
    g = tebd.bh_gates(L, d, 1.0, 2.0, 0.07)
    a = U1MPS.product(d, W.mott_occupations(L))
    tebd.run_tebd(a, g, 3, 20, 1e-10)
    b = a.copy()
    for sites, f in tebd.strang_layers(L):
        for s in sites:
            a.apply_gate2(s, g(s, f), 20, 1e-10)
        for s in reversed(sites):
            b.apply_gate2(s, g(s, f), 20, 1e-10)
    for s in range(L):
        assert a.B[s].keys() == b.B[s].keys()
        for k in a.B[s]:
            assert np.array_equal(a.B[s][k], b.B[s][k])
