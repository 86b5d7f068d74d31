"""Pins the oracle's whole update against dense state-vector evolution.

The dense side builds two-site Hamiltonians from ladder operators and
exponentiates them with scipy.linalg.expm, so it shares neither the charge
blocks nor the eigh-based gate blocks with the oracle.
"""
import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, dense, gates, tebd
from tests.helpers import evolve_bh_both, evolve_xxz_both


def test_xxz_untruncated_matches_dense():
    L = 10
    st, psi, _ = evolve_xxz_both(L, 0.5, 0.05, 20, 64, 0.0, W.neel_occupations(L))
    st.check_structure()
    for s in range(L):
        assert abs(st.expect_local(s, [-0.5, 0.5]) - (dense.density(psi, s) - 0.5)) < 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - dense.bond_entropy(psi, b)) < 1e-12
    assert np.max(np.abs(st.to_dense() - psi)) < 1e-12


@pytest.mark.slow
def test_xxz_L16_cfg1_untruncated_matches_dense():
    """XXZ L=16, Delta=0.5, Neel, dt=0.05 x 20: chi=256 is the exact middle-bond bound."""
    L = 16
    st, psi, infos = evolve_xxz_both(L, 0.5, 0.05, 20, 256, 0.0, W.neel_occupations(L))
    assert len(infos) == 460
    for s in range(L):
        assert abs(st.expect_local(s, [-0.5, 0.5]) - (dense.density(psi, s) - 0.5)) < 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - dense.bond_entropy(psi, b)) < 1e-11


@pytest.mark.slow
def test_xxz_L16_chi64_within_truncation_bound():
    """At chi=64 the deviation from the exact state is bounded by the discarded weight.

    Each update moves the normalised state by at most 2 sqrt(eps_u); a normalised
    expectation of an operator of norm |O| then moves by at most 2 |O| times that.
    """
    L = 16
    st, psi, infos = evolve_xxz_both(L, 0.5, 0.05, 20, 64, 1e-10, W.neel_occupations(L))
    bound = 2 * 0.5 * sum(2 * np.sqrt(i["trunc_err"]) for i in infos)
    dev = max(abs(st.expect_local(s, [-0.5, 0.5]) - (dense.density(psi, s) - 0.5)) for s in range(L))
    assert dev <= bound + 1e-12
    assert max(st.bond_dim(b) for b in range(L + 1)) <= 64


def test_bose_hubbard_matches_dense():
    L, d = 6, 5
    occ = W.mott_occupations(L)
    st, psi, _ = evolve_bh_both(L, d, 1.0, 2.0, 0.05, 8, 4096, 0.0, occ)
    for s in range(L):
        assert abs(st.expect_local(s, np.arange(d)) - dense.density(psi, s)) < 1e-12
    assert np.max(np.abs(st.to_dense() - psi)) < 1e-12


def test_bose_hubbard_end_weights_matter():
    """Non-uniform occupations and the chain-end weights make the gate asymmetric."""
    L, d = 5, 4
    occ = [2, 0, 3, 1, 0]
    st, psi, _ = evolve_bh_both(L, d, 0.7, 3.0, 0.1, 5, 4096, 0.0, occ)
    assert np.max(np.abs(st.to_dense() - psi)) < 1e-12


def test_bose_hubbard_J0_phases():
    """J=0: occupations are frozen and each Fock amplitude picks up exp(-i U/2 sum n(n-1) t)."""
    L, d, U, dt, steps = 6, 4, 1.7, 0.1, 7
    occ = [2, 0, 3, 1, 1, 2]
    st = U1MPS.product(d, occ)
    tebd.run_tebd(st, tebd.bh_gates(L, d, 0.0, U, dt), steps, 64, 1e-10)
    t = steps * dt
    expected = np.exp(-1j * 0.5 * U * sum(n * (n - 1) for n in occ) * t)
    assert abs(st.amplitude(occ) - expected) < 1e-13
    for s in range(L):
        assert abs(st.expect_local(s, np.arange(d)) - occ[s]) < 1e-13


def test_free_bosons_U0():
    """U=0, n_max >= N: <n_i> = sum_j |W_ij|^2 n_j(0) with W the Trotterised 1-particle propagator."""
    L, d, J, dt, steps = 5, 5, 1.0, 0.1, 6
    occ = [2, 0, 1, 1, 0]
    st = U1MPS.product(d, occ)
    tebd.run_tebd(st, tebd.bh_gates(L, d, J, 0.0, dt), steps, 4096, 0.0)
    Wm = np.eye(L, dtype=complex)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            tau = f * dt
            w2 = np.cos(J * tau) * np.eye(2) + 1j * np.sin(J * tau) * np.array([[0, 1], [1, 0]])
            for s in sites:
                E = np.eye(L, dtype=complex)
                E[s:s + 2, s:s + 2] = w2
                Wm = E @ Wm
    expect = (np.abs(Wm) ** 2) @ np.array(occ, dtype=float)
    for s in range(L):
        assert abs(st.expect_local(s, np.arange(d)) - expect[s]) < 1e-12


def test_sigmas_are_schmidt_values():
    """Before truncation the pooled sigmas are the dense Schmidt values of G|psi> at the bond."""
    L = 8
    occ = W.neel_occupations(L)
    st, psi, _ = evolve_xxz_both(L, 0.5, 0.3, 3, 1000, 0.0, occ)
    s = 3
    G = gates.xxz_gate(0.5, 0.4)
    info = st.apply_gate2(s, G, 5, 0.0)
    psi2 = dense.apply_two_site(psi, s, dense.gate_from_h(dense.xxz_two_site(0.5), 0.4))
    ref = np.sort(dense.schmidt_values(psi2, s + 1))[::-1]
    got = np.sort(np.concatenate(list(info["sigmas"].values())))[::-1]
    k = min(len(ref), len(got))
    assert np.max(np.abs(ref[:k] - got[:k])) < 1e-12
    assert np.all(ref[k:] < 1e-12) and np.all(got[k:] < 1e-12)
    # the kept lambdas are the top chi of them, renormalised
    lam = np.sort(np.concatenate(list(st.lam[s + 1].values())))[::-1]
    assert len(lam) == 5
    assert np.max(np.abs(lam - ref[:5] / np.linalg.norm(ref[:5]))) < 1e-12
