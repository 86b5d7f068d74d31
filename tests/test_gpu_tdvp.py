"""Two-site TDVP on the GPU (mps_tdvp) against the oracle's (oracle/dmrg.py) and exact evolution.

From a state whose bonds are at their charge-resolved Hilbert bounds TDVP is exact: after the
steps every amplitude equals exp(-i H t) applied to the dense start vector (1e-10, global
phase included).  From a TEBD-grown Bose-Hubbard state with truncation, the GPU and the
oracle agree step by step: <H_eff> before every forward evolution to 1e-10 relative, bond
tables exactly, lambda to 1e-10, densities and entropies to 1e-9.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import U1MPS, dense, dmrg, hilbert_dim, tebd
from tests.helpers import load_state

pytestmark = pytest.mark.gpu


def test_tdvp_from_a_full_rank_state_equals_exact_evolution(gpu_lib):
    m = gpu_lib
    L, delta, dt, steps = 8, 0.5, 0.1, 3
    st = U1MPS.product(2, W.neel_occupations(L))
    tebd.run_tebd(st, tebd.xxz_gates(L, 1.3, 0.7), 8, 4096, 0.0)
    for b in range(L + 1):
        assert sum(st.bond[b].values()) == sum(hilbert_dim(L, 2, L // 2, b, c) for c in st.bond[b])
    psi0 = st.to_dense().reshape(-1)
    g = m.MPS(2, W.neel_occupations(L), 64)
    load_state(g, st)
    g.tdvp(m.models.chain_bond_terms("xxz", L, 2, delta=delta), steps, dt, 64, 0.0)
    H = np.zeros((2 ** L, 2 ** L), dtype=np.complex128)
    for k in range(L - 1):
        H += np.kron(np.kron(np.eye(2 ** k), dense.xxz_two_site(delta)), np.eye(2 ** (L - k - 2)))
    psi = scipy.linalg.expm(-1j * dt * steps * H) @ psi0
    cfgs = [c for c in itertools.product(range(2), repeat=L) if sum(c) == L // 2]
    amp = g.amplitudes(cfgs)
    idx = [int("".join(map(str, c)), 2) for c in cfgs]
    assert np.max(np.abs(amp - psi[idx])) <= 1e-10
    g.close()


def test_tdvp_with_truncation_matches_the_oracle(gpu_lib):
    m = gpu_lib
    L, d, chi, dt, steps = 10, 5, 32, 0.05, 3
    occ = W.mott_occupations(L)
    st = U1MPS.product(d, occ)
    tebd.run_tebd(st, tebd.bh_gates(L, d, 1.0, 2.0, 0.05), 5, 24, 1e-10)
    g = m.MPS(d, occ, chi)
    load_state(g, st)
    E = g.tdvp(m.models.chain_bond_terms("bh", L, d, J=1.0, U=2.0), steps, dt, chi, 1e-10)
    infos = dmrg.run_tdvp(st, dmrg.bh_bonds(L, d, 1.0, 2.0), steps, dt, chi, 1e-10)
    assert len(E) == len(infos) == steps * 2 * (L - 1)
    for b in range(L + 1):
        assert g.bond_dims(b) == st.bond[b], (b, g.bond_dims(b), st.bond[b])
        for c, v in g.bond(b).items():
            assert np.max(np.abs(v - st.lam[b][c])) <= 1e-10, (b, c)
    nop = np.arange(d, dtype=float)
    for s in range(L):
        a, r = g.expect(s, nop), st.expect_local(s, nop)
        assert abs(a - r) <= 1e-9 * max(abs(r), d - 1), (s, a, r)
    for b in range(1, L):
        assert abs(g.entropy(b) - st.entropy(b)) <= 1e-9 * max(st.entropy(b), np.log(chi))
    # the energy is conserved up to the truncation (the projected evolution conserves <H>)
    assert np.max(np.abs(E - E[0])) <= 1e-5 * abs(E[0])
    print(f"TDVP L={L} chi={chi}: <H> {E[0]:.12f} .. {E[-1]:.12f}, {g.dmrg_stats()}")
    g.close()


def test_tdvp_argument_errors(gpu_lib):
    m = gpu_lib
    L = 6
    hg = m.models.chain_bond_terms("xxz", L, 2, delta=0.5)
    g = m.MPS(2, W.neel_occupations(L), 8)
    with pytest.raises(m.MPSError):
        g.tdvp(hg, 1, 0.1, 8, 1e-10, krylov_dim=41)
    g.close()
