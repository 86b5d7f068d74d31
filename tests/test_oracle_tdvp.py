"""Pins of the two-site TDVP of the oracle (oracle/dmrg.py, DMRG.tdvp_step).

- From a state whose every bond is at its charge-resolved Hilbert bound, the tangent space is the
  whole space, so TDVP is exact: it equals exp(-i H t) applied to the dense vector (no Trotter
  error), global phase included.
- Without truncation it conserves the norm and <H> (the projected equations are symplectic),
  also from a product state whose bonds grow during the evolution.
- A planted mistake (the backward single-site step run forward) fails the exact pin.
"""
import numpy as np
import scipy.linalg

import workloads as W
from oracle import U1MPS, dense, dmrg, hilbert_dim, tebd


def _xxz_dense(L, delta):
    H = np.zeros((2 ** L, 2 ** L), dtype=np.complex128)
    for k in range(L - 1):
        H += np.kron(np.kron(np.eye(2 ** k), dense.xxz_two_site(delta)), np.eye(2 ** (L - k - 2)))
    return H


def _full_rank_state(L):
    st = U1MPS.product(2, W.neel_occupations(L))
    tebd.run_tebd(st, tebd.xxz_gates(L, 1.3, 0.7), 6, 4096, 0.0)
    for b in range(L + 1):
        assert sum(st.bond[b].values()) == sum(hilbert_dim(L, 2, L // 2, b, c) for c in st.bond[b])
    return st


def test_tdvp_from_a_full_rank_state_is_exact():
    L, delta, dt, steps = 6, 0.5, 0.1, 4
    st = _full_rank_state(L)
    psi0 = st.to_dense().reshape(-1).copy()
    dmrg.run_tdvp(st, dmrg.xxz_bonds(L, delta), steps, dt, 4096, 0.0)
    psi = scipy.linalg.expm(-1j * dt * steps * _xxz_dense(L, delta)) @ psi0
    assert np.max(np.abs(st.to_dense().reshape(-1) - psi)) <= 1e-12


def test_tdvp_conserves_norm_and_energy():
    L, delta, dt, steps = 10, 0.5, 0.05, 6
    st = U1MPS.product(2, W.neel_occupations(L))
    H = _xxz_dense(L, delta)
    psi0 = st.to_dense().reshape(-1)
    e0 = np.vdot(psi0, H @ psi0).real
    dmrg.run_tdvp(st, dmrg.xxz_bonds(L, delta), steps, dt, 4096, 0.0)
    psi = st.to_dense().reshape(-1)
    assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-12
    assert abs(np.vdot(psi, H @ psi).real - e0) <= 1e-11
    assert max(sum(st.bond[b].values()) for b in range(L + 1)) > 1


def test_planted_forward_backward_step_fails_the_exact_pin():
    L, delta, dt, steps = 6, 0.5, 0.1, 2
    st = _full_rank_state(L)
    psi0 = st.to_dense().reshape(-1).copy()
    dm = dmrg.DMRG(st, dmrg.xxz_bonds(L, delta))
    good = dm._backward
    dm._backward = lambda j, tau: good(j, -tau)
    for _ in range(steps):
        dm.tdvp_step(dt, 4096, 0.0)
    dm.canonicalize()
    psi = scipy.linalg.expm(-1j * dt * steps * _xxz_dense(L, delta)) @ psi0
    assert np.max(np.abs(st.to_dense().reshape(-1) - psi)) > 1e-3
