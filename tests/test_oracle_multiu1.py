"""Pins of the several-U(1) oracle (oracle/multiu1.py) against what the physics fixes.

- The two-species hard-core boson bond term equals the one built from ladder operators
  with Kronecker products, and conserves both particle numbers.
- Untruncated TEBD equals dense state-vector evolution (amplitudes, densities of both
  species, bond entropies).
- With U = 0 the species decouple into two XX chains: densities and bond entropies equal
  the free-fermion closed form (entropies add).
- With no down particles the run equals the single-U(1) oracle's XX chain.
- A planted slip (the pair order of a gate block reversed) fails the dense pin.
"""
import numpy as np
import scipy.linalg

from oracle import U1MPS, dense, freefermion, gates, multiu1, tebd

Q = multiu1.TWO_SPECIES_Q


def _ladder_h(J, U, wl, wr):
    b = np.array([[0.0, 1.0], [0.0, 0.0]])
    e2 = np.eye(2)
    bu, bd = np.kron(b, e2), np.kron(e2, b)          # index 2 n_up + n_down
    nn = (bu.T @ bu) @ (bd.T @ bd)
    e4 = np.eye(4)
    hop = sum(np.kron(x.T, x) + np.kron(x, x.T) for x in (bu, bd))
    return -J * hop + U * (wl * np.kron(nn, e4) + wr * np.kron(e4, nn))


def _weights(L, s):
    return gates.bh_weights(L, s)


def test_bond_term_equals_ladder_construction_and_conserves_both_charges():
    for J, U, wl, wr in [(1.0, 2.0, 0.5, 0.5), (0.7, -1.3, 1.0, 0.5)]:
        H = multiu1.two_species_h(J, U, wl, wr)
        assert np.array_equal(H, H.T)
        assert np.max(np.abs(H - _ladder_h(J, U, wl, wr))) <= 1e-15
        for a in range(16):
            for c in range(16):
                if H[a, c] != 0:
                    qa = np.add(Q[a // 4], Q[a % 4])
                    qc = np.add(Q[c // 4], Q[c % 4])
                    assert tuple(qa) == tuple(qc)


def _dense_run(L, occ, J, U, dt, steps):
    psi = dense.product_state(4, occ)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                G = scipy.linalg.expm(-1j * f * dt * _ladder_h(J, U, *_weights(L, s)))
                psi = dense.apply_two_site(psi, s, G)
    return psi


def _mps_run(L, occ, J, U, dt, steps, chi=4096, cutoff=0.0, gate=None):
    st = multiu1.MultiU1MPS.product(Q, occ)
    gate = gate or multiu1.two_species_gate
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                st.apply_gate2(s, gate(J, U, *_weights(L, s), f * dt), chi, cutoff)
    return st


def _dense_from_mps(st):
    L = st.L
    psi = np.zeros((4,) * L, dtype=np.complex128)
    for idx in np.ndindex(*(4,) * L):
        psi[idx] = st.amplitude(idx)
    return psi


def test_untruncated_tebd_equals_dense_evolution():
    L, J, U, dt, steps = 5, 1.0, 2.0, 0.1, 4
    occ = [3, 0, 1, 2, 0]
    st = _mps_run(L, occ, J, U, dt, steps)
    st.check_structure()
    psi = _dense_run(L, occ, J, U, dt, steps)
    mp = _dense_from_mps(st)
    assert np.max(np.abs(mp - psi)) <= 1e-12
    nu, nd = np.array([q[0] for q in Q], float), np.array([q[1] for q in Q], float)
    for s in range(L):
        assert abs(st.expect_local(s, nu) - dense.mean_op(psi, s, nu)) <= 1e-12
        assert abs(st.expect_local(s, nd) - dense.mean_op(psi, s, nd)) <= 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - dense.bond_entropy(psi, b)) <= 1e-11
    # both particle numbers stay fixed: every bond charge is the pair (N_up, N_down) to its right
    assert st.N == (2, 2)


def test_decoupled_species_are_two_free_fermion_chains():
    L, dt, steps = 8, 0.1, 6
    occ = [2, 1, 3, 0, 2, 1, 0, 3]
    up = [Q[i][0] for i in occ]
    dn = [Q[i][1] for i in occ]
    st = _mps_run(L, occ, -0.5, 0.0, dt, steps)
    fu, fd = freefermion.FreeFermions(up), freefermion.FreeFermions(dn)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                fu.apply(s, f * dt)
                fd.apply(s, f * dt)
    nu, nd = np.array([q[0] for q in Q], float), np.array([q[1] for q in Q], float)
    for s in range(L):
        assert abs(st.expect_local(s, nu) - fu.densities()[s]) <= 1e-12
        assert abs(st.expect_local(s, nd) - fd.densities()[s]) <= 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - (fu.entropy(b) + fd.entropy(b))) <= 1e-11


def test_single_species_reduces_to_the_u1_oracle():
    L, dt, steps = 8, 0.07, 5
    occ = [2, 0, 2, 0, 2, 0, 2, 0]                    # up particles only
    st = _mps_run(L, occ, -0.5, 3.0, dt, steps)
    u1 = U1MPS.product(2, [Q[i][0] for i in occ])
    g = tebd.xxz_gates(L, 0.0, dt)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                u1.apply_gate2(s, g(s, f), 4096, 0.0)
    nu = np.array([q[0] for q in Q], float)
    for s in range(L):
        assert abs(st.expect_local(s, nu) - u1.expect_local(s, [0, 1])) <= 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - u1.entropy(b)) <= 1e-12


def test_planted_pair_order_slip_fails_the_dense_pin():
    L, J, U, dt, steps = 4, 1.0, 2.0, 0.1, 2
    occ = [3, 0, 1, 2]

    def reversed_gate(*a):
        G = multiu1.two_species_gate(*a)
        return {k: v[::-1, ::-1].T.copy() if v.shape[0] > 1 else v for k, v in G.items()}
    st = _mps_run(L, occ, J, U, dt, steps, gate=reversed_gate)
    psi = _dense_run(L, occ, J, U, dt, steps)
    assert np.max(np.abs(_dense_from_mps(st) - psi)) > 1e-3
