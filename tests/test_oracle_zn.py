"""Pins of the Z_n oracle (oracle/znmps.py) against dense state-vector evolution.

Sec. I of arXiv:2303.11409 names more general Abelian symmetries beside U(1); the Z_n
clock chain (n = 2: the transverse-field Ising chain in the basis where the field is
diagonal) is the example.  The dense side builds its two-site Hamiltonians from clock
operators by Kronecker products and exponentiates them with scipy's expm; the oracle
builds charge blocks by index loops and exponentiates each by eigh.  Untruncated, both
must agree to rounding: amplitudes (no gauge freedom), local <X + X^dag> and bond entropies.
"""
import numpy as np
import pytest

from oracle import dense, gates
from oracle.znmps import ZnMPS


def _schedule(L):
    odd = list(range(0, L - 1, 2))
    even = list(range(1, L - 1, 2))
    return [(odd, 0.5), (even, 1.0), (odd, 0.5)]


def _run(n, L, occ, J, f, dt, steps, chi):
    st = ZnMPS.product(n, occ)
    psi = dense.product_state(n, occ)
    for _ in range(steps):
        for sites, frac in _schedule(L):
            for s in sites:
                st.apply_gate2(s, gates.clock_gate(L, s, n, J, f, frac * dt), chi, 0.0)
                wl, wr = gates.bh_weights(L, s)
                psi = dense.apply_two_site(psi, s, dense.gate_from_h(dense.clock_two_site(n, J, f, wl, wr),
                                                                     frac * dt))
    return st, psi


def test_clock_blocks_are_the_dense_operator_restricted_to_each_charge():
    for n in (2, 3, 4):
        h = dense.clock_two_site(n, 1.3, 0.7, 0.5, 1.0)
        blocks = gates.clock_h_blocks(n, 1.3, 0.7, 0.5, 1.0)
        q_of = np.array([(i + j) % n for i in range(n) for j in range(n)])
        # the dense operator is block diagonal in the Z_n charge
        assert np.max(np.abs(h[q_of[:, None] != q_of[None, :]])) == 0.0
        for q in range(n):
            idx = [i * n + (q - i) % n for i in range(n)]
            assert np.allclose(h[np.ix_(idx, idx)], blocks[q], atol=0, rtol=0)


@pytest.mark.parametrize("n,L,occ,J,f,steps", [
    (2, 8, [0] * 8, 1.0, 0.8, 6),             # transverse-field Ising from |++...+>
    (2, 7, [0, 1, 0, 0, 1, 1, 0], 1.0, 1.3, 5),
    (3, 6, [0, 1, 2, 0, 1, 2], 1.0, 0.6, 4),  # Z_3 clock chain
    (4, 5, [1, 0, 3, 2, 0], 0.7, 1.1, 3),
])
def test_untruncated_zn_tebd_equals_dense_evolution(n, L, occ, J, f, steps):
    st, psi = _run(n, L, occ, J, f, 0.1, steps, chi=10 ** 6)
    # norm preserved, charge of every block consistent with its bond charges
    for b in range(1, L):
        assert abs(sum(float(np.sum(v ** 2)) for v in st.lam[b].values()) - 1.0) < 1e-12
    xs = 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
    for s in range(L):
        assert abs(st.expect_local(s, xs) - dense.mean_op(psi, s, xs)) < 1e-11
    for b in range(1, L):
        assert abs(st.entropy(b) - dense.bond_entropy(psi, b)) < 1e-10
    rng = np.random.default_rng(3)
    for _ in range(20):
        cfg = rng.integers(0, n, size=L)
        assert abs(st.amplitude(cfg) - psi[tuple(cfg)]) < 1e-12
    # the Z_n charge is conserved: amplitudes of the other charge classes vanish exactly
    q0 = sum(occ) % n
    p = np.abs(psi) ** 2
    tot = np.indices(psi.shape).sum(axis=0) % n
    assert np.all(p[tot != q0] < 1e-28)


def test_truncated_zn_run_keeps_the_largest_schmidt_values():
    n, L = 2, 10
    st, psi = _run(n, L, [0] * L, 1.0, 0.9, 0.1, 6, chi=6)
    assert max(sum(st.bond[b].values()) for b in range(L + 1)) == 6
    # the kept spectrum at the middle bond approximates the dense Schmidt values
    sv = dense.schmidt_values(psi, L // 2)
    lam = np.sort(np.concatenate(list(st.lam[L // 2].values())))[::-1]
    assert np.max(np.abs(lam[:3] - sv[:3] / np.linalg.norm(sv))) < 1e-3


def test_planted_sign_mistake_in_the_physical_index_is_caught():
    """Reading the physical index as (m - l) mod n instead of (l - m) mod n (a plausible slip)
    breaks the dense agreement for n = 3."""
    n, L, occ = 3, 5, [0, 1, 2, 1, 0]

    class Wrong(ZnMPS):
        def apply_gate2(self, s, G, chi, cutoff):
            # conjugating the charge labels of the gate blocks models the slip
            Gw = [G[(-q) % n] for q in range(n)]
            return super().apply_gate2(s, Gw, chi, cutoff)

    st = Wrong.product(n, occ)
    psi = dense.product_state(n, occ)
    for sites, frac in _schedule(L):
        for s in sites:
            st.apply_gate2(s, gates.clock_gate(L, s, n, 1.0, 0.6, frac * 0.2), 10 ** 6, 0.0)
            wl, wr = gates.bh_weights(L, s)
            psi = dense.apply_two_site(psi, s, dense.gate_from_h(dense.clock_two_site(n, 1.0, 0.6, wl, wr),
                                                                 frac * 0.2))
    err = max(abs(st.amplitude(c) - psi[tuple(c)]) for c in np.ndindex(*psi.shape))
    assert err > 1e-3
