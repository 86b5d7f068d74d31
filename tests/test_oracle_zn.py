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


# ---- Z_n with d < n: a U(1) model also conserves its particle number mod n ---------------

def _bh_dense_gate(L, s, d, J, U, tau):
    wl, wr = gates.bh_weights(L, s)
    return dense.gate_from_h(dense.bh_two_site(d, J, U, wl, wr), tau)


def test_cyclic_gate_blocks_join_the_u1_totals_of_one_residue():
    """d = 3, n = 4: residue 0 joins the pairs (0, 0) and (2, 2) (totals 0 and 4), residue 1 the
    pairs (0, 1), (1, 0) and residue 3 (1, 2), (2, 1); the dense gate has no entry between
    different totals, and each block equals the dense gate on its pairs."""
    from oracle.znmps import gate_blocks_from_dense, gate_blocks_from_u1, zn_blocks_of, zn_charges
    d, n, L = 3, 4, 6
    G = _bh_dense_gate(L, 2, d, 1.0, 2.0, 0.07)
    assert zn_charges(n, d) == [0, 1, 2, 3]
    assert zn_blocks_of(n, 0, d) == [(0, 0), (2, 2)]
    assert zn_blocks_of(n, 2, d) == [(0, 2), (1, 1), (2, 0)]
    blocks = gate_blocks_from_dense(G, n, d)
    assert blocks[0][0, 1] == 0 and blocks[0][1, 0] == 0
    assert blocks[0][0, 0] == G[0, 0] and blocks[0][1, 1] == G[8, 8]
    # the same blocks from the U(1) gate (eigh per total) agree to rounding
    u1 = gates.bh_gate(L, 2, d, 1.0, 2.0, 0.07)
    for q, b in gate_blocks_from_u1(u1, n, d).items():
        assert np.max(np.abs(b - blocks[q])) < 1e-13


@pytest.mark.parametrize("d,n,L,occ", [
    (3, 4, 6, [1, 0, 2, 1, 0, 1]),
    (3, 5, 6, [2, 0, 2, 1, 2, 0]),
    (2, 3, 8, [1, 0, 1, 1, 0, 0, 1, 0]),
])
def test_untruncated_zn_with_d_below_n_equals_dense_evolution(d, n, L, occ):
    from oracle.znmps import gate_blocks_from_dense
    J, U, dt, steps = 1.0, 2.0, 0.1, 3
    st = ZnMPS.product(n, occ, d=d)
    psi = dense.product_state(d, occ)
    for _ in range(steps):
        for sites, frac in _schedule(L):
            for s in sites:
                G = _bh_dense_gate(L, s, d, J, U, frac * dt)
                st.apply_gate2(s, gate_blocks_from_dense(G, n, d), 10 ** 6, 0.0)
                psi = dense.apply_two_site(psi, s, G)
    nop = np.arange(d, dtype=float)
    for s in range(L):
        assert abs(st.expect_local(s, nop) - dense.mean_op(psi, s, nop)) < 1e-11
    for b in range(1, L):
        assert abs(st.entropy(b) - dense.bond_entropy(psi, b)) < 1e-10
    rng = np.random.default_rng(5)
    for _ in range(20):
        cfg = rng.integers(0, d, size=L)
        assert abs(st.amplitude(cfg) - psi[tuple(cfg)]) < 1e-12
    # some bond carries more U(1) charges (particles right of it, with weight) than Z_n sectors:
    # charges c and c + n share one Z_n sector there
    occ_idx = np.indices(psi.shape)
    p = np.abs(psi) ** 2
    merged = False
    for b in range(1, L):
        right = occ_idx[b:].sum(axis=0)
        charges = {int(c) for c in np.unique(right) if p[right == c].sum() > 1e-20}
        merged = merged or len(charges) > len(st.bond[b])
    assert merged


def test_truncated_zn_with_d_below_n_equals_the_u1_run():
    """With truncation the Z_n run of a Bose-Hubbard chain is the U(1) run in coarser blocks:
    each Theta(c) of the Z_n update is a direct sum of the U(1) blocks of charges c + kn, so
    the pooled singular values, the kept set and the state are the same (no ties at the cuts
    of this asymmetric start): per bond the sorted Schmidt values agree to 1e-12, the Z_n
    dimensions are the U(1) ones summed per residue, densities and entropies agree."""
    from oracle import U1MPS
    from oracle.znmps import gate_blocks_from_u1
    d, n, L, chi, steps = 3, 4, 10, 12, 4
    occ = [2, 0, 1, 1, 0, 2, 1, 1, 0, 1]
    J, U, dt = 1.0, 2.0, 0.1
    zs = ZnMPS.product(n, occ, d=d)
    us = U1MPS.product(d, occ)
    cut_seen = False
    for _ in range(steps):
        for sites, frac in _schedule(L):
            for s in sites:
                u1 = gates.bh_gate(L, s, d, J, U, frac * dt)
                us.apply_gate2(s, u1, chi, 1e-10)
                zs.apply_gate2(s, gate_blocks_from_u1(u1, n, d), chi, 1e-10)
            for b in range(L + 1):
                merged = {}
                for c, k in us.bond[b].items():
                    merged[c % n] = merged.get(c % n, 0) + k
                assert zs.bond[b] == merged, (b, zs.bond[b], us.bond[b])
                lz = np.sort(np.concatenate(list(zs.lam[b].values())))
                lu = np.sort(np.concatenate(list(us.lam[b].values())))
                assert np.max(np.abs(lz - lu)) < 1e-12
                cut_seen = cut_seen or sum(us.bond[b].values()) == chi
    assert cut_seen, "the chi cut never became active"
    nop = np.arange(d, dtype=float)
    for s in range(L):
        assert abs(zs.expect_local(s, nop) - us.expect_local(s, nop)) < 1e-10
    for b in range(1, L):
        assert abs(zs.entropy(b) - us.entropy(b)) < 1e-10


def test_planted_wrong_residue_block_fails_the_dense_pin():
    """Swapping the two pairs of residue 0 (a wrong gate position for d < n) breaks the pin."""
    from oracle.znmps import gate_blocks_from_dense
    d, n, L, occ = 3, 4, 6, [1, 0, 2, 1, 0, 1]
    st = ZnMPS.product(n, occ, d=d)
    psi = dense.product_state(d, occ)
    for sites, frac in _schedule(L):
        for s in sites:
            G = _bh_dense_gate(L, s, d, 1.0, 2.0, frac * 0.1)
            blocks = gate_blocks_from_dense(G, n, d)
            blocks[0] = blocks[0][::-1, ::-1].copy()
            st.apply_gate2(s, blocks, 10 ** 6, 0.0)
            psi = dense.apply_two_site(psi, s, G)
    rng = np.random.default_rng(5)
    cfgs = [rng.integers(0, d, size=L) for _ in range(200)]
    assert max(abs(st.amplitude(c) - psi[tuple(c)]) for c in cfgs) > 1e-6
