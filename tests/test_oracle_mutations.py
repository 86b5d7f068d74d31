"""Planted mistakes in the oracle must be caught by its pins (mutation checks, CPU only)."""
import numpy as np

import workloads as W
from oracle import U1MPS, dense, gates, tebd
from oracle import u1mps as U


def _bh_dense_error(mutate_gate=None, mutate_state=None):
    L, d, J, Uo, dt = 5, 4, 0.7, 3.0, 0.1
    occ = [2, 0, 3, 1, 0]
    st = U1MPS.product(d, occ)
    psi = dense.product_state(d, occ)
    g = tebd.bh_gates(L, d, J, Uo, dt)
    for _ in range(4):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                G = g(s, f)
                if mutate_gate:
                    G = mutate_gate(G)
                st.apply_gate2(s, G, 4096, 0.0)
                wl, wr = gates.bh_weights(L, s)
                psi = dense.apply_two_site(psi, s, dense.gate_from_h(dense.bh_two_site(d, J, Uo, wl, wr), f * dt))
    return np.max(np.abs(st.to_dense() - psi))


def test_unmutated_is_exact():
    assert _bh_dense_error() < 1e-12


def test_swapped_site_order_in_gate_is_caught():
    """Reading the gate basis as (n-i, i) instead of (i, n-i) breaks the end-weighted chain."""
    flip = lambda G: [b[::-1, ::-1] for b in G]
    assert _bh_dense_error(flip) > 1e-3


def test_conjugated_gate_is_caught():
    assert _bh_dense_error(lambda G: [b.conj() for b in G]) > 1e-3


def test_transposed_beam_splitter_is_caught():
    """Transposed Fock blocks equal a mode-phase-conjugated interferometer: multi-photon
    probabilities do not see it, the single-photon amplitude pin <e_j|U|e_i> = U_ji does."""
    M = 5
    layers = W.brickwork_pairs(M, 5)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=2)
    U_ = tebd.interferometer(M, layers, ang)
    worst = 0.0
    for i in range(M):
        st = U1MPS.product(2, [1 if k == i else 0 for k in range(M)])
        k = 0
        for sites in layers:
            for s in sites:
                G = gates.beam_splitter_gate(*ang[k], 2)
                k += 1
                st.apply_gate2(s, [b.T for b in G], 100, 0.0)
        for j in range(M):
            worst = max(worst, abs(st.amplitude([1 if q == j else 0 for q in range(M)]) - U_[j, i]))
    assert worst > 1e-3


def test_dropping_lambda_weights_is_caught(monkeypatch):
    """Truncating Theta' instead of diag(lambda) Theta' no longer keeps the Schmidt values."""
    L = 8
    occ = W.neel_occupations(L)
    st = U1MPS.product(2, occ)
    tebd.run_tebd(st, tebd.xxz_gates(L, 0.5, 0.3), 3, 1000, 0.0)
    psi = st.to_dense()
    G = gates.xxz_gate(0.5, 0.4)
    bad = st.copy()
    bad.lam[3] = {c: np.ones_like(v) for c, v in bad.lam[3].items()}
    info = bad.apply_gate2(3, G, 5, 0.0)
    psi2 = dense.apply_two_site(psi, 3, dense.gate_from_h(dense.xxz_two_site(0.5), 0.4))
    ref = np.sort(dense.schmidt_values(psi2, 4))[::-1][:5]
    got = np.sort(np.concatenate(list(info["sigmas"].values())))[::-1][:5]
    assert np.max(np.abs(ref - got)) > 1e-3
