"""Shared test helpers: drive the oracle and the dense reference on the same schedule."""
import numpy as np

from oracle import U1MPS, dense, gates, tebd


def evolve_xxz_both(L, delta, dt, steps, chi, cutoff, occ):
    st = U1MPS.product(2, occ)
    psi = dense.product_state(2, occ)
    g = tebd.xxz_gates(L, delta, dt)
    infos = []
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            G = dense.gate_from_h(dense.xxz_two_site(delta), f * dt)
            for s in sites:
                infos.append(st.apply_gate2(s, g(s, f), chi, cutoff))
                psi = dense.apply_two_site(psi, s, G)
    return st, psi, infos


def evolve_bh_both(L, d, J, U, dt, steps, chi, cutoff, occ):
    st = U1MPS.product(d, occ)
    psi = dense.product_state(d, occ)
    g = tebd.bh_gates(L, d, J, U, dt)
    infos = []
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                infos.append(st.apply_gate2(s, g(s, f), chi, cutoff))
                wl, wr = gates.bh_weights(L, s)
                psi = dense.apply_two_site(psi, s, dense.gate_from_h(dense.bh_two_site(d, J, U, wl, wr), f * dt))
    return st, psi, infos


def rel_close(a, b, scale, tol):
    return abs(a - b) <= tol * max(abs(b), scale)
