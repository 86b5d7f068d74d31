"""Pins the oracle against the free-fermion closed form of the Trotterised XX chain."""
import numpy as np

import workloads as W
from oracle import U1MPS, freefermion, tebd


def test_xx_quench_matches_free_fermions():
    L, dt, steps = 12, 0.05, 20
    occ = W.neel_occupations(L)
    st = U1MPS.product(2, occ)
    ff = freefermion.FreeFermions(occ)
    g = tebd.xxz_gates(L, 0.0, dt)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                st.apply_gate2(s, g(s, f), 4096, 0.0)
                ff.apply(s, f * dt)
    n = ff.densities()
    for s in range(L):
        assert abs(st.expect_local(s, [0, 1]) - n[s]) < 1e-12
    for b in range(1, L):
        assert abs(st.entropy(b) - ff.entropy(b)) < 1e-12


def test_xx_single_particle_hop():
    """One particle on site 0 of two sites: n_1(t) = sin^2(t/2) exactly for one gate."""
    st = U1MPS.product(2, [1, 0])
    tau = 0.83
    st.apply_gate2(0, tebd.xxz_gates(2, 0.0, tau)(0, 1.0), 4, 0.0)
    assert abs(st.expect_local(1, [0, 1]) - np.sin(tau / 2) ** 2) < 1e-15
