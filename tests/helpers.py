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


# ---------------------------------------------------------------------------
# Random U(1) states (oracle-side) and loading them into the CUDA library
# ---------------------------------------------------------------------------
from oracle.synth import random_state, saturated_dims  # noqa: E402,F401


def load_state(gpu, st):
    for b in range(1, st.L):
        gpu.set_bond(b, st.lam[b])
    for s in range(st.L):
        gpu.set_site(s, st.B[s])


def two_site_product(Bl, Br):
    """Gauge-invariant contraction over the middle bond: {(l, r): sum_m Bl[l,m] Br[m,r]}."""
    out = {}
    for (l, m), a in Bl.items():
        for (m2, r), b in Br.items():
            if m2 == m:
                out[(l, r)] = out.get((l, r), 0) + a @ b
    return out


def compare_update(gpu, st, s, tol_lam=1e-12, tol_prod=1e-9):
    """Exact sector structure of bond s+1, lambdas, and the two-site product of sites s, s+1."""
    gb = gpu.bond(s + 1)
    assert sorted(gb) == sorted(st.bond[s + 1]), (sorted(gb), sorted(st.bond[s + 1]))
    for c in gb:
        assert len(gb[c]) == st.bond[s + 1][c], (c, len(gb[c]), st.bond[s + 1][c])
        assert np.max(np.abs(gb[c] - st.lam[s + 1][c])) <= tol_lam
    pg = two_site_product(gpu.site(s), gpu.site(s + 1))
    po = two_site_product(st.B[s], st.B[s + 1])
    assert pg.keys() == po.keys()
    scale = max(np.max(np.abs(v)) for v in po.values())
    err = max(np.max(np.abs(pg[k] - po[k])) for k in po)
    assert err <= tol_prod * scale, err / scale
    return err / scale
