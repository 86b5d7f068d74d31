"""Two-site DMRG on the GPU (mps_dmrg) against the float64 oracle (oracle/dmrg.py).

Both sides run the same sweeps from the same starting state: the Lanczos eigenvalue of
every local step agrees to 1e-10 relative, the bond tables (sector labels and
dimensions) are identical after the run, the Schmidt values agree to 1e-10, and local
observables and bond entropies to 1e-9 of max(|ref|, |O|).  The oracle's local
eigensolver is exact (dense eigh / ARPACK at tol 1e-13) and the GPU Lanczos stops at a
residual of 1e-12 |E|, so the local ground states agree to about 1e-12 / gap.
Starting states: the Neel / Mott product states, and states that the oracle's TEBD
grew from them (loaded into the handle), so the sweeps start with many sectors.
The untruncated XXZ L=10 run also matches exact diagonalisation.
"""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, dense, dmrg, tebd
from tests.helpers import load_state

pytestmark = pytest.mark.gpu


def _bonds(m, model, L, d):
    if model == "xxz":
        return m.models.chain_bond_terms("xxz", L, 2, delta=0.5), dmrg.xxz_bonds(L, 0.5)
    return m.models.chain_bond_terms("bh", L, d, J=1.0, U=2.0), dmrg.bh_bonds(L, d, 1.0, 2.0)


def _start(model, L, d, steps, chi0, dt):
    occ = W.neel_occupations(L) if model == "xxz" else W.mott_occupations(L)
    st = U1MPS.product(d, occ)
    if steps:
        g = tebd.xxz_gates(L, 0.5, dt) if model == "xxz" else tebd.bh_gates(L, d, 1.0, 2.0, dt)
        tebd.run_tebd(st, g, steps, chi0, 1e-10)
    return occ, st


def _compare(g, st, L, d, E_gpu, E_ref):
    assert len(E_gpu) == len(E_ref)
    dE = np.max(np.abs(np.asarray(E_gpu) - np.asarray(E_ref)) / np.maximum(1.0, np.abs(E_ref)))
    assert dE <= 1e-10, dE
    for b in range(L + 1):
        assert g.bond_dims(b) == st.bond[b], (b, g.bond_dims(b), st.bond[b])
        gb = g.bond(b)
        for c, v in gb.items():
            assert np.max(np.abs(v - st.lam[b][c])) <= 1e-10, (b, c)
        assert abs(sum(float(v @ v) for v in gb.values()) - 1.0) <= 1e-12
    nop = np.arange(d, dtype=float)
    for s in range(L):
        a, r = g.expect(s, nop), st.expect_local(s, nop)
        assert abs(a - r) <= 1e-9 * max(abs(r), d - 1), (s, a, r)
    lnchi = np.log(max(2, max(sum(st.bond[b].values()) for b in range(L + 1))))
    for b in range(1, L):
        assert abs(g.entropy(b) - st.entropy(b)) <= 1e-9 * max(st.entropy(b), lnchi), b
    return dE


def test_dmrg_xxz_L10_matches_exact_diagonalisation_and_the_oracle(gpu_lib):
    m = gpu_lib
    L, d = 10, 2
    hg, ho = _bonds(m, "xxz", L, d)
    occ, st = _start("xxz", L, d, 0, 0, 0.0)
    g = m.MPS(d, occ, 32)
    E = g.dmrg(hg, 3, 32, 1e-12)
    Eo, _ = dmrg.run_dmrg(st, ho, 3, 32, 1e-12)
    _compare(g, st, L, d, E, Eo)
    cfgs = list(itertools.product(range(2), repeat=L))
    idx = [k for k, c in enumerate(cfgs) if sum(c) == L // 2]
    H = np.zeros((2 ** L, 2 ** L), dtype=np.complex128)
    for k in range(L - 1):
        H += np.kron(np.kron(np.eye(2 ** k), dense.xxz_two_site(0.5)), np.eye(2 ** (L - k - 2)))
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert abs(E[-1] - e0) <= 1e-10 * abs(e0)
    # the canonical form the call leaves is the one the amplitude formula reads
    amp = g.amplitudes([cfgs[k] for k in idx[:40]])
    ref = np.array([st.amplitude(cfgs[k]) for k in idx[:40]])
    ph = ref[np.argmax(np.abs(ref))] / amp[np.argmax(np.abs(ref))]
    assert np.max(np.abs(amp * ph - ref)) <= 1e-10
    g.close()


@pytest.mark.parametrize("model,L,d,steps,chi0,dt,chi,sweeps", [
    ("xxz", 16, 2, 10, 32, 0.1, 48, 2),
    ("bh", 10, 5, 5, 24, 0.05, 32, 2),
])
def test_dmrg_from_an_evolved_state_matches_the_oracle(gpu_lib, model, L, d, steps, chi0, dt, chi, sweeps):
    m = gpu_lib
    hg, ho = _bonds(m, model, L, d)
    occ, st = _start(model, L, d, steps, chi0, dt)
    g = m.MPS(d, occ, chi)
    load_state(g, st)
    E = g.dmrg(hg, sweeps, chi, 1e-10)
    Eo, _ = dmrg.run_dmrg(st, ho, sweeps, chi, 1e-10)
    dE = _compare(g, st, L, d, E, Eo)
    print(f"{model} L={L} chi={chi}: E = {E[-1]:.12f}, max energy deviation {dE:.2e}, {g.dmrg_stats()}")
    g.close()


def test_dmrg_multi_tile_blocks(gpu_lib):
    """Sectors of up to ~120 states (two 64-wide tiles with a ragged tail in the block
    kernels): a free-boson quench (U = 0) from the Mott state entangles the chain, then
    one sweep towards the U = 2 ground state."""
    m = gpu_lib
    L, d, chi = 10, 5, 600
    hg, ho = _bonds(m, "bh", L, d)
    occ = W.mott_occupations(L)
    st = U1MPS.product(d, occ)
    tebd.run_tebd(st, tebd.bh_gates(L, d, 1.0, 0.0, 0.1), 16, chi, 1e-10)
    assert max(max(st.bond[b].values()) for b in range(L + 1)) > 64
    g = m.MPS(d, occ, chi)
    load_state(g, st)
    E = g.dmrg(hg, 1, chi, 1e-10)
    Eo, _ = dmrg.run_dmrg(st, ho, 1, chi, 1e-10)
    _compare(g, st, L, d, E, Eo)
    g.close()


def test_dmrg_state_continues_under_tebd(gpu_lib):
    """After mps_dmrg the handle holds the TEBD storage form: a real-time layer on both
    sides still agrees (bond tables, lambda, observables)."""
    m = gpu_lib
    L, d, chi = 12, 5, 24
    hg, ho = _bonds(m, "bh", L, d)
    occ, st = _start("bh", L, d, 2, 16, 0.05)
    g = m.MPS(d, occ, chi)
    load_state(g, st)
    g.dmrg(hg, 1, chi, 1e-10)
    dmrg.run_dmrg(st, ho, 1, chi, 1e-10)
    gates = m.tebd.GateTable("bh", L, d, 0.05, J=1.0, U=2.0)
    og = tebd.bh_gates(L, d, 1.0, 2.0, 0.05)
    for sites, f in m.tebd.strang_layers(L):
        g.apply_layer(sites, [gates(s, f) for s in sites], chi, 1e-10)
        for s in sites:
            st.apply_gate2(s, og(s, f), chi, 1e-10)
    nop = np.arange(d, dtype=float)
    for b in range(L + 1):
        assert g.bond_dims(b) == st.bond[b]
    for s in range(L):
        assert abs(g.expect(s, nop) - st.expect_local(s, nop)) <= 1e-9 * (d - 1)
    g.close()


def test_dmrg_argument_errors(gpu_lib):
    m = gpu_lib
    L, d = 6, 2
    hg, _ = _bonds(m, "xxz", L, d)
    g = m.MPS(d, W.neel_occupations(L), 8, precision=m.MPS_TF32)
    with pytest.raises(m.MPSError):
        g.dmrg(hg, 1, 8, 1e-10)
    g.close()
    g = m.MPS(d, W.neel_occupations(L), 8)
    with pytest.raises(m.MPSError):
        g.dmrg(hg, 1, 8, 1e-10, lanczos_dim=64)
    with pytest.raises(ValueError):
        g.dmrg(hg[:-1], 1, 8, 1e-10)
    g.close()
