"""The two largest workload configurations on their real sizes, for as many steps as
the float64 oracle finishes in about a minute.

Boson sampling, M = 100 modes, one photon in each of modes 0..49, per-mode cutoff 4
(d = 5), a brickwork of seeded Haar beam splitters, chi <= 1024, cutoff 1e-10: the
first seven layers, after which the largest bond has reached the chi cap.  FP64 bar:
every bond table identical to the oracle's after every layer, Schmidt values within
1e-12, <n_j> within 1e-9 n_max, amplitudes of output patterns near the input within
1e-9 of the largest of them.

Bose-Hubbard L = 128, N = 128, J = 1, U = 2, dt = 0.02, chi <= 2048: five Strang
steps from the Mott state in FP64 (same bar, bond tables checked after every layer)
and with the sector GEMMs in TF32 and BF16x3.  Stated error of the reduced modes
against the FP64 oracle after these 15 layers (max over sites and bonds; measured on
GB300 in brackets):
    TF32:   <n_i> 2e-3 [6.3e-4]    bond entropy 2e-3 [5.7e-4]
    BF16x3: <n_i> 4e-5 [8.8e-6]    bond entropy 4e-5 [8.1e-6]
One update of a random chi = 2048 state (Theta(c) up to 1700 x 113 and 796 x 796),
two-site product relative to its largest entry: TF32 2e-3 [4.9e-4], BF16x3 5e-5
[8.4e-6]; FP64 to the bar of the parity tests.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, gates, tebd

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _tables_equal(g, st, L):
    for b in range(L + 1):
        assert g.bond_dims(b) == st.bond[b], (b, g.bond_dims(b), st.bond[b])


def _near_input_patterns(occ, d, n, rng):
    """Output patterns a few photon hops away from the input (inside the light cone)."""
    out = [list(occ)]
    M = len(occ)
    while len(out) < n:
        c = list(occ)
        for _ in range(int(rng.integers(1, 6))):
            j = int(rng.integers(M))
            k = j + (1 if rng.random() < 0.5 else -1)
            if 0 <= k < M and c[j] > 0 and c[k] < d - 1:
                c[j] -= 1
                c[k] += 1
        out.append(c)
    return out


def test_boson_sampling_M100_prefix(gpu_lib):
    M, n, d, chi, cutoff, n_layers = 100, 50, 5, 1024, 1e-10, 7
    occ = W.single_photon_occupations(M, n)
    layers = W.brickwork_pairs(M, 100)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=0)
    g = gpu_lib.MPS(d, occ, chi)
    st = U1MPS.product(d, occ)
    k = 0
    for sites in layers[:n_layers]:
        gs = [gates.beam_splitter_gate(*ang[k + j], d) for j in range(len(sites))]
        k += len(sites)
        g.apply_layer(sites, gs, chi, cutoff)
        for s, G in zip(sites, gs):
            st.apply_gate2(s, G, chi, cutoff)
        _tables_equal(g, st, M)
    assert max(st.bond_dim(b) for b in range(M + 1)) == chi          # the cap is active
    for b in range(1, M):
        gb = g.bond(b)
        for c, lam in gb.items():
            assert np.max(np.abs(lam - st.lam[b][c])) <= 1e-12
    n_op = np.arange(d)
    for j in range(M):
        ref = st.expect_local(j, n_op)
        assert abs(g.expect(j, n_op) - ref) <= 1e-9 * max(abs(ref), d - 1)
    cfgs = _near_input_patterns(occ, d, 40, np.random.default_rng(5))
    ag = g.amplitudes(cfgs)
    ao = np.array([st.amplitude(c) for c in cfgs])
    scale = np.max(np.abs(ao))
    assert scale > 0
    assert np.max(np.abs(ag - ao)) <= 1e-9 * scale
    g.close()


@pytest.fixture(scope="module")
def bh128_oracle():
    L, d, chi, cutoff, steps = 128, 5, 2048, 1e-10, 5
    gate_of = tebd.bh_gates(L, d, 1.0, 2.0, 0.02)
    st = U1MPS.product(d, W.mott_occupations(L))
    tables = []
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            for s in sites:
                st.apply_gate2(s, gate_of(s, f), chi, cutoff)
            tables.append([dict(st.bond[b]) for b in range(L + 1)])
    return st, tables


TOL = {"tf32": dict(obs=2e-3, ent=2e-3), "bf16x3": dict(obs=4e-5, ent=4e-5)}


@pytest.mark.parametrize("name", ["fp64", "tf32", "bf16x3"])
def test_bose_hubbard_L128_prefix(gpu_lib, bh128_oracle, name):
    m = gpu_lib
    L, d, chi, cutoff, steps = 128, 5, 2048, 1e-10, 5
    st, tables = bh128_oracle
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[name]
    g = m.MPS(d, W.mott_occupations(L), chi, precision=prec)
    gt = m.tebd.GateTable("bh", L, d, 0.02, J=1.0, U=2.0)
    layer = 0
    for _ in range(steps):
        for sites, f in m.tebd.strang_layers(L):
            g.apply_layer(sites, [gt(s, f) for s in sites], chi, cutoff)
            if name == "fp64":
                for b in range(L + 1):
                    assert g.bond_dims(b) == tables[layer][b], (layer, b)
            layer += 1
    n_op = np.arange(d)
    dn = max(abs(g.expect(s, n_op) - st.expect_local(s, n_op)) for s in range(L))
    dS = max(abs(g.entropy(b) - st.entropy(b)) for b in range(1, L))
    print(f"Bose-Hubbard L=128 {name}: max |d<n_i>| {dn:.3e}, max |dS| {dS:.3e}")
    if name == "fp64":
        for s in range(L):
            ref = st.expect_local(s, n_op)
            assert abs(g.expect(s, n_op) - ref) <= 1e-9 * max(abs(ref), d - 1)
        for b in range(1, L):
            ref = st.entropy(b)
            assert abs(g.entropy(b) - ref) <= 1e-9 * max(abs(ref), math.log(chi))
    else:
        assert dn <= TOL[name]["obs"], dn
        assert dS <= TOL[name]["ent"], dS
    g.close()


@pytest.mark.parametrize("name", ["fp64", "tf32", "bf16x3"])
def test_single_update_at_chi2048_sector_sizes(gpu_lib, name):
    """One middle update of a random chi = 2048 state (d = 5): the Theta(c) blocks are
    the size of a saturated L = 128, chi <= 2048 chain's (up to about 600 x 600), so the
    large-sector SVD kernels and the tensor-core tiles run at their full sizes."""
    from tests.helpers import compare_update, load_state, random_state, two_site_product
    m = gpu_lib
    L, d, N, chi = 16, 5, 16, 2048
    s = L // 2 - 1
    st = random_state(L, d, N, chi, seed=21)
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[name]
    g = m.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), chi, precision=prec)
    load_state(g, st)
    G = gates.bh_gate(L, s, d, 1.0, 2.0, 0.3)
    g.apply_gate2(s, G, chi, 1e-10)
    st.apply_gate2(s, G, chi, 1e-10)
    sizes = [g.stats()["n_sectors"]]
    assert sizes[0] >= 15
    if name == "fp64":
        compare_update(g, st, s)
    else:
        pg = two_site_product(g.site(s), g.site(s + 1))
        po = two_site_product(st.B[s], st.B[s + 1])
        scale = max(np.max(np.abs(v)) for v in po.values())
        err = max(np.max(np.abs(pg.get(k, 0) - po[k])) for k in po)
        print(f"chi=2048 update {name}: two-site product error {err / scale:.3e}")
        assert err / scale <= {"tf32": 2e-3, "bf16x3": 5e-5}[name]
    g.close()
