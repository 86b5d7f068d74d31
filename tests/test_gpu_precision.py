"""Reduced-precision sector GEMMs (TF32 and BF16x3 on tcgen05) against the float64 oracle.

In these modes only the two contractions of an update run on the tensor cores: the
Theta' build and the reassembly product Theta' Y / |S_kept|.  The SVD, the global
truncation and the renormalisation stay FP64 and follow the FP64 rules unchanged, so
the rounding of Theta' shows up as small singular values that the cutoff keeps and the
chi cap trims like any others.

Stated error against the FP64 oracle, after the whole run (max over sites/bonds);
measured on GB300 in brackets (with FP64 operand staging; the stated tolerances hold with the
FP32 staging of the tensor-core kernel, whose two-site products measure 5.4e-4 (TF32) and
1.3e-5 (BF16x3)):
    XXZ L=16, Neel, dt=0.05 x 20 steps, chi<=64, cutoff 1e-10 (600 updates)
        TF32:   <Sz_i> 5e-3 [1.5e-3]   bond entropy 5e-3 [1.6e-3]   amplitude 1.5e-3 [3.1e-4]
        BF16x3: <Sz_i> 8e-5 [2.1e-5]   bond entropy 1e-4 [2.7e-5]   amplitude 2e-5 [3.9e-6]
    Bose-Hubbard L=12, d=5, Mott, dt=0.05 x 8 steps, chi<=24 (176 updates)
        TF32:   <n_i> 5e-3 [1.6e-3]    bond entropy 5e-3 [1.1e-3]
        BF16x3: <n_i> 8e-5 [2.2e-5]    bond entropy 1e-4 [2.1e-5]
    one update on a random state, two-site product relative to its largest entry
        TF32: 2e-3 [5.6e-4]            BF16x3: 5e-5 [1.3e-5]
Each update perturbs the state by about u times a small factor (the number of terms
summed per element enters as sqrt, the rounding is unbiased), u = 2^-11 for TF32 and
about 2^-17 for BF16x3, so the deviation grows like u sqrt(updates) to u * updates.
On the XXZ run the bond tables (sector labels and dimensions) equal the oracle's after
at least 90% of the layers (measured: BF16x3 all, TF32 58 of 60): the reduced modes
guarantee the observable errors stated above, not the labels of values that their
rounding moves across the truncation cut.
"""
import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, gates, tebd
from tests.helpers import load_state, random_state, two_site_product

pytestmark = pytest.mark.gpu

TOL = {
    "tf32": dict(obs=5e-3, ent=5e-3, amp=1.5e-3, prod=2e-3),
    "bf16x3": dict(obs=8e-5, ent=1e-4, amp=2e-5, prod=5e-5),
}


def _prec(m, name):
    return {"tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[name]


def _run(m, L, d, occ, gate_of, steps, chi, cutoff, prec):
    """Both evolutions; returns them and the fraction of layers after which every bond
    table (sector labels and dimensions) equals the oracle's."""
    g = m.MPS(d, occ, chi, precision=prec)
    st = U1MPS.product(d, occ)
    same = layers = 0
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            g.apply_layer(sites, [gate_of(s, f) for s in sites], chi, cutoff)
            for s in sites:
                st.apply_gate2(s, gate_of(s, f), chi, cutoff)
            layers += 1
            same += all(g.bond_dims(b) == st.bond[b] for b in range(L + 1))
    return g, st, same / layers


@pytest.mark.parametrize("name", ["tf32", "bf16x3"])
def test_xxz_mixed_precision_observables(gpu_lib, name):
    L = 16
    g, st, same = _run(gpu_lib, L, 2, W.neel_occupations(L), tebd.xxz_gates(L, 0.5, 0.05), 20, 64, 1e-10,
                       _prec(gpu_lib, name))
    print(f"XXZ {name}: fraction of layers with the oracle's bond tables {same:.3f}")
    assert same >= 0.9
    t = TOL[name]
    dz = max(abs(g.expect(s, [-0.5, 0.5]) - st.expect_local(s, [-0.5, 0.5])) for s in range(L))
    dS = max(abs(g.entropy(b) - st.entropy(b)) for b in range(1, L))
    assert dz <= t["obs"], dz
    assert dS <= t["ent"], dS
    rng = np.random.default_rng(3)
    cfgs = [W.random_occupations(L, 2, 8, rng) for _ in range(64)] + [W.neel_occupations(L)]
    da = np.max(np.abs(g.amplitudes(cfgs) - np.array([st.amplitude(c) for c in cfgs])))
    assert da <= t["amp"], da
    # the charge structure stays exact: every bond's sectors are charges the oracle also has
    for b in range(L + 1):
        assert set(g.bond_dims(b)) <= set(st.bond[b])


@pytest.mark.parametrize("name", ["tf32", "bf16x3"])
def test_bose_hubbard_mixed_precision_observables(gpu_lib, name):
    L, d = 12, 5
    g, st, same = _run(gpu_lib, L, d, W.mott_occupations(L), tebd.bh_gates(L, d, 1.0, 2.0, 0.05), 8, 24, 1e-10,
                       _prec(gpu_lib, name))
    print(f"Bose-Hubbard {name}: fraction of layers with the oracle's bond tables {same:.3f}")
    t = TOL[name]
    n_op = np.arange(d)
    dn = max(abs(g.expect(s, n_op) - st.expect_local(s, n_op)) for s in range(L))
    dS = max(abs(g.entropy(b) - st.entropy(b)) for b in range(1, L))
    assert dn <= t["obs"], dn
    assert dS <= t["ent"], dS


@pytest.mark.parametrize("name", ["tf32", "bf16x3"])
@pytest.mark.parametrize("d,L,N,chi_state,chi", [(2, 8, 4, 40, 64), (5, 6, 6, 150, 400)])
def test_single_update_two_site_product(gpu_lib, name, d, L, N, chi_state, chi):
    """One update on a random state (blocks of up to ~150, several tiles and ragged
    tails): the gauge-invariant two-site product after the update is within the
    precision's tolerance of the oracle's, and lambda stays normalised in FP64."""
    st = random_state(L, d, N, chi_state, seed=d * 100 + chi)
    g = gpu_lib.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), max(chi_state, chi),
                    precision=_prec(gpu_lib, name))
    G = gates.bh_gate(L, 2, d, 1.0, 2.0, 0.3) if d > 2 else gates.xxz_gate(0.5, 0.4)
    worst = 0.0
    for s in range(L - 1):
        load_state(g, st)
        g.apply_gate2(s, G, chi, 0.0)
        o = random_state(L, d, N, chi_state, seed=d * 100 + chi)
        o.apply_gate2(s, G, chi, 0.0)
        pg = two_site_product(g.site(s), g.site(s + 1))
        po = two_site_product(o.B[s], o.B[s + 1])
        assert pg.keys() <= po.keys()
        scale = max(np.max(np.abs(v)) for v in po.values())
        err = max(np.max(np.abs(pg.get(k, 0) - po[k])) for k in po)
        worst = max(worst, err / scale)
        lam = np.concatenate(list(g.bond(s + 1).values()))
        assert abs(np.sum(lam ** 2) - 1.0) <= 1e-12
    print(f"two-site product error {name} d={d}: {worst:.3e}")
    assert worst <= TOL[name]["prod"], worst
