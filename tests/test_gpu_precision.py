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
Sector labels on the XXZ run: in BF16x3 every bond table (labels and dimensions) equals
the oracle's after every layer.  In TF32 a bond may differ only where the oracle's own
update of that bond had a singular value within the run's stated accuracy (5e-3 sigma_max,
the <Sz_i> tolerance above) of its cut: the smallest kept and the largest discarded value
when chi set the cut, or the cutoff threshold cutoff * |sigma|_2 when the cutoff did.  A
TF32 rounding of Theta' moves singular values by about 2^-11 sigma_max per update, so such
values can cross the cut; a label or dimension change anywhere else fails the test.
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


def _cut_distance(info, chi):
    """Distance (relative to sigma_max) of the oracle update's nearest singular value to
    its cut: the chi-th / (chi+1)-th gap when chi set the cut, else the distance of the
    nearest value to the cutoff threshold."""
    vals = np.sort(np.concatenate([np.asarray(v) for v in info["sigmas"].values()]))[::-1]
    smax = vals[0]
    cand = vals[vals > info["threshold"]]
    if len(cand) > chi:
        return (cand[chi - 1] - cand[chi]) / smax
    return float(np.min(np.abs(vals - info["threshold"]))) / smax


def _run(m, L, d, occ, gate_of, steps, chi, cutoff, prec):
    """Both evolutions; returns them and every (layer, bond, cut distance) at which a bond
    table (sector labels and dimensions) differs from the oracle's."""
    g = m.MPS(d, occ, chi, precision=prec)
    st = U1MPS.product(d, occ)
    mism = []
    layer = 0
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            g.apply_layer(sites, [gate_of(s, f) for s in sites], chi, cutoff)
            infos = {s: st.apply_gate2(s, gate_of(s, f), chi, cutoff) for s in sites}
            for b in range(L + 1):
                if g.bond_dims(b) != st.bond[b]:
                    # only the bonds this layer rewrote can differ first; an older difference
                    # stays visible until its bond is updated again
                    dist = _cut_distance(infos[b - 1], chi) if (b - 1) in infos else None
                    mism.append((layer, b, dist))
            layer += 1
    return g, st, mism


@pytest.mark.parametrize("name", ["tf32", "bf16x3"])
def test_xxz_mixed_precision_observables(gpu_lib, name):
    L = 16
    g, st, mism = _run(gpu_lib, L, 2, W.neel_occupations(L), tebd.xxz_gates(L, 0.5, 0.05), 20, 64, 1e-10,
                       _prec(gpu_lib, name))
    t = TOL[name]
    print(f"XXZ {name}: bonds differing from the oracle's tables (layer, bond, cut distance): {mism}")
    if name == "bf16x3":
        assert mism == []
    else:
        # every difference at a bond the layer rewrote comes from a cut the mode cannot
        # resolve; a bond the layer did not touch (None) can only carry an earlier difference
        seen = set()
        for layer, b, dist in mism:
            if dist is None:
                assert b in seen, (layer, b)
            else:
                assert dist <= t["obs"], (layer, b, dist)
            seen.add(b)
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
    g, st, mism = _run(gpu_lib, L, d, W.mott_occupations(L), tebd.bh_gates(L, d, 1.0, 2.0, 0.05), 8, 24, 1e-10,
                       _prec(gpu_lib, name))
    print(f"Bose-Hubbard {name}: bonds differing from the oracle's tables: {len(mism)}")
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
