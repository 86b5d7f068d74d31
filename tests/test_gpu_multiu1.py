"""Handles with several U(1) charges (mps_create_multi) against the tuple-charge oracle.

Two-species hard-core bosons, charges (N_up, N_down): the rows of a Theta(c) block are the
left sectors l with l - c in {(0,0), (0,1), (1,0), (1,1)}, which are not one run of the
sorted bond table once the bonds hold several charges per species, so these runs exercise
the gathered row scale and the listed row / column offsets of the update.  After every
Strang layer the bond tables (charge vectors and dimensions) are those of the oracle; at the
end lambda agrees to 1e-12, the densities of both species and the bond entropies to 1e-9,
and gauge-invariant amplitude ratios to 1e-10.
"""
import numpy as np
import pytest

from oracle import multiu1, tebd
from oracle.gates import bh_weights

pytestmark = pytest.mark.gpu

Q = multiu1.TWO_SPECIES_Q


def _run(m, L, occ, J, U, dt, steps, chi, cutoff, precision=None):
    """Both evolutions; in FP64 every bond table equals the oracle's after every layer; with
    reduced-precision GEMMs the number of (layer, bond) tables that differ is returned."""
    g = m.MPS(4, occ, chi, charges=Q, precision=m.MPS_FP64 if precision is None else precision)
    differ = 0
    st = multiu1.MultiU1MPS.product(Q, occ)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            gates = [multiu1.two_species_gate(J, U, *bh_weights(L, s), f * dt) for s in sites]
            g.apply_layer(sites, gates, chi, cutoff)
            for s, G in zip(sites, gates):
                st.apply_gate2(s, G, chi, cutoff)
            for b in range(L + 1):
                if precision is None:
                    assert g.bond_dims(b) == st.bond[b], (b, g.bond_dims(b), st.bond[b])
                else:
                    differ += g.bond_dims(b) != st.bond[b]
    return (g, st) if precision is None else (g, st, differ)


@pytest.mark.parametrize("L,chi,steps", [(10, 24, 8), (16, 64, 10)])
def test_two_species_bosons_match_the_oracle(gpu_lib, L, chi, steps):
    m = gpu_lib
    rng = np.random.default_rng(L)
    occ = [int(x) for x in rng.integers(0, 4, L)]
    g, st = _run(m, L, occ, 1.0, 2.0, 0.05, steps, chi, 1e-10)
    assert g.N == st.N
    for b in range(L + 1):
        for c, v in g.bond(b).items():
            assert np.max(np.abs(v - st.lam[b][c])) <= 1e-12
    nu = np.array([q[0] for q in Q], float)
    nd = np.array([q[1] for q in Q], float)
    for s in range(L):
        assert abs(g.expect(s, nu) - st.expect_local(s, nu)) <= 1e-9
        assert abs(g.expect(s, nd) - st.expect_local(s, nd)) <= 1e-9
    lnchi = np.log(chi)
    for b in range(1, L):
        assert abs(g.entropy(b) - st.entropy(b)) <= 1e-9 * max(st.entropy(b), lnchi)
    # amplitudes of random configurations with the right charges, relative to the largest
    cfgs = []
    while len(cfgs) < 48:
        c = [int(x) for x in rng.integers(0, 4, L)]
        if tuple(sum(Q[i][k] for i in c) for k in range(2)) == st.N:
            cfgs.append(c)
    cfgs.append(occ)
    a = g.amplitudes(cfgs)
    r = np.array([st.amplitude(c) for c in cfgs])
    k = int(np.argmax(np.abs(r)))
    ph = r[k] / a[k]
    assert abs(abs(ph) - 1.0) <= 1e-10
    assert np.max(np.abs(a * ph - r)) <= 1e-10 * max(1.0, np.max(np.abs(r)))
    g.close()


# stated accuracy of the reduced-precision modes against the FP64 oracle (the densities' and
# entropies' tolerances of the single-U(1) precision tests, whose runs are of this length)
TOL = {"tf32": dict(obs=5e-3, ent=5e-3), "bf16x3": dict(obs=8e-5, ent=1e-4)}


@pytest.mark.parametrize("name", ["tf32", "bf16x3"])
def test_two_species_bosons_with_tensor_core_gemms(gpu_lib, name):
    """The sector GEMMs of a several-U(1) handle on the tensor cores (listed rows and columns
    in the tensor-core Theta' build and reassembly); the SVD and truncation stay FP64."""
    m = gpu_lib
    L, chi, steps = 10, 24, 8
    rng = np.random.default_rng(L)
    occ = [int(x) for x in rng.integers(0, 4, L)]
    prec = {"tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[name]
    g, st, differ = _run(m, L, occ, 1.0, 2.0, 0.05, steps, chi, 1e-10, precision=prec)
    t = TOL[name]
    for b in range(L + 1):   # the truncation's invariants hold whatever the GEMM precision
        lam = g.bond(b)
        assert sum(len(v) for v in lam.values()) <= chi
        assert abs(sum(float(v @ v) for v in lam.values()) - 1.0) <= 1e-12
    nu = np.array([q[0] for q in Q], float)
    nd = np.array([q[1] for q in Q], float)
    dn = max(max(abs(g.expect(s, nu) - st.expect_local(s, nu)), abs(g.expect(s, nd) - st.expect_local(s, nd)))
             for s in range(L))
    dS = max(abs(g.entropy(b) - st.entropy(b)) for b in range(1, L))
    print(f"two species, {name}: densities {dn:.2e}, entropies {dS:.2e}, {differ} bond tables "
          f"(layer, bond) differing from the oracle's")
    assert dn <= t["obs"], dn
    assert dS <= t["ent"], dS
    g.close()


def test_multi_handle_rejects_bad_charges(gpu_lib):
    m = gpu_lib
    with pytest.raises(m.MPSError):
        m.MPS(4, [0, 1, 2, 3], 8, precision=7, charges=Q)
    with pytest.raises(m.MPSError):
        m.MPS(4, [0, 1, 2, 3], 8, charges=[(0, 0), (1, 0), (0, 1), (1, 1)])   # not ascending
