"""The benchmark's own chain at full size, in the launch configuration bench.py times.

Bose-Hubbard L=128, N=128, chi<=2048, the seeded synthetic saturated chain of the benchmark
(workloads.saturated_random_state with beta = 0.3), CUDA graphs on, the chi deflation and the
mixed-precision SVD start at their defaults: one whole odd Strang layer (64 updates in one
call, dt/2 gates).  The updates of a layer touch disjoint sites, so the oracle can redo any
one of them alone from the same chain; sampled updates (both chain ends and the middle) are
compared: in FP64 the new bond table exactly, lambda to 1e-12 and the gauge-invariant
two-site product to 1e-8; with TF32 sector GEMMs (the benchmark's precision) the two-site
product to the TF32 tolerance of the precision tests (2e-3 of its largest entry) and the
bond charges as a subset of the oracle's.  Every bond of the layer keeps unit-norm lambda
and at most chi states.
"""
import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, tebd
from tests.helpers import compare_update, two_site_product

pytestmark = pytest.mark.gpu

L, D, N, CHI, DT, CUTOFF = 128, 5, 128, 2048, 0.02, 1e-10


@pytest.fixture(scope="module")
def chain():
    lam, blocks = W.saturated_random_state(L, D, N, CHI, seed=0, beta=0.3)
    return lam, blocks


def _oracle(lam, blocks):
    st = U1MPS(L, D, N)
    st.bond = [None] * (L + 1)
    st.lam = [None] * (L + 1)
    st.bond[0], st.bond[L] = {N: 1}, {0: 1}
    st.lam[0], st.lam[L] = {N: np.ones(1)}, {0: np.ones(1)}
    for b in range(1, L):
        st.lam[b] = {c: np.array(v) for c, v in lam[b].items()}
        st.bond[b] = {c: len(v) for c, v in lam[b].items()}
    st.B = [dict(bl) for bl in blocks]
    return st


@pytest.mark.parametrize("name", ["fp64", "tf32"])
def test_benchmark_layer_sampled_against_the_oracle(gpu_lib, chain, name):
    m = gpu_lib
    lam, blocks = chain
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32}[name]
    g = m.MPS(D, W.mott_occupations(L), CHI, precision=prec)
    g.set_graphs(True)
    g.set_chi_deflation(3e-4)
    for b in range(1, L):
        g.set_bond(b, lam[b])
    for s in range(L):
        g.set_site(s, blocks[s])
    gates = m.tebd.GateTable("bh", L, D, DT, J=1.0, U=2.0)
    sites = list(range(0, L - 1, 2))
    g.apply_layer(sites, [gates(s, 0.5) for s in sites], CHI, CUTOFF)
    og = tebd.bh_gates(L, D, 1.0, 2.0, DT)
    for s in sites:
        gb = g.bond(s + 1)
        assert sum(len(v) for v in gb.values()) <= CHI
        assert abs(sum(float(v @ v) for v in gb.values()) - 1.0) <= 1e-12
    for s in (0, 62, 126):
        ref = _oracle(lam, blocks)
        ref.apply_gate2(s, og(s, 0.5), CHI, CUTOFF)
        if name == "fp64":
            compare_update(g, ref, s, tol_lam=1e-12, tol_prod=1e-8)
        else:
            assert set(g.bond_dims(s + 1)) <= set(ref.bond[s + 1])
            pg = two_site_product(g.site(s), g.site(s + 1))
            po = two_site_product(ref.B[s], ref.B[s + 1])
            scale = max(np.max(np.abs(v)) for v in po.values())
            err = max(np.max(np.abs(pg.get(k, 0) - po[k])) for k in po)
            print(f"bench chain, TF32, update {s}: two-site product error {err / scale:.3e}")
            assert err / scale <= 2e-3
    g.close()
