"""CUDA-graph launches and the SVD tile-shape autotuner.

Graph mode replays the same kernels with the same arguments as direct launches, so
a run with graphs must be bit-identical to one without.  The autotuner changes the
Jacobi pair order of the large-sector SVD kernel, so a tuned update agrees with an
untuned one to rounding (identical sector structure, Schmidt values within 1e-12,
gauge-invariant two-site products within 1e-9), matches the oracle to the same bar,
and reuses its stored choice on the next batch with the same sector-size histogram.
"""
import numpy as np
import pytest

import workloads as W
from oracle import gates
from tests.helpers import compare_update, load_state, random_state

pytestmark = pytest.mark.gpu


def _same_state(a, b, L):
    for bnd in range(L + 1):
        ba, bb = a.bond(bnd), b.bond(bnd)
        assert ba.keys() == bb.keys()
        for c in ba:
            assert np.array_equal(ba[c], bb[c]), (bnd, c)
    for s in range(L):
        sa, sb = a.site(s), b.site(s)
        assert sa.keys() == sb.keys()
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), (s, k)


def test_graph_mode_is_bit_identical(gpu_lib):
    import torch
    m = gpu_lib
    L, chi, steps = 16, 64, 6
    st = torch.cuda.Stream()
    a = m.MPS(2, W.neel_occupations(L), chi, stream=st.cuda_stream)
    b = m.MPS(2, W.neel_occupations(L), chi, stream=st.cuda_stream)
    b.set_graphs(True)
    b.set_profiling(True)
    gt = m.tebd.GateTable("xxz", L, 2, 0.05, delta=0.5)
    for _ in range(steps):
        m.tebd.trotter_step(a, gt, chi, 1e-10)
        m.tebd.trotter_step(b, gt, chi, 1e-10)
    _same_state(a, b, L)
    gs = b.graph_stats()
    assert gs["launches"] == 2 * 3 * steps          # two phases per layer
    assert gs["updates"] > 0                         # parameters changed, topology held
    assert gs["instantiations"] + gs["updates"] == gs["launches"]
    ks = b.kernel_stats()
    redos = b.deflation_stats()["redos"]            # a redone SVD phase is one more launch
    assert ks["svd"]["launches"] == 3 * steps + redos and ks["svd"]["ms"] > 0   # events inside the graph
    assert a.graph_stats()["launches"] == 0
    a.close()
    b.close()


def test_graph_mode_on_default_stream_launches_directly(gpu_lib):
    m = gpu_lib
    L, chi = 8, 16
    a = m.MPS(2, W.neel_occupations(L), chi, stream=0)
    a.set_graphs(True)
    gt = m.tebd.GateTable("xxz", L, 2, 0.05, delta=0.5)
    m.tebd.trotter_step(a, gt, chi, 1e-10)
    assert a.graph_stats()["launches"] == 0
    a.close()


def test_executor_graphs_match_direct(gpu_lib):
    import torch
    m = gpu_lib
    st = torch.cuda.Stream()
    runs = []
    for graphs in (False, True):
        ex = m.Executor(stream=st.cuda_stream)
        ex.set_graphs(graphs)
        psis = [m.MPS(2, W.neel_occupations(12), 32, stream=st.cuda_stream),
                m.MPS(3, W.mott_occupations(10), 24, stream=st.cuda_stream)]
        gts = [m.tebd.GateTable("xxz", 12, 2, 0.05, delta=1.1), m.tebd.GateTable("bh", 10, 3, 0.02, U=4.0)]
        for _ in range(4):
            for (sa, fa), (sb, fb) in zip(m.tebd.strang_layers(12), m.tebd.strang_layers(10)):
                items = [(psis[0], s, gts[0](s, fa), 32, 1e-10) for s in sa]
                items += [(psis[1], s, gts[1](s, fb), 24, 1e-10) for s in sb]
                ex.apply(items)
        torch.cuda.synchronize()
        runs.append(psis)
        if graphs:
            assert ex.graph_stats()["launches"] > 0
        ex.close()
    _same_state(runs[0][0], runs[1][0], 12)
    _same_state(runs[0][1], runs[1][1], 10)


def test_autotune_tunes_once_and_keeps_parity(gpu_lib):
    m = gpu_lib
    L, d, N, chi = 10, 5, 10, 300          # the middle update has three cluster-kernel sectors
    st0 = random_state(L, d, N, chi, seed=11)
    G = gates.bh_gate(L, 4, d, 1.0, 2.0, 0.3)
    s = 4
    m.autotune_clear()
    m.autotune_min_flops(0.0)
    try:
        plain = m.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), chi)
        load_state(plain, st0)
        plain.apply_gate2(s, G, chi, 1e-10)

        tuned = []
        for rep in range(2):
            g = m.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), chi)
            g.set_autotune(True)
            load_state(g, st0)
            g.apply_gate2(s, G, chi, 1e-10)
            tuned.append(g)
        stats = m.autotune_stats()
        assert stats["keys"] == 1 and stats["tuning_runs"] == 1 and stats["hits"] == 1, stats
        assert "bw=" in m.autotune_table()
        # the second tuned update reused the stored shape: bit-identical to the first
        _same_state(tuned[0], tuned[1], L)
        # tuned vs untuned and vs the oracle: same structure, agreement to rounding
        st = random_state(L, d, N, chi, seed=11)
        st.apply_gate2(s, G, chi, 1e-10)
        compare_update(tuned[0], st, s)
        compare_update(plain, st, s)
        for g in tuned + [plain]:
            g.close()
    finally:
        m.autotune_min_flops(2e10)
        m.autotune_clear()


def test_every_tile_shape_matches_the_oracle_on_large_sectors(gpu_lib):
    """Each of the autotuner's twelve candidates, forced in turn, on one middle update of a
    random chi = 2048 state (Theta(c) up to 1700 x 113 and 796 x 796, so candidates 8 and 9
    put the largest sectors on 16-CTA clusters and 10 and 11 on the round-robin kernel):
    every one keeps the oracle's sector structure, Schmidt values and two-site product."""
    m = gpu_lib
    L, d, N, chi = 16, 5, 16, 2048
    s = L // 2 - 1
    st0 = random_state(L, d, N, chi, seed=21)
    G = gates.bh_gate(L, s, d, 1.0, 2.0, 0.3)
    ref = random_state(L, d, N, chi, seed=21)
    ref.apply_gate2(s, G, chi, 1e-10)
    try:
        for cand in range(12):
            m.autotune_force(cand)
            g = m.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), chi)
            load_state(g, st0)
            g.apply_gate2(s, G, chi, 1e-10)
            compare_update(g, ref, s)
            g.close()
    finally:
        m.autotune_force(-1)
    with pytest.raises(m.MPSError):
        m.autotune_force(12)
