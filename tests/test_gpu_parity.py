"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Bar (FP64 mode): kept sector labels and per-sector dimensions identical to the
oracle; Schmidt values within 1e-12 absolute (they are normalised); local
observables within 1e-9 * max(|ref|, |O|), |O| = 1/2 for Sz, n_max for n and
ln(chi) for bond entropies; gauge-invariant two-site products within 1e-9
relative.  Amplitudes are gauge invariant (the SVD gauge of every bond cancels in the
chain of blocks) and are compared directly.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, gates, permanent, tebd
from tests.helpers import compare_update, load_state, random_state

pytestmark = pytest.mark.gpu


def _gpu(m, d, occ, chi_max):
    return m.MPS(d, occ, chi_max)


def _bond_tables_equal(g, st):
    for b in range(st.L + 1):
        assert g.bond_dims(b) == st.bond[b], (b, g.bond_dims(b), st.bond[b])


# ---------------------------------------------------------------------------
# single updates on random states: several tiles, ragged tails, truncation on/off
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d,L,N,chi_state,chi,cutoff", [
    (2, 8, 4, 40, 64, 1e-10),
    (3, 7, 7, 60, 25, 1e-10),
    (5, 6, 6, 150, 90, 1e-10),
    (5, 6, 6, 150, 400, 0.0),
])
def test_single_update_random_state(gpu_lib, d, L, N, chi_state, chi, cutoff):
    st = random_state(L, d, N, chi_state, seed=d * 100 + chi)
    # the initial occupations only fix N; every inner bond and site is then loaded
    g = _gpu(gpu_lib, d, W.random_occupations(L, d, N, np.random.default_rng(0)), max(chi_state, chi))
    load_state(g, st)
    G = gates.bh_gate(L, 2, d, 1.0, 2.0, 0.3) if d > 2 else gates.xxz_gate(0.5, 0.4)
    for s in range(L - 1):
        # reload so both sides share the gauge of the left bond (the two-site product is
        # invariant only under the gauge of the middle bond the update rewrites)
        load_state(g, st)
        te_g = g.apply_gate2(s, G, chi, cutoff)
        info = st.apply_gate2(s, G, chi, cutoff)
        compare_update(g, st, s)
        assert abs(te_g - info["trunc_err"]) <= 1e-12 + 1e-9 * info["trunc_err"]


def test_layer_equals_sequential_updates(gpu_lib):
    L, d, N, chi = 10, 3, 10, 50
    st = random_state(L, d, N, chi, seed=7)
    a = _gpu(gpu_lib, d, [1] * L, chi)
    b = _gpu(gpu_lib, d, [1] * L, chi)
    load_state(a, st)
    load_state(b, st)
    G = gates.bh_gate(L, 3, d, 1.0, 3.0, 0.2)
    sites = [0, 2, 4, 6, 8]
    a.apply_layer(sites, [G] * len(sites), 30, 1e-10)
    for s in sites:
        b.apply_gate2(s, G, 30, 1e-10)
    for s in range(L):
        sa, sb = a.site(s), b.site(s)
        assert sa.keys() == sb.keys()
        for k in sa:
            assert np.array_equal(sa[k], sb[k])


# ---------------------------------------------------------------------------
# whole TEBD runs
# ---------------------------------------------------------------------------
def _run_both(m, L, d, occ, gate_of, steps, chi, cutoff, check_every_layer=True):
    g = _gpu(m, d, occ, chi)
    st = U1MPS.product(d, occ)
    for _ in range(steps):
        for sites, f in tebd.strang_layers(L):
            g.apply_layer(sites, [gate_of(s, f) for s in sites], chi, cutoff)
            for s in sites:
                st.apply_gate2(s, gate_of(s, f), chi, cutoff)
            if check_every_layer:
                _bond_tables_equal(g, st)
    return g, st


def test_xxz_cfg1_parity(gpu_lib):
    """XXZ L=16, Delta=0.5, Neel, dt=0.05 x 20, chi<=64, cutoff 1e-10."""
    L = 16
    gate_of = tebd.xxz_gates(L, 0.5, 0.05)
    g, st = _run_both(gpu_lib, L, 2, W.neel_occupations(L), gate_of, 20, 64, 1e-10)
    for s in range(L):
        ref = st.expect_local(s, [-0.5, 0.5])
        assert abs(g.expect(s, [-0.5, 0.5]) - ref) <= 1e-9 * max(abs(ref), 0.5)
    for b in range(1, L):
        ref = st.entropy(b)
        assert abs(g.entropy(b) - ref) <= 1e-9 * max(abs(ref), math.log(64))
    rng = np.random.default_rng(3)
    cfgs = [W.random_occupations(L, 2, 8, rng) for _ in range(64)] + [W.neel_occupations(L)]
    ag = g.amplitudes(cfgs)
    ao = np.array([st.amplitude(c) for c in cfgs])
    assert np.max(np.abs(ag - ao)) < 1e-10


def test_bose_hubbard_truncated_parity(gpu_lib):
    """BH d=5 with the chi cap active in most updates."""
    L, d = 12, 5
    gate_of = tebd.bh_gates(L, d, 1.0, 2.0, 0.05)
    g, st = _run_both(gpu_lib, L, d, W.mott_occupations(L), gate_of, 8, 24, 1e-10)
    n_op = np.arange(d)
    for s in range(L):
        ref = st.expect_local(s, n_op)
        assert abs(g.expect(s, n_op) - ref) <= 1e-9 * max(abs(ref), d - 1)
    assert max(st.bond_dim(b) for b in range(L + 1)) == 24


def test_boson_sampling_amplitudes(gpu_lib):
    M, n = 8, 4
    d = n + 1
    occ = W.single_photon_occupations(M, n)
    layers = W.brickwork_pairs(M, 8)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=0)
    g = _gpu(gpu_lib, d, occ, 512)
    st = U1MPS.product(d, occ)
    k = 0
    for sites in layers:
        gs = []
        for s in sites:
            gs.append(gates.beam_splitter_gate(*ang[k], d))
            k += 1
        g.apply_layer(sites, gs, 512, 0.0)
        for s, G in zip(sites, gs):
            st.apply_gate2(s, G, 512, 0.0)
    U = tebd.interferometer(M, layers, ang)
    rng = np.random.default_rng(4)
    cfgs = [W.random_occupations(M, d, n, rng) for _ in range(40)]
    ag = g.amplitudes(cfgs)
    for c, a in zip(cfgs, ag):
        rows = [j for j in range(M) for _ in range(c[j])]
        p = abs(permanent.permanent_bruteforce(U[np.ix_(rows, list(range(n)))])) ** 2
        p /= np.prod([math.factorial(x) for x in c])
        assert abs(abs(a) ** 2 - p) < 1e-12
    # an amplitude is gauge invariant (bond gauges cancel in the chain), so compare it directly
    ao = np.array([st.amplitude(c) for c in cfgs])
    assert np.max(np.abs(ag - ao)) < 1e-10


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_two_sites_and_chi_one(gpu_lib):
    g = _gpu(gpu_lib, 2, [1, 0], 4)
    st = U1MPS.product(2, [1, 0])
    G = gates.xxz_gate(0.3, 0.7)
    g.apply_gate2(0, G, 1, 1e-10)
    st.apply_gate2(0, G, 1, 1e-10)
    compare_update(g, st, 0)
    assert g.bond_dims(1) == st.bond[1]


def test_product_state_amplitudes_and_bad_configs(gpu_lib):
    occ = [2, 0, 1, 3, 0]
    g = _gpu(gpu_lib, 4, occ, 8)
    assert g.amplitude(occ) == 1.0
    assert g.amplitude([2, 0, 1, 2, 1]) == 0.0        # same N, absent block
    assert g.amplitude([2, 0, 1, 3, 1]) == 0.0        # wrong N
    assert g.amplitude([5, 0, 1, 0, 0]) == 0.0        # occupation out of range
    assert abs(g.expect(3, [0, 1, 2, 3]) - 3.0) < 1e-15


def test_invalid_arguments(gpu_lib):
    m = gpu_lib
    g = _gpu(m, 2, [1, 0, 1, 0], 8)
    G = gates.xxz_gate(0.5, 0.1)
    with pytest.raises(m.MPSError):
        g.apply_gate2(3, G, 4, 1e-10)          # site + 1 out of range
    with pytest.raises(m.MPSError):
        g.apply_gate2(0, G, 9, 1e-10)          # chi > chi_max
    with pytest.raises(m.MPSError):
        g.apply_gate2(0, G, 4, -1.0)           # negative cutoff
    with pytest.raises(m.MPSError):
        g.apply_layer([0, 1], [G, G], 4, 1e-10)  # overlapping pairs
    with pytest.raises(m.MPSError):
        m.MPS(2, [1, 2], 4)                    # occupation outside [0, d-1]
    with pytest.raises(m.MPSError):
        m.MPS(2, [1, 0], 4, precision=7)        # no such precision mode


def test_annihilating_gate_leaves_state_unchanged(gpu_lib):
    m = gpu_lib
    g = _gpu(m, 2, [1, 0, 1, 0], 8)
    zero = [np.zeros_like(b) for b in gates.xxz_gate(0.5, 0.1)]
    before = g.site(1)
    with pytest.raises(m.MPSError):
        g.apply_gate2(1, zero, 4, 1e-10)
    after = g.site(1)
    assert before.keys() == after.keys()


# ---------------------------------------------------------------------------
# full size: the Bose-Hubbard L=64, chi=512 chain at saturation, one odd layer
# launched like the benchmark; sampled updates recomputed by the oracle
# ---------------------------------------------------------------------------
def test_full_size_bose_hubbard_layer_sampled(gpu_lib):
    L, d, N, chi = 64, 5, 64, 512
    st = random_state(L, d, N, chi, seed=11, occ=W.mott_occupations(L))
    g = _gpu(gpu_lib, d, W.mott_occupations(L), chi)
    load_state(g, st)
    gate_of = tebd.bh_gates(L, d, 1.0, 2.0, 0.02)
    sites = list(range(0, L - 1, 2))
    g.apply_layer(sites, [gate_of(s, 0.5) for s in sites], chi, 1e-10)
    for s in (0, 30, 32, 62):
        ref = st.copy()
        ref.apply_gate2(s, gate_of(s, 0.5), chi, 1e-10)
        compare_update(g, ref, s, tol_lam=1e-12, tol_prod=1e-8)


# ---------------------------------------------------------------------------
# checkpoint: mps_save / mps_load
# ---------------------------------------------------------------------------
def test_save_load_round_trip_continues_bit_for_bit(gpu_lib, tmp_path):
    m = gpu_lib
    L, d = 10, 3
    gate_of = tebd.bh_gates(L, d, 1.0, 2.0, 0.05)
    a = _gpu(m, d, W.mott_occupations(L), 40)
    layers = tebd.strang_layers(L)
    for sites, f in layers * 3:
        a.apply_layer(sites, [gate_of(s, f) for s in sites], 40, 1e-10)
    path = tmp_path / "state.u1mps"
    a.save(path)
    b = m.MPS.load(path)
    assert (b.L, b.d, b.N, b.chi_max) == (a.L, a.d, a.N, a.chi_max)
    for bond in range(L + 1):
        ba, bb = a.bond(bond), b.bond(bond)
        assert ba.keys() == bb.keys() and all(np.array_equal(ba[c], bb[c]) for c in ba)
    for sites, f in layers * 2:   # both continue identically
        a.apply_layer(sites, [gate_of(s, f) for s in sites], 40, 1e-10)
        b.apply_layer(sites, [gate_of(s, f) for s in sites], 40, 1e-10)
    for s in range(L):
        sa, sb = a.site(s), b.site(s)
        assert sa.keys() == sb.keys() and all(np.array_equal(sa[k], sb[k]) for k in sa)


def _round_trip(m, a, layers, gate_of, chi, tmp_path, name):
    """Save a, load it back, continue both by the same layers: identical bonds and blocks."""
    path = tmp_path / f"{name}.u1mps"
    a.save(path)
    b = m.MPS.load(path)
    assert (b.L, b.d, b.N, b.chi_max, b.zn, b.charges) == (a.L, a.d, a.N, a.chi_max, a.zn, a.charges)
    for bond in range(a.L + 1):
        ba, bb = a.bond(bond), b.bond(bond)
        assert ba.keys() == bb.keys() and all(np.array_equal(ba[c], bb[c]) for c in ba)
    for sites, f in layers:
        a.apply_layer(sites, [gate_of(s, f) for s in sites], chi, 1e-10)
        b.apply_layer(sites, [gate_of(s, f) for s in sites], chi, 1e-10)
    for s in range(a.L):
        sa, sb = a.site(s), b.site(s)
        assert sa.keys() == sb.keys() and all(np.array_equal(sa[k], sb[k]) for k in sa)
    b.close()


def test_round_trip_of_every_charge_rule_and_of_the_deflation_ages(gpu_lib, tmp_path):
    """Checkpoints of Z_n (d = n and d < n) and several-U(1) handles; and a U(1) handle saved
    after an even layer and continued by an odd one: the odd bonds' cuts are two update calls
    old there, on the loaded handle as on the saved one (their deflation level depends on it)."""
    m = gpu_lib
    from oracle import multiu1
    from oracle.gates import bh_weights
    L = 10
    layers = tebd.strang_layers(L)
    # U(1), saved after an even layer
    gate_of = tebd.bh_gates(L, 3, 1.0, 2.0, 0.05)
    a = _gpu(m, 3, W.mott_occupations(L), 24)
    for sites, f in layers * 2 + layers[:2]:
        a.apply_layer(sites, [gate_of(s, f) for s in sites], 24, 1e-10)
    _round_trip(m, a, layers, gate_of, 24, tmp_path, "u1")
    # Z_3 clock chain (d = n) and Bose-Hubbard on Z_4 (d = 3 < n)
    for d, n, model, p in ((3, 3, "clock", dict(J=1.0, f=0.6)), (3, 4, "bh", dict(J=1.0, U=2.0, zn=4))):
        table = m.tebd.GateTable(model, L, d, 0.1, **p)
        a = m.MPS(d, [(2 * s) % d for s in range(L)], 16, zn=n)
        for sites, f in layers * 2:
            a.apply_layer(sites, [table(s, f) for s in sites], 16, 1e-10)
        _round_trip(m, a, layers, table, 16, tmp_path, f"z{n}_{d}")
    # two species of hard-core bosons
    Q = multiu1.TWO_SPECIES_Q
    a = m.MPS(4, [s % 4 for s in range(L)], 16, charges=Q)
    gq = lambda s, f: multiu1.two_species_gate(1.0, 2.0, *bh_weights(L, s), f * 0.05)
    for sites, f in layers * 2:
        a.apply_layer(sites, [gq(s, f) for s in sites], 16, 1e-10)
    _round_trip(m, a, layers, gq, 16, tmp_path, "two_species")
    a.close()


def test_load_rejects_missing_and_damaged_files(gpu_lib, tmp_path):
    m = gpu_lib
    with pytest.raises(m.MPSError):
        m.MPS.load(tmp_path / "missing.u1mps")
    a = _gpu(m, 2, W.neel_occupations(8), 16)
    G = gates.xxz_gate(0.5, 0.1)
    a.apply_layer([0, 2, 4, 6], [G] * 4, 16, 1e-10)
    good = tmp_path / "good.u1mps"
    a.save(good)
    raw = good.read_bytes()
    for name, blob in [("truncated", raw[: len(raw) // 2]), ("no_trailer", raw[:-8]),
                       ("bad_magic", b"X" + raw[1:])]:
        p = tmp_path / f"{name}.u1mps"
        p.write_bytes(blob)
        with pytest.raises(m.MPSError):
            m.MPS.load(p)
    # a charge table with a charge outside the bond's range is refused
    import struct
    hdr = struct.calcsize("<8s6i") + 4   # magic, header, the rule record of a U(1) handle (kind 0)
    assert struct.unpack_from("<i", raw, 8)[0] == 3 and struct.unpack_from("<i", raw, hdr - 4)[0] == 0
    L = 8
    off = hdr
    for b in range(L + 1):   # walk to bond 1's first charge
        n = struct.unpack_from("<i", raw, off)[0]
        if b == 1:
            bad = bytearray(raw)
            struct.pack_into("<i", bad, off + 4, 99)
            p = tmp_path / "bad_charge.u1mps"
            p.write_bytes(bytes(bad))
            with pytest.raises(m.MPSError):
                m.MPS.load(p)
            break
        dims = struct.unpack_from(f"<{n}i", raw, off + 4 + 4 * n)
        off += 4 + 8 * n + 8 * sum(dims)


def test_deflation_from_the_previous_cut_and_its_redo(gpu_lib):
    """The second update of a bond deflates its SVDs from the first one's cut.  With a
    much larger chi the new cut falls far below that estimate, so the update must be
    redone without the deflation level; both updates match the oracle."""
    L, d, N = 8, 3, 8
    st = random_state(L, d, N, 60, seed=5)
    g = _gpu(gpu_lib, d, [1] * L, 80)
    load_state(g, st)
    G = gates.bh_gate(L, 3, d, 1.0, 2.0, 0.4)
    s = 3
    seen = []
    for chi in (6, 6, 40):        # no history, then a similar cut, then a far lower cut
        g.apply_gate2(s, G, chi, 1e-10)
        st.apply_gate2(s, G, chi, 1e-10)
        compare_update(g, st, s)
        seen.append(g.deflation_stats())
    assert seen[0] == dict(deflated_updates=0, redos=0), seen
    assert seen[2]["deflated_updates"] == 2, seen
    assert seen[2]["redos"] - seen[1]["redos"] == 1, seen      # the 40th value is far below the 6th


# ---------------------------------------------------------------------------
# the benchmark chain's own trajectory: Bose-Hubbard L=64, n_max=4, N=64, J=1, U=2,
# dt=0.02, chi<=512, cutoff 1e-10, evolved from the Mott state on both sides
# ---------------------------------------------------------------------------
BH64_STEPS = 30        # Strang steps the float64 oracle finishes in about a minute on 16 cores


def test_bose_hubbard_L64_trajectory_from_mott(gpu_lib):
    """Sec. II update, evolved the way the benchmark launches it (a stream of its own,
    CUDA graphs on, one mps_apply_layer per Strang layer).  After every layer the kept
    sector labels and dimensions of every bond equal the oracle's and every Schmidt
    value agrees to 1e-12; after every step <n_i> and the bond entropies agree to
    1e-9 * max(|ref|, |O|) (|O| = n_max for n, ln chi for the entropy)."""
    import torch
    m = gpu_lib
    L, d, N, J, U, dt, chi, cutoff = 64, 5, 64, 1.0, 2.0, 0.02, 512, 1e-10
    stream = torch.cuda.Stream()
    g = m.MPS(d, W.mott_occupations(L), chi, stream=stream.cuda_stream)
    g.set_graphs(True)
    st = U1MPS.product(d, W.mott_occupations(L))
    gate_of = tebd.bh_gates(L, d, J, U, dt)
    n_op = np.arange(d)
    worst_lam = worst_obs = 0.0
    for step in range(BH64_STEPS):
        for sites, f in tebd.strang_layers(L):
            g.apply_layer(sites, [gate_of(s, f) for s in sites], chi, cutoff)
            for s in sites:
                st.apply_gate2(s, gate_of(s, f), chi, cutoff)
            for b in range(L + 1):
                gb = g.bond(b)
                assert {c: len(v) for c, v in gb.items()} == st.bond[b], (step, b)
                for c, v in gb.items():
                    e = float(np.max(np.abs(v - st.lam[b][c])))
                    worst_lam = max(worst_lam, e)
                    assert e <= 1e-12, (step, b, c, e)
        for s in range(L):
            ref = st.expect_local(s, n_op)
            e = abs(g.expect(s, n_op) - ref)
            worst_obs = max(worst_obs, e / max(abs(ref), d - 1))
            assert e <= 1e-9 * max(abs(ref), d - 1), (step, s, e)
        for b in range(1, L):
            ref = st.entropy(b)
            e = abs(g.entropy(b) - ref)
            assert e <= 1e-9 * max(abs(ref), math.log(chi)), (step, b, e)
    print(f"L=64 trajectory, {BH64_STEPS} steps: largest bond {max(st.bond_dim(b) for b in range(L + 1))}, "
          f"lambda err {worst_lam:.2e}, <n_i> rel err {worst_obs:.2e}")
    assert g.graph_stats()["launches"] > 0
    g.close()
