"""Chain segmentation across ranks (gloo, world size 2 and 3, on the CPU).

One chain split into contiguous segments, one per rank, with one exchange of the sites
next to each cut before every layer that has updates across a cut (Sec. II: independent
two-site updates are distributed across GPUs and nodes).  The segmentation logic is the
library's (paper_2303_11409_gb300.segment); the per-rank engine here is the float64
oracle, so the test runs without a GPU.  The segmented run must equal the single-process
run bit for bit: every update is computed from the same inputs by the same code.
"""
import os
import pickle
import socket

import numpy as np
import pytest

from oracle import U1MPS, tebd
from paper_2303_11409_gb300.segment import Segment, SegmentedTEBD, cuts, place_blocks, unpack
import workloads as W

CASES = {
    "xxz": dict(L=12, d=2, occ=W.neel_occupations(12), chi=8, steps=4),
    "bh": dict(L=10, d=3, occ=W.mott_occupations(10), chi=12, steps=3),
}


class OracleEngine:
    """The engine interface of SegmentedTEBD over the oracle's state."""

    def __init__(self, d, occ):
        self.st = U1MPS.product(d, occ)

    def apply_layer(self, sites, gates, chi, cutoff):
        for s, G in zip(sites, gates):
            self.st.apply_gate2(s, G, chi, cutoff)

    def bond(self, b):
        return {c: v.copy() for c, v in self.st.lam[b].items()}

    def site(self, s):
        return {k: v.copy() for k, v in self.st.B[s].items()}

    def bond_dims(self, b):
        return dict(self.st.bond[b])

    def load(self, bond, lam, site, blocks):
        self.st.lam[bond] = {c: np.array(v) for c, v in lam.items()}
        self.st.bond[bond] = {c: len(v) for c, v in lam.items()}
        self.st.B[site] = blocks


def _gates(case):
    c = CASES[case]
    if case == "xxz":
        return tebd.xxz_gates(c["L"], 0.5, 0.1)
    return tebd.bh_gates(c["L"], c["d"], 1.0, 2.0, 0.1)


def _worker(rank, world, port, case, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = CASES[case]
    seg = Segment(c["L"], world, rank)
    run = SegmentedTEBD(seg, OracleEngine(c["d"], c["occ"]), dist)
    gate_of = _gates(case)
    for _ in range(c["steps"]):
        for sites, f in tebd.strang_layers(c["L"]):
            run.layer(sites, gate_of, f, c["chi"], 1e-10)
    got = run.gather()
    if rank == 0:
        with open(out_path, "wb") as fh:
            pickle.dump((got, run.exchanges), fh)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_cuts_are_even_and_cover_the_chain():
    for L in range(4, 40):
        for world in range(1, L // 2 + 1):
            b = cuts(L, world)
            assert b[0] == 0 and b[-1] == L and len(b) == world + 1
            assert all(x % 2 == 0 for x in b[1:-1])
            assert all(b[i + 1] - b[i] >= 2 for i in range(world))
    seg = Segment(12, 2, 1)
    assert (seg.lo, seg.hi) == (6, 12)
    assert seg.updates([1, 3, 5, 7, 9]) == [5, 7, 9]        # 5 straddles the cut at 6
    assert seg.updates([0, 2, 4, 6, 8, 10]) == [6, 8, 10]
    assert seg.straddles([1, 3, 5, 7, 9]) and not seg.straddles([0, 2, 4, 6, 8, 10])


@pytest.mark.parametrize("case,world", [("xxz", 2), ("xxz", 3), ("bh", 2)])
def test_segmented_run_equals_single_process_bit_for_bit(tmp_path, case, world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = str(tmp_path / "gathered.pkl")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    with open(out, "rb") as fh:
        (bonds, sites), exchanges = pickle.load(fh)
    c = CASES[case]
    ref = U1MPS.product(c["d"], c["occ"])
    tebd.run_tebd(ref, _gates(case), c["steps"], c["chi"], 1e-10)
    L = c["L"]
    assert exchanges == c["steps"]                           # one per even layer
    assert max(ref.bond_dim(b) for b in range(L + 1)) == c["chi"]   # the cut was active
    for b in range(L):
        assert bonds[b].keys() == ref.lam[b].keys()
        for ch in bonds[b]:
            assert np.array_equal(bonds[b][ch], ref.lam[b][ch])
    for s in range(L):
        pairs, data = sites[s]
        right = ref.bond[s + 1]
        blocks = place_blocks(pairs, data, {ch: len(v) for ch, v in bonds[s].items()}, right)
        assert blocks.keys() == ref.B[s].keys()
        for k in blocks:
            assert np.array_equal(blocks[k], ref.B[s][k]), (s, k)


def test_pack_round_trip():
    from paper_2303_11409_gb300.segment import pack
    rng = np.random.default_rng(0)
    lam = {2: np.array([0.8, 0.1]), 3: np.array([0.5])}
    blocks = {(2, 1): W.random_complex((2, 3), rng), (3, 3): W.random_complex((1, 4), rng)}
    site, bond, lam2, pairs, data = unpack(pack(5, 5, lam, blocks))
    assert (site, bond) == (5, 5)
    assert all(np.array_equal(lam[c], lam2[c]) for c in lam)
    got = place_blocks(pairs, data, {2: 2, 3: 1}, {1: 3, 3: 4})
    assert all(np.array_equal(got[k], blocks[k]) for k in blocks)
