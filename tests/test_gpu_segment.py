"""Chain segmentation on the GPU: two ranks, each a process with its own segment handle
(mps_create_segment) on the same GPU, exchanging the sites next to the cut over gloo
(host buffers) before every layer that has an update across the cut (Sec. II: independent
two-site updates are distributed across GPUs).  The ranks' kernels never wait on one
another: every exchange goes through the host between layers.

The gathered segmented state must equal a single-handle run of the same chain bit for
bit (each update is computed from the same inputs by the same kernels, whichever other
updates share its launches), and match the float64 oracle within the FP64 tolerances.
"""
import os
import pickle
import socket

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "xxz": dict(L=16, d=2, occ=W.neel_occupations(16), chi=16, steps=8, model="xxz", param=0.5, dt=0.1),
    "bh": dict(L=12, d=4, occ=W.mott_occupations(12), chi=40, steps=4, model="bh", param=2.0, dt=0.05),
}


def _gate_table(m, c):
    if c["model"] == "xxz":
        return m.tebd.GateTable("xxz", c["L"], c["d"], c["dt"], delta=c["param"])
    return m.tebd.GateTable("bh", c["L"], c["d"], c["dt"], J=1.0, U=c["param"])


def _worker(rank, world, port, case, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_2303_11409_gb300 as m
    from paper_2303_11409_gb300.segment import GpuEngine, Segment, SegmentedTEBD
    c = CASES[case]
    seg = Segment(c["L"], world, rank)
    run = SegmentedTEBD(seg, GpuEngine(seg, c["d"], c["occ"], c["chi"]), dist)
    gates = _gate_table(m, c)
    for _ in range(c["steps"]):
        for sites, f in m.tebd.strang_layers(c["L"]):
            run.layer(sites, gates, f, c["chi"], 1e-10)
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


@pytest.mark.parametrize("case", ["xxz", "bh"])
def test_segmented_gpu_run_equals_one_handle_bit_for_bit(gpu_lib, tmp_path, case):
    import multiprocessing as mp
    from oracle import U1MPS, tebd as otebd
    from paper_2303_11409_gb300.segment import place_blocks
    m = gpu_lib
    c = CASES[case]
    world = 2
    out = str(tmp_path / "gathered.pkl")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    with open(out, "rb") as fh:
        (bonds, sites), exchanges = pickle.load(fh)
    assert exchanges == c["steps"]                    # one exchange per even layer

    # the same chain on one handle
    L = c["L"]
    one = m.MPS(c["d"], c["occ"], c["chi"])
    gates = _gate_table(m, c)
    for _ in range(c["steps"]):
        for s_, f in m.tebd.strang_layers(L):
            one.apply_layer(s_, [gates(x, f) for x in s_], c["chi"], 1e-10)
    assert max(sum(one.bond_dims(b).values()) for b in range(L + 1)) == c["chi"]   # the cut was active
    for b in range(1, L):
        ref = one.bond(b)
        assert bonds[b].keys() == ref.keys(), b
        for ch in ref:
            assert np.array_equal(bonds[b][ch], ref[ch]), (b, ch)
    for s in range(L):
        pairs, data = sites[s]
        right = one.bond_dims(s + 1)
        blocks = place_blocks(pairs, data, {ch: len(v) for ch, v in bonds[s].items()}, right)
        ref = one.site(s)
        assert blocks.keys() == ref.keys(), s
        for k in ref:
            assert np.array_equal(blocks[k], ref[k]), (s, k)

    # and the oracle agrees (FP64 tolerances: exact bond tables, lambda to 1e-12)
    o = U1MPS.product(c["d"], c["occ"])
    og = (otebd.xxz_gates(L, c["param"], c["dt"]) if c["model"] == "xxz"
          else otebd.bh_gates(L, c["d"], 1.0, c["param"], c["dt"]))
    otebd.run_tebd(o, og, c["steps"], c["chi"], 1e-10)
    for b in range(1, L):
        assert {ch: len(v) for ch, v in bonds[b].items()} == o.bond[b], b
        for ch, v in o.lam[b].items():
            assert np.max(np.abs(bonds[b][ch] - v)) <= 1e-12, (b, ch)
    one.close()
