"""The C-ABI library on the CPU: it loads, exports every declared symbol, and its
integer planner (host code) is bit-exact with the oracle's enumeration."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^MPS_API\s+[\w\s\*]+?\b(mps_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    b = g._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_library_exports_every_declared_symbol(built):
    declared = _declared_symbols()
    assert len(declared) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mps_\w+)", out))
    assert declared <= exported, declared - exported
    import paper_2303_11409_gb300 as m
    for name in declared:
        assert hasattr(m.lib, name)
    assert set(m.EXPORTED) == declared


def _rand_table(rng, lo, hi):
    ch = sorted(rng.choice(np.arange(lo, hi + 1), size=int(rng.integers(1, hi - lo + 2)), replace=False))
    return {int(c): int(rng.integers(1, 40)) for c in ch}


@pytest.mark.parametrize("d", [2, 3, 5, 8])
def test_planner_matches_oracle(built, d):
    import paper_2303_11409_gb300 as m
    from oracle import plan_update
    rng = np.random.default_rng(100 + d)
    for _ in range(50):
        base = int(rng.integers(0, 9))
        left = _rand_table(rng, base + 2 * (d - 1), base + 4 * (d - 1))
        mid = _rand_table(rng, base + (d - 1), base + 3 * (d - 1))
        right = _rand_table(rng, base, base + 2 * (d - 1))
        tri, sec = m.plan_sectors(d, left, mid, right)
        p = plan_update(left, mid, right, d)
        assert [tuple(t) for t in tri.tolist()] == p.triples
        assert sec[:, 0].tolist() == p.sectors
        for (c, rows, cols) in sec.tolist():
            assert rows == sum(left[l] for l in p.rows[c])
            assert cols == sum(right[r] for r in p.cols[c])


def test_planner_rejects_bad_tables(built):
    import paper_2303_11409_gb300 as m
    with pytest.raises(m.MPSError):
        m.plan_sectors(1, {1: 1}, {0: 1}, {0: 1})
    with pytest.raises(m.MPSError):
        m.lib_plan = m.plan_sectors(2, {1: 0}, {0: 1}, {0: 1})


def test_svd_work_bytes_host(built):
    import paper_2303_11409_gb300 as m
    assert m.svd_work_bytes([4, 5], [3, 2]) > 0
    assert m.svd_work_bytes([0], [3]) == -1
    small = m.svd_work_bytes([10], [10])
    big = m.svd_work_bytes([300], [300])
    assert big >= 16 * 300 * 300 > small


def test_load_rejects_impossible_headers_without_touching_the_gpu(built, tmp_path):
    """mps_load checks the header and every size against the file before it creates a
    handle or sizes anything: a damaged or hostile checkpoint is refused with MPS_EINVAL
    (no exception crosses the C boundary, no device call is made)."""
    import ctypes
    import struct
    import paper_2303_11409_gb300 as m
    h = ctypes.c_void_p()
    cases = {
        "huge_L": struct.pack("<8s6i", b"U1MPSCK1", 2, 1 << 30, 5, 10, 64, 0),
        "L_times_d_overflows": struct.pack("<8s6i", b"U1MPSCK1", 2, (1 << 24), 8, (1 << 31) - 1, 64, 0),
        "short_file": struct.pack("<8s6i", b"U1MPSCK1", 2, 1000, 5, 10, 64, 0) + b"\0" * 64,
        "negative_N": struct.pack("<8s6i", b"U1MPSCK1", 2, 8, 2, -1, 8, 0),
    }
    for name, blob in cases.items():
        p = tmp_path / f"{name}.u1mps"
        p.write_bytes(blob)
        rc = m.lib.mps_load(ctypes.byref(h), str(p).encode(), None)
        assert rc == m.MPS_EINVAL, (name, rc)
        assert not h.value


def _check_rule_plan(got, p, left, right):
    triples, sectors = got
    assert triples == p.triples
    assert [s[0] for s in sectors] == p.sectors
    for c, rows, cols, rl, cl in sectors:
        assert rl == p.rows[c] and cl == p.cols[c]
        assert rows == sum(left[l] for l in rl)
        assert cols == sum(right[r] for r in cl)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_rule_planner_u1_equals_the_u1_planner(built, d):
    import paper_2303_11409_gb300 as m
    from oracle import plan_update
    rng = np.random.default_rng(300 + d)
    for _ in range(20):
        base = int(rng.integers(0, 9))
        left = _rand_table(rng, base + 2 * (d - 1), base + 4 * (d - 1))
        mid = _rand_table(rng, base + (d - 1), base + 3 * (d - 1))
        right = _rand_table(rng, base, base + 2 * (d - 1))
        _check_rule_plan(m.plan_sectors_rule(d, left, mid, right), plan_update(left, mid, right, d), left, right)


@pytest.mark.parametrize("n,d", [(2, 2), (3, 3), (4, 4), (7, 7), (3, 2), (4, 3), (5, 3), (7, 4), (9, 5)])
def test_rule_planner_matches_the_zn_oracle(built, n, d):
    """Z_n (oracle/znmps.py): for d = n all triples, every residue a sector, all rows and
    columns; for d < n the triples, sectors, rows and columns whose residue differences are
    physical indices (listed, in general not one run of the table)."""
    import paper_2303_11409_gb300 as m
    from oracle import znmps
    rng = np.random.default_rng(400 + 10 * n + d)
    for _ in range(20):
        left, mid, right = (_rand_table(rng, 0, n - 1) for _ in range(3))
        got = m.plan_sectors_rule(d, left, mid, right, zn=n)
        _check_rule_plan(got, znmps.plan_update(left, mid, right, n, d), left, right)


def _rand_tuple_table(rng, lo, hi, k):
    """A random set of charge vectors with components in [lo_j, hi_j] and random dims."""
    pts = {tuple(int(rng.integers(lo[j], hi[j] + 1)) for j in range(len(lo))) for _ in range(k)}
    return {c: int(rng.integers(1, 30)) for c in pts}


@pytest.mark.parametrize("q", [
    [(0, 0), (0, 1), (1, 0), (1, 1)],                         # two boson species, at most one each
    [(0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0), (1, 1, 0)],  # three species, one pair allowed
    [(0,), (2,), (3,)],                                        # one charge with gaps (listed rows)
])
def test_rule_planner_matches_the_several_u1_oracle(built, q):
    """Several U(1) charges (oracle/multiu1.py): listed rows and columns, encoded charges."""
    import paper_2303_11409_gb300 as m
    from oracle import multiu1
    rng = np.random.default_rng(500 + len(q))
    nc = len(q[0])
    top = [max(x[j] for x in q) for j in range(nc)]
    for _ in range(25):
        base = [int(rng.integers(0, 4)) for _ in range(nc)]
        right = _rand_tuple_table(rng, base, [b + 2 * t for b, t in zip(base, top)], 8)
        mid = _rand_tuple_table(rng, base, [b + 3 * t for b, t in zip(base, top)], 10)
        left = _rand_tuple_table(rng, base, [b + 4 * t for b, t in zip(base, top)], 12)
        got = m.plan_sectors_rule(len(q), left, mid, right, charges=q)
        p = multiu1.plan_update(left, mid, right, q)
        assert p.sectors, "no sector: the random tables do not couple"
        _check_rule_plan(got, p, left, right)


def test_rule_planner_rejects_bad_rules(built):
    import paper_2303_11409_gb300 as m
    t = {0: 1, 1: 2}
    with pytest.raises(m.MPSError):
        m.plan_sectors_rule(3, t, t, t, zn=2)                  # Z_n only for d <= n
    with pytest.raises(m.MPSError):
        m.plan_sectors_rule(3, {0: 1, 3: 1}, t, t, zn=3)       # residue outside [0, n-1]
    q = [(0, 0), (0, 1), (1, 0), (1, 1)]
    tt = {(0, 0): 1, (1, 1): 2}
    with pytest.raises(m.MPSError):                            # a component beyond radix / 2
        m.plan_sectors_rule(4, {(3, 0): 1}, tt, tt, charges=q, radix=[5, 5])
    with pytest.raises(m.MPSError):                            # physical charges not ascending
        m.plan_sectors_rule(4, tt, tt, tt, charges=[(0, 1), (0, 0), (1, 0), (1, 1)])
    with pytest.raises(m.MPSError):                            # radix below 2
        m.plan_sectors_rule(4, tt, tt, tt, charges=q, radix=[1, 5])


def test_load_rejects_bad_rule_records_without_touching_the_gpu(built, tmp_path):
    """Version-3 checkpoints carry the charge rule after the header; an unknown kind, a Z_n
    with n below d, a residue total charge at or above n, or a bad several-U(1) record is
    refused before any handle exists."""
    import ctypes
    import struct
    import paper_2303_11409_gb300 as m
    h = ctypes.c_void_p()
    head = lambda N: struct.pack("<8s6i", b"U1MPSCK1", 3, 8, 3, N, 16, 0)
    pad = b"\0" * 4096
    cases = {
        "unknown_kind": head(2) + struct.pack("<i", 7) + pad,
        "zn_below_d": head(1) + struct.pack("<2i", 1, 2) + pad,
        "residue_too_large": head(5) + struct.pack("<2i", 1, 4) + pad,
        "no_components": head(0) + struct.pack("<2i", 2, 0) + pad,
        "radix_below_two": head(0) + struct.pack("<4i", 2, 2, 1, 9) + pad,
        "version_4": struct.pack("<8s6i", b"U1MPSCK1", 4, 8, 3, 2, 16, 0) + pad,
    }
    for name, blob in cases.items():
        p = tmp_path / f"{name}.u1mps"
        p.write_bytes(blob)
        rc = m.lib.mps_load(ctypes.byref(h), str(p).encode(), None)
        assert rc == m.MPS_EINVAL, (name, rc)
        assert not h.value


def test_gate_layout_matches_the_oracles_gate_bases(built):
    """mps_gate_layout against the oracle's gate bases: U(1) blocks over (i, n - i)
    (oracle.gate_basis), Z_n blocks over (i, (q - i) mod n) with both entries below d
    (oracle.znmps.zn_blocks_of), several U(1) charges over the pairs of each vector total
    (oracle.multiu1.pair_blocks); the binding checks every gate against this length."""
    import paper_2303_11409_gb300 as m
    from oracle import gate_basis
    from oracle.multiu1 import pair_blocks
    from oracle.znmps import zn_blocks_of, zn_charges
    for d in range(2, 9):
        sizes, length = m.gate_layout(d)
        want = [len(gate_basis(n, d)) for n in range(2 * d - 1)]
        assert sizes == want and length == sum(k * k for k in want)
        assert length == m.gate_length(d)
        for n in (d, d + 1, d + 3, 2 * d + 1):
            sizes, length = m.gate_layout(d, zn=n)
            want = [len(zn_blocks_of(n, q, d)) for q in zn_charges(n, d)]
            assert sizes == want and length == sum(k * k for k in want)
            assert length == sum(len(p) ** 2 for p in m._binding.cyclic_pair_blocks(n, d).values())
    for q in ([(0, 0), (0, 1), (1, 0), (1, 1)], [(0,), (2,), (3,)],
              [(0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0), (1, 1, 0)]):
        sizes, length = m.gate_layout(len(q), charges=q)
        keys, pairs = pair_blocks(q)
        want = [len(pairs[k]) for k in keys]
        assert sizes == want and length == sum(k * k for k in want)
        assert length == sum(len(p) ** 2 for p in m._binding.multi_pair_blocks(q).values())
    with pytest.raises(m.MPSError):
        m.gate_layout(3, zn=2)                                     # Z_n needs d <= n
    with pytest.raises(m.MPSError):
        m.gate_layout(2, charges=[(1, 0), (0, 1)])                 # not ascending
