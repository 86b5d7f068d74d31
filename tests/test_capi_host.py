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
