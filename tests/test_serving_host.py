"""Host-side serving logic (no GPU): footprint estimates used for admission."""
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    b = g._build_module()
    import os
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2303_11409_gb300 as m
    return m


def test_footprint_grows_with_chi_and_length(lib):
    a1, w1 = lib.footprint_bytes(32, 5, 32, 64)
    a2, w2 = lib.footprint_bytes(32, 5, 32, 256)
    a3, w3 = lib.footprint_bytes(64, 5, 64, 256)
    assert 0 < a1 < a2 < a3
    assert 0 < w1 < w2 < w3


def test_footprint_saturates_at_the_hilbert_bound(lib):
    # L=8 spin-1/2 at half filling: the middle bond's Hilbert bound is 16, so beyond that
    # the arena stops growing with chi
    a_small, _ = lib.footprint_bytes(8, 2, 4, 64)
    a_big, _ = lib.footprint_bytes(8, 2, 4, 4096)
    assert a_small == a_big


def test_footprint_rejects_bad_arguments(lib):
    with pytest.raises(lib.MPSError):
        lib.footprint_bytes(1, 2, 0, 4)
    with pytest.raises(lib.MPSError):
        lib.footprint_bytes(8, 2, 9, 4)          # more particles than the chain holds


def test_request_too_big_for_the_budget_is_refused_up_front(lib):
    big = lib.serve.Request(0, "bh", 64, 512, 1, 2.0)
    small = lib.serve.Request(1, "xxz", 8, 8, 1, 0.5)
    lib.serve.check_admissible([small], 1 << 30)
    with pytest.raises(ValueError):
        lib.serve.check_admissible([small, big], 1 << 30)
    assert lib.serve.footprint(big) > lib.serve.footprint(small)
