"""Pins the oracle's sector enumeration (brute force) and its global truncation rule."""
import math

import numpy as np
import pytest

from oracle import TIE_REL, gate_basis, plan_update, select_kept


def _random_bond(rng, lo, hi):
    charges = sorted(rng.choice(np.arange(lo, hi + 1), size=rng.integers(1, hi - lo + 2), replace=False))
    return {int(c): int(rng.integers(1, 9)) for c in charges}


@pytest.mark.parametrize("d", [2, 3, 5])
def test_plan_matches_bruteforce(d):
    rng = np.random.default_rng(d)
    for _ in range(40):
        base = int(rng.integers(0, 6))
        left = _random_bond(rng, base + 2 * (d - 1), base + 4 * (d - 1))
        mid = _random_bond(rng, base + (d - 1), base + 3 * (d - 1))
        right = _random_bond(rng, base, base + 2 * (d - 1))
        plan = plan_update(left, mid, right, d)
        brute = set()
        for l in left:
            for i in range(d):
                for j in range(d):
                    m, r = l - i, l - i - j
                    if m in mid and r in right:
                        brute.add((l, m, r))
        assert sorted(brute) == plan.triples
        # every (l, r) pair and every output occupation split gives one sector entry
        brute_sec = {}
        for l in left:
            for r in right:
                for ip in range(d):
                    c = l - ip
                    if 0 <= c - r <= d - 1:
                        brute_sec.setdefault(c, set()).add((l, r))
        assert sorted(brute_sec) == plan.sectors
        for c in plan.sectors:
            assert {(l, r) for l in plan.rows[c] for r in plan.cols[c]} == brute_sec[c]


def test_gate_basis():
    assert gate_basis(0, 5) == [0]
    assert gate_basis(4, 5) == [0, 1, 2, 3, 4]
    assert gate_basis(8, 5) == [4]
    assert gate_basis(6, 5) == [2, 3, 4]
    assert sum(len(gate_basis(n, 5)) for n in range(9)) == 25


def _brute_select(sig, chi, cutoff):
    allv = [(v, c, i) for c in sorted(sig) for i, v in enumerate(sig[c])]
    norm = math.sqrt(sum(v * v for v, _, _ in allv))
    cand = [t for t in allv if t[0] > cutoff * norm]
    cand.sort(key=lambda t: (-t[0], t[1], t[2]))
    kept = {c: 0 for c in sig}
    for _, c, _ in cand[:chi]:
        kept[c] += 1
    return kept


def test_selection_matches_sort_without_ties():
    rng = np.random.default_rng(7)
    for _ in range(200):
        sig = {}
        for c in range(int(rng.integers(1, 8))):
            k = int(rng.integers(1, 12))
            sig[c] = np.sort(rng.random(k) ** 3)[::-1]
        chi = int(rng.integers(1, 40))
        cutoff = float(rng.choice([0.0, 1e-3, 1e-1]))
        kept, info = select_kept(sig, chi, cutoff)
        assert kept == _brute_select(sig, chi, cutoff)
        assert sum(kept.values()) <= chi
        tot = sum(float(np.sum(v ** 2)) for v in sig.values())
        disc = sum(float(np.sum(sig[c][kept[c]:] ** 2)) for c in sig)
        assert abs(info["trunc_err"] - disc / tot) < 1e-15


def test_ties_at_the_cut_go_to_the_lower_charge():
    sig = {3: np.array([1.0, 0.5]), 5: np.array([0.5 * (1 + 1e-15), 0.1]), 7: np.array([0.5])}
    kept, info = select_kept(sig, 2, 0.0)
    assert kept == {3: 2, 5: 0, 7: 0}
    kept, _ = select_kept(sig, 3, 0.0)
    assert kept == {3: 2, 5: 1, 7: 0}
    # a gap larger than the tie band is an ordinary order
    sig = {3: np.array([1.0, 0.5]), 5: np.array([0.5 + 1e-6])}
    kept, _ = select_kept(sig, 2, 0.0)
    assert kept == {3: 1, 5: 1}
    assert TIE_REL < 1e-9


def test_cutoff_is_strict_and_relative_to_the_norm():
    sig = {0: np.array([3.0, 4.0 * 1e-3])}
    norm = math.sqrt(9 + 16e-6)
    kept, _ = select_kept(sig, 10, 4e-3 / norm)          # equal to threshold: dropped
    assert kept == {0: 1}
    kept, _ = select_kept(sig, 10, 4e-3 / norm * 0.999)  # just above: kept
    assert kept == {0: 2}


def test_zero_spectrum_is_an_error():
    with pytest.raises(FloatingPointError):
        select_kept({0: np.zeros(3)}, 4, 0.0)
