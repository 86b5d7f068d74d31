"""The package's model set-up (paper_2303_11409_gb300/models.py, tebd.py) against the oracle's
independent constructions, on the CPU.

The library takes gate and bond-term blocks as inputs; the package builds them once per workload
(closed forms, scipy's expm per block, the Fock-space beam splitter by its generator), the oracle
by eigh per block and brute-force permanents.  Both must give the same blocks in the layout of
the C ABI: U(1) block n over (i, n - i), i ascending; Z_n block q over (i, (q - i) mod n); for a
Z_n handle with d < n the U(1) blocks of totals q, q + n, ... joined in block q.
"""
import math

import numpy as np
import pytest

from oracle import dmrg, gates, tebd
from oracle.znmps import gate_blocks_from_u1, zn_charges


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    b = g._build_module()
    import os
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2303_11409_gb300 as m
    return m


def _close(a, b, tol=1e-13):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.asarray(x).shape == np.asarray(y).shape
        assert np.max(np.abs(np.asarray(x) - np.asarray(y))) <= tol


@pytest.mark.parametrize("delta,tau", [(0.5, 0.05), (1.3, -0.2)])
def test_xxz_gate_blocks(pkg, delta, tau):
    _close(pkg.models.xxz_gate(delta, tau), gates.xxz_gate(delta, tau))


@pytest.mark.parametrize("d", [2, 3, 5])
def test_bose_hubbard_gate_blocks(pkg, d):
    L, J, U, tau = 9, 1.0, 2.0, 0.035
    for s in (0, 4, L - 2):
        wl, wr = pkg.models.bose_hubbard_weights(L, s)
        assert (wl, wr) == gates.bh_weights(L, s)
        _close(pkg.models.bose_hubbard_gate(d, J, U, tau, wl, wr), gates.bh_gate(L, s, d, J, U, tau))


@pytest.mark.parametrize("d", [2, 3, 5])
def test_beam_splitter_gate_blocks(pkg, d):
    rng = np.random.default_rng(d)
    for _ in range(3):
        th, ph = float(rng.uniform(0, math.pi / 2)), float(rng.uniform(0, 2 * math.pi))
        _close(pkg.models.beam_splitter_gate(th, ph, d), gates.beam_splitter_gate(th, ph, d), tol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_clock_gate_blocks(pkg, n):
    L, J, f, tau = 7, 1.0, 0.6, 0.1
    for s in (0, 3, L - 2):
        wl, wr = gates.bh_weights(L, s)
        _close(pkg.models.clock_gate(n, J, f, tau, wl, wr), gates.clock_gate(L, s, n, J, f, tau))


@pytest.mark.parametrize("d,n", [(2, 3), (3, 4), (3, 5), (5, 6), (2, 2), (3, 3)])
def test_cyclic_blocks_of_a_u1_gate(pkg, d, n):
    """The Z_n layout of a U(1) gate (d <= n): same residues, same pairs, same entries."""
    L, s, tau = 8, 3, 0.07
    u1 = gates.bh_gate(L, s, d, 1.0, 2.0, tau)
    mine = pkg.models.cyclic_blocks(pkg.models.bose_hubbard_gate(d, 1.0, 2.0, tau, *gates.bh_weights(L, s)), d, n)
    ref = gate_blocks_from_u1(u1, n, d)
    assert list(pkg._binding.cyclic_pair_blocks(n, d)) == zn_charges(n, d)
    _close(mine, [ref[q] for q in zn_charges(n, d)])
    table = pkg.tebd.GateTable("bh", L, d, tau, J=1.0, U=2.0, zn=n)
    flat = table(s, 1.0)
    assert flat.size == sum(len(p) ** 2 for p in pkg._binding.cyclic_pair_blocks(n, d).values())
    assert np.max(np.abs(flat - np.concatenate([ref[q].reshape(-1) for q in zn_charges(n, d)]))) <= 1e-13


def test_bond_terms(pkg):
    L = 7
    for mine, ref in zip(pkg.models.chain_bond_terms("xxz", L, 2, delta=0.7), dmrg.xxz_bonds(L, 0.7)):
        _close(mine, ref, tol=1e-15)
    for mine, ref in zip(pkg.models.chain_bond_terms("bh", L, 4, J=1.0, U=3.0), dmrg.bh_bonds(L, 4, 1.0, 3.0)):
        _close(mine, ref, tol=1e-15)


def test_strang_schedule(pkg):
    for L in (2, 7, 8):
        assert pkg.tebd.strang_layers(L) == tebd.strang_layers(L)


def test_gate_lengths(pkg):
    """The flattened length the binding checks every gate against, per charge rule."""
    for d in (2, 3, 5, 8):
        assert pkg.gate_length(d) == sum(len(b) ** 2 for b in gates.bh_gate(6, 2, d, 1.0, 1.0, 0.1))
    q = [(0, 0), (0, 1), (1, 0), (1, 1)]
    pairs = pkg._binding.multi_pair_blocks(q)
    total = {}
    for a in q:
        for b in q:
            t = (a[0] + b[0], a[1] + b[1])
            total[t] = total.get(t, 0) + 1
    assert sum(len(p) ** 2 for p in pairs.values()) == sum(k * k for k in total.values())
