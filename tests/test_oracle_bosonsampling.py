"""Pins the oracle's beam-splitter gates and updates against brute-force permanents."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, dense, gates, permanent, tebd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _patterns(M, n, d):
    for t in itertools.product(range(d), repeat=M):
        if sum(t) == n:
            yield t


def _perm_prob(U, t, s):
    rows = [j for j in range(len(t)) for _ in range(t[j])]
    cols = [i for i in range(len(s)) for _ in range(s[i])]
    p = abs(permanent.permanent_bruteforce(U[np.ix_(rows, cols)])) ** 2
    return p / (np.prod([math.factorial(x) for x in t]) * np.prod([math.factorial(x) for x in s]))


def test_permanent_small_cases():
    a = np.array([[1.0, 2.0], [3.0, 4.0]])
    assert permanent.permanent_bruteforce(a) == 10.0
    rng = np.random.default_rng(3)
    m = W.random_complex((5, 5), rng)
    assert abs(permanent.permanent_ryser(m) - permanent.permanent_bruteforce(m)) < 1e-10
    # permanent of the all-ones n x n matrix is n!
    assert abs(permanent.permanent_ryser(np.ones((6, 6))) - 720) < 1e-9


def test_hom_dip_golden():
    g = json.load(open(os.path.join(GOLDEN, "hom_50_50.json")))
    st = U1MPS.product(3, g["input"])
    st.apply_gate2(0, gates.beam_splitter_gate(g["theta"], g["phi"], 3), 16, 0.0)
    for key, p in g["probabilities"].items():
        cfg = [int(x) for x in key.split(",")]
        assert abs(abs(st.amplitude(cfg)) ** 2 - p) < 1e-15


def test_single_photon_amplitudes_are_U_entries():
    M = 6
    layers = W.brickwork_pairs(M, 5)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=11)
    U = tebd.interferometer(M, layers, ang)
    for i in range(M):
        occ = [1 if k == i else 0 for k in range(M)]
        st = U1MPS.product(2, occ)
        tebd.run_brickwork(st, layers, ang, 64, 0.0)
        for j in range(M):
            e = [1 if k == j else 0 for k in range(M)]
            assert abs(st.amplitude(e) - U[j, i]) < 1e-14


def test_three_photons_all_patterns():
    M, n = 6, 3
    d = n + 1
    occ = W.single_photon_occupations(M, n)
    layers = W.brickwork_pairs(M, 6)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=0)
    st = U1MPS.product(d, occ)
    tebd.run_brickwork(st, layers, ang, 10_000, 0.0)
    U = tebd.interferometer(M, layers, ang)
    tot = 0.0
    for t in _patterns(M, n, d):
        p = abs(st.amplitude(list(t))) ** 2
        assert abs(p - _perm_prob(U, t, occ)) < 1e-14
        tot += p
    assert abs(tot - 1.0) < 1e-13


@pytest.mark.slow
def test_six_photons_sampled_patterns():
    M, n = 12, 6
    d = n + 1
    occ = W.single_photon_occupations(M, n)
    layers = W.brickwork_pairs(M, M)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=5)
    st = U1MPS.product(d, occ)
    tebd.run_brickwork(st, layers, ang, 100_000, 0.0)
    U = tebd.interferometer(M, layers, ang)
    rng = np.random.default_rng(0)
    for _ in range(60):
        t = W.random_occupations(M, d, n, rng)
        assert abs(abs(st.amplitude(t)) ** 2 - _perm_prob(U, t, occ)) < 1e-13
    assert abs(st.norm2() - 1.0) < 1e-12


def test_beam_splitter_blocks_match_fock_exponential():
    """For n <= d-1 the block is complete and equals the truncated-space exponential."""
    d = 4
    th, ph = 0.61, 2.2
    G = gates.beam_splitter_gate(th, ph, d)
    D = dense.beam_splitter_two_site(th, ph, d)
    for n in range(d):
        basis = list(range(max(0, n - d + 1), min(d - 1, n) + 1))
        idx = [i * d + (n - i) for i in basis]
        assert np.max(np.abs(D[np.ix_(idx, idx)] - G[n])) < 1e-14
        assert np.max(np.abs(G[n] @ G[n].conj().T - np.eye(len(basis)))) < 1e-14
