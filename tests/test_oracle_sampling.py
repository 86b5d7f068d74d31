"""Pins of the oracle's sequential pattern sampling (boson sampling follow-on of the
U(1) amplitude formula, Sec. II; the paper's boson-sampling example, Sec. I).

On an exactly canonical, untruncated state the product of the sequential conditionals
along a pattern is its Born probability |<t|psi>|^2, which for boson sampling is the
brute-force permanent |Perm(U_{t,s})|^2 / (prod t! prod s!).  Drawn patterns then follow
that distribution (a chi-square test on a seeded draw), and the probability reported
with each draw is the one of the pattern it returns.
"""
import itertools
import math

import numpy as np

import workloads as W
from oracle import U1MPS, gates, permanent, tebd
from oracle.sampling import pattern_probability, sample_patterns


def _boson_state(M, n, depth, seed):
    d = n + 1
    occ = W.single_photon_occupations(M, n)
    layers = W.brickwork_pairs(M, depth)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=seed)
    st = U1MPS.product(d, occ)
    tebd.run_brickwork(st, layers, ang, 4096, 0.0)
    return st, tebd.interferometer(M, layers, ang), occ


def _perm_prob(U, t, s):
    rows = [j for j in range(len(t)) for _ in range(t[j])]
    cols = [i for i in range(len(s)) for _ in range(s[i])]
    p = abs(permanent.permanent_bruteforce(U[np.ix_(rows, cols)])) ** 2
    return p / (np.prod([math.factorial(x) for x in t]) * np.prod([math.factorial(x) for x in s]))


def _patterns(M, n):
    return [t for t in itertools.product(range(n + 1), repeat=M) if sum(t) == n]


def test_sequential_probability_is_the_permanent():
    M, n = 6, 3
    st, U, occ = _boson_state(M, n, 6, seed=5)
    tot = 0.0
    for t in _patterns(M, n):
        p = pattern_probability(st, t)
        assert abs(p - _perm_prob(U, t, occ)) < 1e-13, t
        tot += p
    assert abs(tot - 1.0) < 1e-12
    assert pattern_probability(st, [3, 0, 0, 0, 0, 1]) == 0.0      # wrong total charge


def test_draws_follow_the_born_distribution():
    M, n = 6, 3
    st, U, occ = _boson_state(M, n, 6, seed=5)
    pats = _patterns(M, n)
    exact = np.array([_perm_prob(U, t, occ) for t in pats])
    draws, probs = sample_patterns(st, W.uniforms(20000, M, seed=9))
    index = {t: k for k, t in enumerate(pats)}
    counts = np.zeros(len(pats))
    for row, p in zip(draws, probs):
        t = tuple(int(x) for x in row)
        counts[index[t]] += 1
        assert abs(p - exact[index[t]]) < 1e-13
    # chi-square over the patterns with an expected count of at least 5; for this fixed
    # seed the statistic must stay under dof + 6 sqrt(2 dof) (far in the tail for a correct
    # sampler, exceeded at once by a sampler that skews the conditionals)
    ok = exact * len(draws) >= 5
    chi2 = float(np.sum((counts[ok] - exact[ok] * len(draws)) ** 2 / (exact[ok] * len(draws))))
    dof = int(ok.sum()) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
    assert np.all(counts[exact < 1e-14] == 0)


def test_hom_pair_is_never_drawn():
    st = U1MPS.product(3, [1, 1])
    st.apply_gate2(0, gates.beam_splitter_gate(math.pi / 4, 0.0, 3), 16, 0.0)
    draws, probs = sample_patterns(st, W.uniforms(4000, 2, seed=1))
    rows = {tuple(int(x) for x in r) for r in draws}
    assert rows <= {(2, 0), (0, 2)}
    assert np.allclose(probs, 0.5, atol=1e-14)
    # inverse CDF: u below 1/2 takes the lower occupation of the first site
    d2, _ = sample_patterns(st, np.array([[0.49, 0.0], [0.51, 0.0]]))
    assert d2.tolist() == [[0, 2], [2, 0]]
