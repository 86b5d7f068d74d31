"""Sequential pattern sampling on the GPU (mps_sample) against the oracle and the permanent.

Boson sampling in M = 10 modes with 5 photons, no Fock truncation (d = 6) and no bond
truncation, so the state is exactly canonical and a pattern's probability is
|Perm(U_{t,s})|^2 / prod t! (Sec. I names boson-sampling circuits as a U(1) example;
Sec. II gives the amplitude formula whose one-block-per-site structure the sampler walks).
With the same uniform numbers the GPU draws the oracle's patterns (integers, exact), with
the same probabilities to 1e-12 relative; 40000 GPU draws pass a chi-square test against
the permanents.
"""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import U1MPS, gates, permanent, tebd
from oracle.sampling import sample_patterns

pytestmark = pytest.mark.gpu

M, N_PH = 10, 5
D = N_PH + 1


def _both(m):
    occ = W.single_photon_occupations(M, N_PH)
    layers = W.brickwork_pairs(M, M)
    ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=21)
    g = m.MPS(D, occ, 4096)
    st = U1MPS.product(D, occ)
    k = 0
    for sites in layers:
        gs = []
        for s in sites:
            gs.append(gates.beam_splitter_gate(*ang[k], D))
            k += 1
        g.apply_layer(sites, gs, 4096, 0.0)
        for s, G in zip(sites, gs):
            st.apply_gate2(s, G, 4096, 0.0)
    return g, st, tebd.interferometer(M, layers, ang), occ


def test_gpu_draws_the_oracles_patterns(gpu_lib):
    g, st, _, _ = _both(gpu_lib)
    u = W.uniforms(3000, M, seed=4)
    pg, prg = g.sample(u)
    po, pro = sample_patterns(st, u)
    assert np.array_equal(pg, po)
    assert np.max(np.abs(prg - pro) / pro) < 1e-12
    assert np.all(pg.sum(axis=1) == N_PH)


def test_gpu_draws_follow_the_permanents(gpu_lib):
    g, _, U, occ = _both(gpu_lib)
    pats = [t for t in itertools.product(range(D), repeat=M) if sum(t) == N_PH]
    index = {t: k for k, t in enumerate(pats)}
    exact = np.zeros(len(pats))
    cols = [i for i in range(M) for _ in range(occ[i])]
    for k, t in enumerate(pats):
        rows = [j for j in range(M) for _ in range(t[j])]
        exact[k] = abs(permanent.permanent_ryser(U[np.ix_(rows, cols)])) ** 2 / np.prod(
            [math.factorial(x) for x in t])
    assert abs(exact.sum() - 1.0) < 1e-12
    n = 40000
    draws, probs = g.sample(W.uniforms(n, M, seed=5))
    counts = np.zeros(len(pats))
    for row, p in zip(draws, probs):
        kk = index[tuple(int(x) for x in row)]
        counts[kk] += 1
        assert abs(p - exact[kk]) <= 1e-12 * max(exact[kk], 1e-3)
    ok = exact * n >= 5
    chi2 = float(np.sum((counts[ok] - exact[ok] * n) ** 2 / (exact[ok] * n)))
    dof = int(ok.sum()) - 1
    print(f"chi-square {chi2:.1f} on {dof} degrees of freedom")
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


def test_sampling_edge_cases(gpu_lib):
    m = gpu_lib
    g = m.MPS(3, [1, 1], 8)
    g.apply_gate2(0, gates.beam_splitter_gate(math.pi / 4, 0.0, 3), 8, 0.0)
    pats, probs = g.sample(np.array([[0.49, 0.0], [0.51, 0.9], [0.0, 0.0]]))
    assert pats.tolist() == [[0, 2], [2, 0], [0, 2]]       # the HOM pair (1, 1) has weight 0
    assert np.allclose(probs, 0.5, atol=1e-14)
    empty, _ = g.sample(np.zeros((0, 2)))
    assert empty.shape == (0, 2)
    with pytest.raises(m.MPSError):
        g.sample(np.array([[1.0, 0.5]]))                  # a uniform outside [0, 1)
