"""The seeded input generators (no GPU): the recipes the workloads are built from."""
import numpy as np

import workloads as W
from oracle.synth import saturated_dims


def test_saturated_sector_dims_match_the_oracle_recipe():
    # the CUDA benchmark and the oracle's CPU sample build their saturated chains from
    # separate implementations of the same recipe; they must give the same sector sizes
    for L, d, N, chi in [(16, 5, 16, 2048), (24, 3, 24, 300), (12, 2, 6, 40), (64, 5, 64, 512)]:
        for b in range(1, L):
            assert W.saturated_sector_dims(L, d, N, b, chi) == saturated_dims(L, d, N, b, chi), (L, b)


def test_saturated_random_state_structure():
    L, d, N, chi = 10, 3, 10, 60
    lam, blocks = W.saturated_random_state(L, d, N, chi, seed=3)
    for b in range(1, L):
        w = np.concatenate([lam[b][c] for c in sorted(lam[b])])
        assert abs(np.linalg.norm(w) - 1.0) < 1e-12
        for c, v in lam[b].items():
            assert np.all(np.diff(v) <= 0) and np.all(v > 0)
    for s in range(L):
        for (l, m), B in blocks[s].items():
            assert 0 <= l - m <= d - 1
            left = {N: 1} if s == 0 else {c: len(v) for c, v in lam[s].items()}
            right = {0: 1} if s == L - 1 else {c: len(v) for c, v in lam[s + 1].items()}
            assert B.shape == (left[l], right[m])


def test_haar_unitaries_and_u1_gate_blocks():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5):
        U = W.haar_unitary(n, rng)
        assert np.allclose(U.conj().T @ U, np.eye(n), atol=1e-13)
    # the phase recipe makes the distribution Haar: E|U_00|^2 = 1/n
    samples = [abs(W.haar_unitary(3, rng)[0, 0]) ** 2 for _ in range(4000)]
    assert abs(np.mean(samples) - 1 / 3) < 0.02
    d = 5
    blocks = W.random_u1_gate(d, rng)
    assert [b.shape[0] for b in blocks] == [1, 2, 3, 4, 5, 4, 3, 2, 1]
    for b in blocks:
        assert np.allclose(b.conj().T @ b, np.eye(b.shape[0]), atol=1e-13)
