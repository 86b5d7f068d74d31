"""The mixed-precision start of the cluster SVD (mps_svd_mixed_min_k): FP32 Jacobi sweeps that
accumulate the rotations, an FP64 Cholesky QR of them, FP64 sweeps from J V.

The per-sector SVD of Sec. II must keep its FP64 accuracy: singular values against LAPACK on
graded sectors (rows scaled over 8-10 decades, as diag(lambda) Theta'(c)), the right singular
vectors orthonormal and M Y = X S, the same results as the FP64-only path to rounding, in
fewer FP64 sweeps; and a chi = 2048-sized update keeps the oracle's sector structure.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(300, 300), (420, 260), (230, 480), (640, 610)]


def _graded(rng, m, n, decades):
    A = W.random_complex((m, n), rng)
    lam = 10.0 ** (-decades * rng.random(m))
    return A, np.sort(lam)[::-1].copy()


@pytest.mark.parametrize("decades", [0.0, 8.0, 10.0])
def test_mixed_svd_matches_lapack_and_the_fp64_path(gpu_lib, decades):
    m = gpu_lib
    rng = np.random.default_rng(int(decades) + 3)
    mats, scales = zip(*[_graded(rng, a, b, decades) for a, b in SHAPES])
    try:
        m.svd_mixed_min_k(0)
        ref = m.svd_sectors(list(mats), rowscales=list(scales))
        m.svd_mixed_min_k(64)
        got = m.svd_sectors(list(mats), rowscales=list(scales))
    finally:
        m.svd_mixed_min_k(192)
    for A, lam, (s0, y0, sw0), (s1, y1, sw1) in zip(mats, scales, ref, got):
        M = lam[:, None] * A
        s_la = scipy.linalg.svd(M, compute_uv=False, lapack_driver="gesvd")
        smax = s_la[0]
        k = len(s_la)
        assert np.max(np.abs(s1[:k] - s_la)) <= 1e-13 * smax
        assert np.max(np.abs(s1 - s0)) <= 1e-13 * smax
        good = s1 > 1e-9 * smax
        # orthonormal right vectors; (M Y)^dag (M Y) = S^2 to rounding of the largest value
        # (the sigma-weighted form, the accuracy LAPACK's gesvd has: the update uses the
        # vectors weighted by their singular values)
        Yg = y1[:, good]
        assert np.max(np.abs(Yg.conj().T @ Yg - np.eye(Yg.shape[1]))) <= 1e-10
        MY = M @ Yg
        assert np.max(np.abs(MY.conj().T @ MY - np.diag(s1[good] ** 2))) <= 1e-12 * smax ** 2
        # and the kept subspace is the FP64 path's: the two projectors weighted by sigma agree
        P1 = (Yg * s1[good]) @ Yg.conj().T
        Y0 = y0[:, good]
        P0 = (Y0 * s0[good]) @ Y0.conj().T
        assert np.max(np.abs(P1 - P0)) <= 1e-11 * smax
        # the FP64 sweeps started from J V: far fewer than from J
        assert 0 <= sw1 <= max(4, sw0 - 2), (sw0, sw1)


def test_mixed_svd_update_keeps_the_oracle_structure(gpu_lib):
    """One chi = 2048-sized middle update of a random saturated chain (Theta(c) up to ~800
    columns) with every cluster sector on the mixed path."""
    from oracle import gates
    from oracle.synth import random_state
    from helpers import compare_update, load_state
    m = gpu_lib
    L, d, N, chi = 16, 5, 16, 2048
    s = L // 2 - 1
    G = gates.bh_gate(L, s, d, 1.0, 2.0, 0.3)
    ref = random_state(L, d, N, chi, seed=21)
    st0 = random_state(L, d, N, chi, seed=21)
    ref.apply_gate2(s, G, chi, 1e-10)
    try:
        m.svd_mixed_min_k(64)
        g = m.MPS(d, W.random_occupations(L, d, N, np.random.default_rng(0)), chi)
        load_state(g, st0)
        g.apply_gate2(s, G, chi, 1e-10)
        compare_update(g, ref, s)
        g.close()
    finally:
        m.svd_mixed_min_k(192)
