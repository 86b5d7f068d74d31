"""Kernel-level GPU tests: the batched Jacobi SVD (through mps_svd_sectors) against LAPACK."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _check(M, sig, Y, sweeps, tol=1e-12):
    ref = np.linalg.svd(M, compute_uv=False)
    k = min(M.shape)
    assert sig.shape == (k,)
    smax = max(ref[0], 1e-300)
    assert np.all(np.diff(sig) <= 0)
    assert np.max(np.abs(sig - ref[:k])) <= tol * smax * max(1.0, np.sqrt(max(M.shape)) / 4)
    assert sweeps >= 0
    good = sig > 1e-8 * smax
    Yg = Y[:, good]
    assert np.max(np.abs(Yg.conj().T @ Yg - np.eye(Yg.shape[1]))) < 1e-10
    # M y_j has norm sigma_j and the y_j span the row space of M for the kept part
    assert np.max(np.abs(np.linalg.norm(M @ Yg, axis=0) - sig[good])) <= 1e-12 * smax * np.sqrt(M.shape[1])


# one-CTA shared-memory sectors (wide and tall), cluster sectors (wide, tall with V, and
# more than 512 rows, the register-cache limit)
SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (5, 5), (30, 20), (20, 30), (64, 64), (100, 110),
          (150, 170), (200, 90), (33, 257), (600, 300), (300, 600), (420, 410), (130, 600), (64, 1100)]


def test_svd_random_shapes(gpu_lib):
    rng = np.random.default_rng(0)
    mats = [W.random_complex(s, rng) for s in SHAPES]
    for M, (sig, Y, sw) in zip(mats, gpu_lib.svd_sectors(mats)):
        _check(M, sig, Y, sw)


def test_svd_rowscale_graded_and_rank_deficient(gpu_lib):
    rng = np.random.default_rng(1)
    mats, scales = [], []
    # graded rows spanning 12 decades (the lambda weighting of a Schmidt spectrum)
    A = W.random_complex((60, 50), rng)
    mats.append(A)
    scales.append(np.logspace(0, -12, 60))
    # wide cluster sector (Jacobi on the K x K factor of R^dag) with graded rows
    mats.append(W.random_complex((110, 320), rng))
    scales.append(np.logspace(0, -10, 110))
    # exact rank 3
    B = W.random_complex((40, 3), rng) @ W.random_complex((3, 45), rng)
    mats.append(B)
    scales.append(np.ones(40))
    # zero matrix block with a single nonzero row
    C = np.zeros((8, 9), complex)
    C[3] = W.random_complex(9, rng)
    mats.append(C)
    scales.append(np.ones(8))
    out = gpu_lib.svd_sectors(mats, rowscales=scales)
    for M, r, (sig, Y, sw) in zip(mats, scales, out):
        Ms = r[:, None] * M
        ref = np.linalg.svd(Ms, compute_uv=False)
        k = min(Ms.shape)
        assert np.max(np.abs(sig - ref[:k])) <= 1e-13 * ref[0]
    # rank 3: everything past the third value is at rounding level
    assert np.all(out[2][0][3:] < 1e-13 * out[2][0][0])
    # graded wide sector: right singular vectors orthonormal and M y_j = sigma_j to relative accuracy
    Ms = scales[1][:, None] * mats[1]
    sig, Y, _ = out[1]
    good = sig > 1e-6 * sig[0]      # where numpy's own product M y is accurate to 1e-10 relative
    Yg = Y[:, good]
    assert np.max(np.abs(Yg.conj().T @ Yg - np.eye(Yg.shape[1]))) < 1e-10
    assert np.max(np.abs(np.linalg.norm(Ms @ Yg, axis=0) / sig[good] - 1.0)) < 1e-8


def test_svd_many_sectors_one_launch(gpu_lib):
    rng = np.random.default_rng(2)
    shapes = [(int(rng.integers(1, 90)), int(rng.integers(1, 90))) for _ in range(200)]
    mats = [W.random_complex(s, rng) for s in shapes]
    for M, (sig, Y, sw) in zip(mats, gpu_lib.svd_sectors(mats)):
        _check(M, sig, Y, sw)


# ---------------------------------------------------------------------------
# tensor-core (tcgen05) complex GEMM, TF32 and BF16x3
# ---------------------------------------------------------------------------
TC_SHAPES = [(1, 1, 1), (8, 16, 4), (100, 70, 90), (129, 65, 33), (128, 64, 32), (300, 200, 150), (37, 300, 257)]


@pytest.mark.parametrize("M,N,K", TC_SHAPES)
def test_zgemm_tc_tf32(gpu_lib, M, N, K):
    """TF32 keeps 10 mantissa bits (unit roundoff 2^-11); with FP32 accumulation the error of
    each output is bounded by about sqrt(K) * 2^-11 * sum |a||b|; checked against that."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = W.random_complex((M, K), rng)
    B = W.random_complex((K, N), rng)
    C = gpu_lib.zgemm_tc(A, B)
    ref = A @ B
    bound = (np.abs(A) @ np.abs(B)) * (4 * 2.0 ** -11) * np.sqrt(K) + 1e-12
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    # and it is really a product, not noise: relative error well below 1
    assert np.linalg.norm(C - ref) <= 5e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("M,N,K", TC_SHAPES)
def test_zgemm_tc_bf16x3(gpu_lib, M, N, K):
    """BF16x3: x = hi + lo represents x to about 2^-17 relative; the dropped lo.lo term and
    the split errors leave each product within about 3 * 2^-18 |a||b|, and FP32 accumulation
    adds at most K * 2^-24 sum |a||b|.  The bound 2^-15 + K 2^-24 is 16x below the error of a
    dropped cross term (2^-9), so a missing hi.lo or lo.hi product fails it."""
    rng = np.random.default_rng(M * 5 + N * 11 + K)
    A = W.random_complex((M, K), rng)
    B = W.random_complex((K, N), rng)
    C = gpu_lib.zgemm_tc(A, B, precision=gpu_lib.MPS_BF16X3)
    ref = A @ B
    bound = (np.abs(A) @ np.abs(B)) * (2.0 ** -15 + 2 * K * 2.0 ** -24) + 1e-14
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert np.linalg.norm(C - ref) <= 1e-4 * np.linalg.norm(ref)


def test_zgemm_tc_rejects_bad_arguments(gpu_lib):
    A = np.ones((4, 4), np.complex128)
    with pytest.raises(gpu_lib.MPSError):
        gpu_lib.zgemm_tc(A, A, precision=gpu_lib.MPS_FP64)


def test_cluster_kernels_on_sectors_that_fit_one_cta(gpu_lib):
    """mps_svd_cluster_min_k puts small and medium sectors on the cluster kernels (how mps_dmrg
    spreads a step's few sectors over the GPU): same accuracy as the one-CTA kernel, graded rows
    included."""
    rng = np.random.default_rng(5)
    shapes = [(16, 16), (17, 40), (48, 48), (64, 31), (85, 85), (90, 120), (130, 70)]
    mats = [W.random_complex(s, rng) for s in shapes]
    scales = [np.logspace(0, -10, s[0]) for s in shapes]
    try:
        gpu_lib.svd_cluster_min_k(16)
        out = gpu_lib.svd_sectors(mats, rowscales=scales)
    finally:
        gpu_lib.svd_cluster_min_k(0)
    for M, r, (sig, Y, sw) in zip(mats, scales, out):
        Ms = r[:, None] * M
        ref = np.linalg.svd(Ms, compute_uv=False)
        assert np.max(np.abs(sig - ref[:len(sig)])) <= 1e-12 * ref[0] * 4
        assert sw >= 0
        good = sig > 1e-8 * ref[0]
        Yg = Y[:, good]
        assert np.max(np.abs(Yg.conj().T @ Yg - np.eye(Yg.shape[1]))) < 1e-10
        assert np.max(np.abs(np.linalg.norm(Ms @ Yg, axis=0) - sig[good])) <= 1e-12 * ref[0] * np.sqrt(M.shape[1])
