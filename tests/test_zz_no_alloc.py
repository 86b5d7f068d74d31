"""The allocation-free sector SVD entry point (mps_svd_sectors_noalloc).

Some callers cannot hand the library a scratch buffer or let it call cudaMalloc
(a framework that owns the whole device-memory budget, or a hot loop that cannot
afford the implicit synchronisation of cudaMalloc/cudaFree).  For them the batched
sector SVD has a variant whose scratch is a fixed device array inside the
library.  This file checks, through the C ABI, that it returns what the regular
entry point returns, on two calls in a row (the array keeps the previous call's
contents), and that a batch larger than the fixed array is refused up front.
It is collected last so that a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

# one-CTA shared-memory sectors and cluster sectors (the ones that use the scratch)
SHAPES = [(1, 1), (7, 3), (30, 20), (64, 64), (150, 170), (200, 90), (300, 300), (33, 257)]


def _batch(seed):
    rng = np.random.default_rng(seed)
    mats = [W.random_complex(s, rng) for s in SHAPES]
    scales = [np.sort(0.05 + rng.random(s[0]))[::-1] for s in SHAPES]
    return mats, scales


def test_noalloc_matches_regular_entry_point_twice(gpu_lib):
    m = gpu_lib
    for call, seed in enumerate((5, 6)):          # two calls in a row, different data
        mats, scales = _batch(seed)
        ref = m.svd_sectors(mats, rowscales=scales)
        got = m.svd_sectors_noalloc(mats, rowscales=scales)
        for M, (s_ref, y_ref, sw_ref), (s_got, y_got, sw_got) in zip(mats, ref, got):
            smax = max(s_ref[0], 1e-300)
            assert s_got.shape == s_ref.shape
            assert np.max(np.abs(s_got - s_ref)) <= 1e-12 * smax, call
            good = s_ref > 1e-8 * smax
            assert np.max(np.abs(y_got[:, good] - y_ref[:, good])) <= 1e-10, call
            assert sw_got >= 0


def test_noalloc_rejects_batches_beyond_its_scratch(gpu_lib):
    m = gpu_lib
    big = [(1200, 1200)]                            # needs about 23 MB of scratch
    assert m.svd_work_bytes([1200], [1200]) > m.MPS_NOALLOC_SCRATCH_BYTES
    rng = np.random.default_rng(0)
    with pytest.raises(m.MPSError) as e:
        m.svd_sectors_noalloc([W.random_complex(big[0], rng)])
    assert e.value.code == m.MPS_ENOMEM
