"""The FP64 -> FP32 operand rounding of the tensor-core GEMM, seen through mps_zgemm_tc.

The reduced-precision modes round the FP64 operands to FP32 (round to nearest, ties to
even, on the IEEE-754 binary64 / binary32 layouts; magnitudes below 2^-126 become a signed
zero, magnitudes beyond the FP32 range infinity, NaN stays NaN) and then to TF32 (round
to nearest, ties away from zero) or to a BF16 pair hi + lo (each round to nearest even).
A product with a unit partner is exact in FP32, so C = A . 1 exposes the operand exactly
as the tensor core saw it.  The expected values below are computed from the bit layouts
with integer numpy operations; an FP32 tie that the first rounding resolves upwards moves
a TF32 tie, which is what makes the first rounding's tie rule visible through the second.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F32_MIN_NORMAL = 2.0 ** -126


def _f32_rn_flush(x: np.ndarray) -> np.ndarray:
    """FP64 -> FP32 by IEEE round to nearest even, then magnitudes below 2^-126 (FP32
    subnormals) as signed zeros.  The flush applies to the FP64 input: a value just
    under 2^-126 is zero even where round-to-nearest would reach 2^-126."""
    with np.errstate(over="ignore"):
        f = x.astype(np.float32)
    tiny = np.abs(x) < F32_MIN_NORMAL
    f[tiny] = np.copysign(np.float32(0.0), x[tiny]).astype(np.float32)
    return f


def _tf32_rna(f: np.ndarray) -> np.ndarray:
    """FP32 -> TF32 (10 fraction bits): round half away from zero on the magnitude bits."""
    u = f.view(np.uint32).copy()
    fin = np.isfinite(f)
    u[fin] = (u[fin] + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def _bf16_rne(f: np.ndarray) -> np.ndarray:
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _from_bits(sign, exp, frac52):
    b = (np.uint64(sign) << np.uint64(63)) | (np.uint64(exp) << np.uint64(52)) | np.uint64(frac52)
    return np.array([b], dtype=np.uint64).view(np.float64)[0]


def _tie_cases(rng):
    """Doubles whose FP32 rounding is a tie or one ulp either side of it, with the top 23
    fraction bits ending in 0x0FFF (odd: a tie rounds them to 0x1000, which is itself a
    TF32 tie), 0x0FFE (even) or all ones (the rounding carries into the exponent)."""
    out = []
    for _ in range(12):
        hi = int(rng.integers(0, 1 << 10))
        exp = int(rng.integers(1023 - 100, 1023 + 100))
        sign = int(rng.integers(0, 2))
        for low13 in (0x0FFF, 0x0FFE):
            fm = (hi << 13) | low13
            for rem in (0x10000000, 0x0FFFFFFF, 0x10000001):
                out.append(_from_bits(sign, exp, (fm << 29) | rem))
        out.append(_from_bits(sign, exp, (0x7FFFFF << 29) | 0x10000000))
    return out


def _specials():
    return [F32_MIN_NORMAL, -F32_MIN_NORMAL, 1.5 * F32_MIN_NORMAL, F32_MIN_NORMAL * (1 - 2.0 ** -30),
            1e-39, -1e-39, 1e-45, -3e-44, 1e-300, 0.0, -0.0,
            3.0e38, -3.0e38, 3.5e38, -3.5e38, 1e39, 1e300, -1e300, np.nan]


def _column(rng, values, n_rows=256):
    """Values padded with random normals of many magnitudes to n_rows (two 128-row tiles)."""
    v = list(values)
    while len(v) < n_rows:
        v.append(float(rng.standard_normal() * 10.0 ** rng.integers(-30, 30)))
    return np.array(v[:n_rows], dtype=np.float64)


def test_tf32_operand_rounding(gpu_lib):
    m = gpu_lib
    rng = np.random.default_rng(17)
    x = _column(rng, _tie_cases(rng) + _specials())
    A = x.astype(np.complex128).reshape(-1, 1)
    C = m.zgemm_tc(A, np.ones((1, 1), np.complex128), precision=m.MPS_TF32)
    got = C[:, 0].real
    want = _tf32_rna(_f32_rn_flush(x)).astype(np.float64)
    # an operand the conversion makes infinite or NaN gives a non-finite product (how the
    # tensor core combines inf and NaN with the zero terms of the lowered GEMM is its own
    # business); every finite operand must come out exactly as modelled
    fin = np.isfinite(want)
    assert np.all(~np.isfinite(got[~fin])), [(x[i], got[i]) for i in np.nonzero(~fin)[0]]
    bad = np.nonzero(got[fin] != want[fin])[0]
    assert bad.size == 0, [(x[fin][i], got[fin][i], want[fin][i]) for i in bad[:8]]
    # the overflow cases (+-3.5e38, 1e39, +-1e300) and the NaN are among the non-finite ones
    assert np.count_nonzero(~fin) >= 6
    # the tie cases do decide: truncating instead of rounding would change some results
    trunc = (x.view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)).view(np.float64)
    alt = _tf32_rna(_f32_rn_flush(trunc)).astype(np.float64)
    assert np.any((alt != want) & fin)


def test_bf16x3_operand_rounding(gpu_lib):
    m = gpu_lib
    rng = np.random.default_rng(18)
    # finite values only (hi x (a zero lo partner) would turn an infinite operand into NaN),
    # magnitudes that keep the lo term a normal BF16 number
    vals = [v for v in _tie_cases(rng) if 1e-20 < abs(v) < 1e20]
    vals += [F32_MIN_NORMAL * 2.0 ** 40, 1e-39, -1e-39, 1e-45]
    x = _column(rng, vals)
    x = np.where(np.abs(x) > 1e20, 1.0, x)
    x = np.where((np.abs(x) < 1e-20) & (np.abs(x) >= F32_MIN_NORMAL), 1e-20, x)
    A = x.astype(np.complex128).reshape(-1, 1)
    C = m.zgemm_tc(A, np.ones((1, 1), np.complex128), precision=m.MPS_BF16X3)
    f = _f32_rn_flush(x)
    hi = _bf16_rne(f)
    lo = _bf16_rne((f - hi).astype(np.float32))
    want = (hi.astype(np.float64) + lo.astype(np.float64))
    got = C[:, 0].real
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(x[i], got[i], want[i]) for i in bad[:8]]
