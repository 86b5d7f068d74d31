"""Z_n-symmetric chains on the GPU (mps_create_zn) against the Z_n oracle.

Sec. I of arXiv:2303.11409 names more general Abelian symmetries beside U(1); the block
construction of Sec. II carries over with charges mod n.  The clock chain (n = 2: the
transverse-field Ising chain in the basis where the field is diagonal) is evolved by the
same Strang schedule on both sides, with truncation active.  FP64 mode: identical bond
tables after every layer, Schmidt values within 1e-12, local <X + X^dag> within 1e-9 of
its scale, amplitudes within 1e-10.
"""
import numpy as np
import pytest

from oracle import gates as ogates
from oracle.znmps import ZnMPS

pytestmark = pytest.mark.gpu

CASES = [
    # n, L, initial charges, J, f, chi, steps
    (2, 12, [0] * 12, 1.0, 0.9, 16, 8),
    (3, 9, [0, 1, 2, 0, 1, 2, 0, 1, 2], 1.0, 0.6, 24, 5),
    (4, 7, [1, 0, 3, 2, 0, 1, 2], 0.8, 1.1, 30, 4),
]


@pytest.mark.parametrize("n,L,occ,J,f,chi,steps", CASES)
def test_zn_tebd_matches_the_oracle(gpu_lib, n, L, occ, J, f, chi, steps):
    m = gpu_lib
    dt, cutoff = 0.1, 1e-10
    gpu = m.MPS(n, occ, chi, zn=n)
    ref = ZnMPS.product(n, occ)
    table = m.tebd.GateTable("clock", L, n, dt, J=J, f=f)
    xs = 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
    cut_seen = False
    for _ in range(steps):
        for sites, frac in m.tebd.strang_layers(L):
            gpu.apply_layer(sites, [table(s, frac) for s in sites], chi, cutoff)
            for s in sites:
                ref.apply_gate2(s, ogates.clock_gate(L, s, n, J, f, frac * dt), chi, cutoff)
            for b in range(L + 1):
                got = gpu.bond(b)
                assert {c: len(v) for c, v in got.items()} == ref.bond[b], b
                for c, v in ref.lam[b].items():
                    assert np.max(np.abs(got[c] - v)) <= 1e-12, (b, c)
            cut_seen = cut_seen or max(sum(ref.bond[b].values()) for b in range(L + 1)) == chi
        for s in range(L):
            a, r = gpu.expect(s, xs), ref.expect_local(s, xs)
            assert abs(a - r) <= 1e-9 * 2.0, (s, a, r)
    assert cut_seen, "the chi cut never became active"
    rng = np.random.default_rng(1)
    cfgs = rng.integers(0, n, size=(40, L)).astype(np.int32)
    amps = gpu.amplitudes(cfgs)
    want = np.array([ref.amplitude(c) for c in cfgs])
    scale = max(1e-300, float(np.max(np.abs(want))))
    # amplitudes are gauge invariant (the SVD's phase freedom cancels between neighbouring sites)
    assert np.max(np.abs(amps - want)) <= 1e-10 * scale
    gpu.close()


@pytest.mark.parametrize("name,tol", [("tf32", 5e-3), ("bf16x3", 8e-5)])
def test_zn_tensor_core_gemms_against_the_fp64_oracle(gpu_lib, name, tol):
    """The Z_3 clock chain with the sector GEMMs on the tensor cores: <X + X^dag> within the
    stated accuracy of the reduced-precision modes (5e-3 TF32, 8e-5 BF16x3, of the observable's
    scale 2), unit-norm lambda and at most chi states on every bond."""
    m = gpu_lib
    n, L, occ, J, f, chi, steps = 3, 9, [0, 1, 2, 0, 1, 2, 0, 1, 2], 1.0, 0.6, 24, 5
    dt, cutoff = 0.1, 1e-10
    prec = {"tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[name]
    gpu = m.MPS(n, occ, chi, zn=n, precision=prec)
    ref = ZnMPS.product(n, occ)
    table = m.tebd.GateTable("clock", L, n, dt, J=J, f=f)
    for _ in range(steps):
        for sites, frac in m.tebd.strang_layers(L):
            gpu.apply_layer(sites, [table(s, frac) for s in sites], chi, cutoff)
            for s in sites:
                ref.apply_gate2(s, ogates.clock_gate(L, s, n, J, f, frac * dt), chi, cutoff)
    xs = 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
    dx = max(abs(gpu.expect(s, xs) - ref.expect_local(s, xs)) for s in range(L))
    print(f"Z_3 clock chain, {name}: <X + X^dag> {dx:.2e}")
    assert dx <= tol * 2.0, dx
    for b in range(L + 1):
        lam = gpu.bond(b)
        assert sum(len(v) for v in lam.values()) <= chi
        assert abs(sum(float(v @ v) for v in lam.values()) - 1.0) <= 1e-12
    gpu.close()


CYCLIC = [
    # d, n, L, initial occupations, chi, steps (Bose-Hubbard, n_max = d - 1, on a Z_n handle)
    (3, 4, 10, [2, 0, 1, 1, 0, 2, 1, 1, 0, 1], 12, 4),
    (3, 5, 8, [2, 0, 2, 1, 2, 0, 1, 1], 16, 3),
    (2, 3, 12, [1, 0, 1, 1, 0, 0, 1, 0, 1, 1, 0, 1], 10, 4),
]


@pytest.mark.parametrize("d,n,L,occ,chi,steps", CYCLIC)
def test_cyclic_handle_with_d_below_n_matches_the_oracle(gpu_lib, d, n, L, occ, chi, steps):
    """mps_create_cyclic (Z_n with d < n): a Bose-Hubbard chain, whose particle number is also
    conserved mod n, evolved in the Z_n blocks (Theta(c) rows listed, lambda gathered) on both
    sides; FP64: identical bond tables and lambda within 1e-12 after every layer, densities
    within 1e-9, amplitudes within 1e-10."""
    from oracle.znmps import gate_blocks_from_u1
    m = gpu_lib
    J, U, dt, cutoff = 1.0, 2.0, 0.1, 1e-10
    gpu = m.MPS(d, occ, chi, zn=n)
    ref = ZnMPS.product(n, occ, d=d)
    table = m.tebd.GateTable("bh", L, d, dt, J=J, U=U, zn=n)
    cut_seen = False
    for _ in range(steps):
        for sites, frac in m.tebd.strang_layers(L):
            gpu.apply_layer(sites, [table(s, frac) for s in sites], chi, cutoff)
            for s in sites:
                ref.apply_gate2(s, gate_blocks_from_u1(ogates.bh_gate(L, s, d, J, U, frac * dt), n, d), chi, cutoff)
            for b in range(L + 1):
                got = gpu.bond(b)
                assert {c: len(v) for c, v in got.items()} == ref.bond[b], b
                for c, v in ref.lam[b].items():
                    assert np.max(np.abs(got[c] - v)) <= 1e-12, (b, c)
            cut_seen = cut_seen or max(sum(ref.bond[b].values()) for b in range(L + 1)) == chi
    assert cut_seen, "the chi cut never became active"
    nop = np.arange(d, dtype=float)
    for s in range(L):
        a, r = gpu.expect(s, nop), ref.expect_local(s, nop)
        assert abs(a - r) <= 1e-9 * max(abs(r), d - 1), (s, a, r)
    rng = np.random.default_rng(2)
    cfgs = rng.integers(0, d, size=(40, L)).astype(np.int32)
    amps = gpu.amplitudes(cfgs)
    want = np.array([ref.amplitude(c) for c in cfgs])
    scale = max(1e-300, float(np.max(np.abs(want))))
    assert np.max(np.abs(amps - want)) <= 1e-10 * scale
    gpu.close()


def test_zn_handle_rejects_bad_arguments(gpu_lib):
    m = gpu_lib
    with pytest.raises(m.MPSError):
        m.MPS(3, [0, 1, 3], 8, zn=3)              # occupation outside [0, n-1]
    with pytest.raises(ValueError):
        m.MPS(3, [0, 1, 1], 8, zn=2)              # d must not exceed n
    h = m._binding._h()
    occ = np.array([0, 1, 1], dtype=np.int32)
    ptr = occ.ctypes.data_as(m._binding._i32p)
    assert m.lib.mps_create_cyclic(m._binding.ctypes.byref(h), 3, 3, 2, ptr, m.MPS_FP64, 8, None) == m.MPS_EINVAL
    assert m.lib.mps_create_cyclic(m._binding.ctypes.byref(h), 3, 2, 1 << 21, ptr, m.MPS_FP64, 8, None) == m.MPS_EINVAL
    g = m.MPS(2, [0, 1, 1, 0], 8, zn=2)
    assert g.bond_dims(0) == {0: 1}               # (0 + 1 + 1 + 0) mod 2
    assert g.bond_dims(1) == {0: 1} and g.bond_dims(2) == {1: 1} and g.bond_dims(3) == {0: 1}
    g.close()
