"""DMRG and TDVP at the size bench.py times (Bose-Hubbard L=64, N=64, chi<=256), checked through
properties that hold at any size (the oracle cannot sweep this chain in seconds):

- the energy at the end of each sweep does not rise (beyond the truncated weight's bound) and
  lands below the energy of the first sweep;
- every bond keeps at most chi states and unit-norm lambda;
- sampled sites are right-canonical (sum_r B B^dag = 1 per left sector) and satisfy the Vidal
  condition (diag(lambda_s) B has orthogonal columns of norm lambda_{s+1});
- one TDVP step of the U = 2 -> 4 quench keeps <H_eff> constant to 1e-6 relative (the
  projected evolution conserves the energy up to truncation) and the norm at 1.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

L, D, CHI, CUTOFF = 64, 5, 256, 1e-10


def _check_canonical(g, sites):
    for s in sites:
        blocks = g.site(s)
        lam_l, lam_r = g.bond(s), g.bond(s + 1)
        acc = {}
        for (l, m), b in blocks.items():
            acc[l] = acc.get(l, 0) + b @ b.conj().T
        for l, a in acc.items():
            assert np.max(np.abs(a - np.eye(a.shape[0]))) <= 1e-10, (s, l)
        cols = {}
        for (l, m), b in blocks.items():
            cols.setdefault(m, []).append(lam_l[l][:, None] * b)
        for m, parts in cols.items():
            M = np.vstack(parts)
            G = M.conj().T @ M
            assert np.max(np.abs(G - np.diag(lam_r[m] ** 2))) <= 1e-10, (s, m)


def test_dmrg_and_tdvp_at_the_benchmark_size(gpu_lib):
    m = gpu_lib
    terms = m.models.chain_bond_terms("bh", L, D, J=1.0, U=2.0)
    g = m.MPS(D, W.mott_occupations(L), CHI)
    ends = []
    for _ in range(3):
        e = g.dmrg(terms, 1, CHI, CUTOFF)
        ends.append(e[-1])
    assert ends[-1] <= ends[0] + 1e-9 * abs(ends[0])
    for k in range(1, len(ends)):
        assert ends[k] <= ends[k - 1] + 1e-6 * abs(ends[k - 1]), ends
    for b in range(L + 1):
        lam = g.bond(b)
        assert sum(len(v) for v in lam.values()) <= CHI
        assert abs(sum(float(v @ v) for v in lam.values()) - 1.0) <= 1e-12
    assert max(sum(len(v) for v in g.bond(b).values()) for b in range(L + 1)) == CHI
    _check_canonical(g, [0, 31, 32, 63])
    quench = m.models.chain_bond_terms("bh", L, D, J=1.0, U=4.0)
    E = g.tdvp(quench, 1, 0.02, CHI, CUTOFF)
    assert np.max(np.abs(E - E[0])) <= 1e-6 * abs(E[0])
    for b in (1, 32, 63):
        lam = g.bond(b)
        assert abs(sum(float(v @ v) for v in lam.values()) - 1.0) <= 1e-12
    _check_canonical(g, [16, 47])
    g.close()
