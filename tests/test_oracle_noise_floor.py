"""Pin of the oracle's noise floor: within one update, a sector's singular values at or
below 32 eps |M(c)|_F count as exact zeros (the reading that makes a zero cutoff keep
exactly the numerically nonzero spectrum; the paper states no floor).

The test plants a spectrum in one middle-charge sector of an update.  With every gate
block the identity, Theta'(c)[l, r] = B^[s][l, c] B^[s+1][c, r] (only m = c survives the
gate), so choosing B^[s][:, c] = diag(1 / lambda^[s]) Q and B^[s+1][c, :] = diag(sigma) Y^dag
with isometries Q, Y makes M(c) = diag(lambda^[s]) Theta'(c) = Q diag(sigma) Y^dag exactly
up to rounding.  The planted sigma are sixteen ones (|M|_F = 4) and two values just above
and just below 32 eps * 4.  The other sectors are scaled up so that a floor taken against
the whole update's norm, or against the sector's largest value instead of its Frobenius
norm, would keep a different number of values.
"""
import math

import numpy as np

import workloads as W
from oracle import U1MPS, gate_basis, plan_update, synth
from oracle.u1mps import NOISE_REL

L, D, N, CHI, S, C = 10, 3, 10, 120, 4, 5


def _planted_state():
    st = synth.random_state(L, D, N, CHI, seed=1)
    plan = plan_update(st.bond[S], st.bond[S + 1], st.bond[S + 2], D)
    rows, cols = plan.rows[C], plan.cols[C]
    k = st.bond[S + 1][C]
    rng = np.random.default_rng(2)
    m_rows = sum(st.bond[S][l] for l in rows)
    n_cols = sum(st.bond[S + 2][r] for r in cols)
    Q = np.linalg.qr(W.random_complex((m_rows, k), rng))[0]
    Y = np.linalg.qr(W.random_complex((n_cols, k), rng))[0]
    floor = NOISE_REL * 4.0
    sigma = np.zeros(k)
    sigma[:16] = 1.0
    sigma[16] = 1.3 * floor          # survives
    sigma[17] = 0.7 * floor          # rounding noise by the reading
    lam_rows = np.concatenate([st.lam[S][l] for l in rows])
    left = Q / lam_rows[:, None]
    ro = 0
    for l in rows:
        st.B[S][(l, C)] = left[ro:ro + st.bond[S][l]].copy()
        ro += st.bond[S][l]
    right = sigma[:, None] * Y.conj().T
    co = 0
    for r in cols:
        st.B[S + 1][(C, r)] = right[:, co:co + st.bond[S + 2][r]].copy()
        co += st.bond[S + 2][r]
    for (c, r), blk in st.B[S + 1].items():     # every other sector much larger
        if c != C:
            st.B[S + 1][(c, r)] = 100.0 * blk
    M = Q @ np.diag(sigma) @ Y.conj().T
    return st, sigma, M


def _identity_gate():
    return [np.eye(len(gate_basis(n, D)), dtype=np.complex128) for n in range(2 * (D - 1) + 1)]


def test_floor_is_32_eps_of_the_sectors_frobenius_norm():
    st, sigma, M = _planted_state()
    raw = np.linalg.svd(M, compute_uv=False)
    # LAPACK resolves both planted values to well under their distance from the floor
    assert abs(raw[16] - sigma[16]) < 0.05 * sigma[16] and abs(raw[17] - sigma[17]) < 0.05 * sigma[17]
    info = st.apply_gate2(S, _identity_gate(), CHI, 0.0)
    got = info["sigmas"][C]
    assert np.count_nonzero(got) == 17
    assert got[16] > 0.0 and got[17] == 0.0 and np.all(got[18:] == 0.0)
    assert np.max(np.abs(got[:16] - 1.0)) < 1e-13
    assert abs(got[16] - sigma[16]) < 0.05 * sigma[16]
    assert info["kept"][C] == 17              # cutoff 0: every numerically nonzero value is kept
    # other floors would keep other counts: against the sector's largest value (spectral
    # norm) both planted values survive; against the whole update's norm neither does
    norm_all = math.sqrt(sum(float(np.sum(v * v)) for v in info["sigmas"].values()))
    assert np.count_nonzero(raw > NOISE_REL * raw[0]) >= 18
    assert np.count_nonzero(raw > NOISE_REL * norm_all) == 16


def test_floor_sits_between_the_planted_values_after_renormalisation():
    """The kept planted value reappears as a Schmidt value of the new bond, scaled by the
    renormalisation 1 / |S_kept| like every other value."""
    st, sigma, _ = _planted_state()
    info = st.apply_gate2(S, _identity_gate(), CHI, 0.0)
    lam = st.lam[S + 1][C]
    assert len(lam) == 17
    assert abs(lam[16] * info["kept_norm"] - sigma[16]) < 0.05 * sigma[16]
    assert isinstance(st, U1MPS)
