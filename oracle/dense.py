"""Dense state-vector evolution (TEST INFRASTRUCTURE ONLY).

An independent check of the block-sparse oracle: two-site Hamiltonians are
built from ladder operators with Kronecker products (no charge blocks), gates
come from scipy's general matrix exponential, and the state is the full
d^L vector.  Used only for small chains.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def ladder(d: int):
    """Annihilation b (b|k> = sqrt(k)|k-1>), creation b^dag and number operator."""
    b = np.diag(np.sqrt(np.arange(1, d, dtype=float)), k=1)
    return b, b.T.copy(), np.diag(np.arange(d, dtype=float))


def xxz_two_site(delta: float, J: float = 1.0) -> np.ndarray:
    b, bd, n = ladder(2)
    sz = n - 0.5 * np.eye(2)
    return 0.5 * J * (np.kron(bd, b) + np.kron(b, bd)) + delta * np.kron(sz, sz)


def bh_two_site(d: int, J: float, U: float, w_left: float, w_right: float) -> np.ndarray:
    b, bd, n = ladder(d)
    eye = np.eye(d)
    onsite = n @ (n - eye)
    return (-J * (np.kron(bd, b) + np.kron(b, bd))
            + 0.5 * U * (w_left * np.kron(onsite, eye) + w_right * np.kron(eye, onsite)))


def beam_splitter_two_site(theta: float, phi: float, d: int) -> np.ndarray:
    """exp(theta (-e^{-i phi} a0^dag a1 + e^{i phi} a1^dag a0)) on two truncated modes."""
    b, bd, _ = ladder(d)
    gen = theta * (-np.exp(-1j * phi) * np.kron(bd, b) + np.exp(1j * phi) * np.kron(b, bd))
    return scipy.linalg.expm(gen)


def gate_from_h(h: np.ndarray, tau: float) -> np.ndarray:
    return scipy.linalg.expm(-1j * tau * h)


def product_state(d: int, occupations) -> np.ndarray:
    psi = np.zeros((d,) * len(occupations), dtype=np.complex128)
    psi[tuple(occupations)] = 1.0
    return psi


def apply_two_site(psi: np.ndarray, s: int, gate: np.ndarray) -> np.ndarray:
    """psi'[.., a, b, ..] = sum_{i,j} gate[(a,b),(i,j)] psi[.., i, j, ..] on sites s, s+1."""
    d = psi.shape[0]
    L = psi.ndim
    x = psi.reshape(d ** s, d * d, d ** (L - s - 2))
    y = np.einsum("ai,xiy->xay", gate, x)
    return y.reshape(psi.shape)


def density(psi: np.ndarray, s: int) -> float:
    d = psi.shape[0]
    p = np.abs(psi) ** 2
    axes = tuple(a for a in range(psi.ndim) if a != s)
    marg = p.sum(axis=axes)
    return float(np.dot(marg, np.arange(d)) / p.sum())


def bond_entropy(psi: np.ndarray, b: int) -> float:
    d = psi.shape[0]
    m = psi.reshape(d ** b, -1)
    sv = np.linalg.svd(m, compute_uv=False)
    p = sv ** 2 / np.sum(sv ** 2)
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def schmidt_values(psi: np.ndarray, b: int) -> np.ndarray:
    d = psi.shape[0]
    return np.linalg.svd(psi.reshape(d ** b, -1), compute_uv=False)


def clock_ops(n: int):
    """Z_n clock operators in the charge basis: X = diag(w^k), Z|k> = |k+1 mod n>."""
    X = np.diag(np.exp(2j * np.pi * np.arange(n) / n))
    Z = np.roll(np.eye(n), 1, axis=0)
    return X, Z


def clock_two_site(n: int, J: float, f: float, w_left: float, w_right: float) -> np.ndarray:
    """-J (Z1 Z2^dag + h.c.) - f (w1 (X1 + X1^dag) + w2 (X2 + X2^dag)) by Kronecker products."""
    X, Z = clock_ops(n)
    eye = np.eye(n)
    zz = np.kron(Z, Z.conj().T)
    xx = X + X.conj().T
    return -J * (zz + zz.conj().T) - f * (w_left * np.kron(xx, eye) + w_right * np.kron(eye, xx))


def mean_op(psi: np.ndarray, s: int, diag: np.ndarray) -> float:
    """<psi| O_s |psi> / <psi|psi> for O diagonal in the local basis."""
    p = np.abs(psi) ** 2
    axes = tuple(a for a in range(psi.ndim) if a != s)
    marg = p.sum(axis=axes)
    return float(np.dot(marg, diag) / p.sum())
