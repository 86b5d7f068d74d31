"""Charge-block two-site gates for the oracle (TEST INFRASTRUCTURE ONLY).

A U(1)-conserving two-site gate is block diagonal in the total charge
n = i + j of the pair (Sec. II: [H, N] = 0, so the dynamics preserve the total
charge).  Block n acts on the basis (i, n - i), i ascending, with
0 <= i, n - i <= d - 1; rows are outputs, columns inputs.

Models are the paper's examples of U(1) symmetry (Sec. I): the XXZ chain, the
Bose-Hubbard chain and boson-sampling beam splitters.  Conventions the paper
leaves open (J = 1, spin-1/2 operators, on-site weights, the beam-splitter
matrix) are readings made here; the CUDA path's gate builders use the same ones.
"""
from __future__ import annotations

import math

import numpy as np

from .permanent import permanent_ryser
from .u1mps import gate_basis


def _expm_hermitian(h: np.ndarray, tau: float) -> np.ndarray:
    """exp(-i h tau) of a Hermitian matrix through its eigendecomposition."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(-1j * w * tau)) @ v.conj().T


def xxz_h_blocks(delta: float, J: float = 1.0):
    """h = J (S+S- + S-S+)/2 + Delta Sz Sz on two spin-1/2 sites, by charge n.

    Occupation 1 is spin up; Sz = i - 1/2.
    """
    blocks = []
    for n in range(3):
        basis = gate_basis(n, 2)
        h = np.zeros((len(basis), len(basis)))
        for a, i in enumerate(basis):
            j = n - i
            h[a, a] = delta * (i - 0.5) * (j - 0.5)
            for b, i2 in enumerate(basis):
                if i2 == i + 1 and j >= 1:  # S+_1 S-_2 |i, j> = |i+1, j-1>
                    h[b, a] += 0.5 * J
                if i2 == i - 1:             # S-_1 S+_2
                    h[b, a] += 0.5 * J
        blocks.append(h)
    return blocks


def bh_h_blocks(d: int, J: float, U: float, w_left: float, w_right: float):
    """h = -J (b1^dag b2 + b1 b2^dag) + U/2 (w1 n1(n1-1) + w2 n2(n2-1)) by charge n.

    b^dag |k> = sqrt(k+1) |k+1>, truncated at k = d - 1.
    """
    blocks = []
    for n in range(2 * d - 1):
        basis = gate_basis(n, d)
        idx = {i: a for a, i in enumerate(basis)}
        h = np.zeros((len(basis), len(basis)))
        for a, i in enumerate(basis):
            j = n - i
            h[a, a] = 0.5 * U * (w_left * i * (i - 1) + w_right * j * (j - 1))
            # b1^dag b2 |i, j> = sqrt(i+1) sqrt(j) |i+1, j-1>
            if i + 1 in idx and j >= 1:
                h[idx[i + 1], a] += -J * math.sqrt(i + 1) * math.sqrt(j)
            # b1 b2^dag |i, j> = sqrt(i) sqrt(j+1) |i-1, j+1>
            if i - 1 in idx and i >= 1:
                h[idx[i - 1], a] += -J * math.sqrt(i) * math.sqrt(j + 1)
        blocks.append(h)
    return blocks


def bh_weights(L: int, s: int) -> tuple[float, float]:
    """On-site weight of the two sites of bond (s, s+1): 1 at chain ends, 1/2 inside."""
    wl = 1.0 if s == 0 else 0.5
    wr = 1.0 if s + 1 == L - 1 else 0.5
    return wl, wr


def exp_blocks(h_blocks, tau: float):
    return [_expm_hermitian(h, tau) for h in h_blocks]


def xxz_gate(delta: float, tau: float, J: float = 1.0):
    return exp_blocks(xxz_h_blocks(delta, J), tau)


def bh_gate(L: int, s: int, d: int, J: float, U: float, tau: float):
    wl, wr = bh_weights(L, s)
    return exp_blocks(bh_h_blocks(d, J, U, wl, wr), tau)


def beam_splitter_u(theta: float, phi: float) -> np.ndarray:
    """2x2 mode transformation a_i^dag -> sum_j u_ji a_j^dag of one beam splitter."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -np.exp(-1j * phi) * s],
                     [np.exp(1j * phi) * s, c]], dtype=np.complex128)


def beam_splitter_gate(theta: float, phi: float, d: int):
    """Fock-space blocks <p,q|U|s,t> = Perm(u[0^p 1^q ; 0^s 1^t]) / sqrt(p! q! s! t!).

    Restricted to occupations <= d - 1 (truncated Fock space).
    """
    u = beam_splitter_u(theta, phi)
    blocks = []
    for n in range(2 * d - 1):
        basis = gate_basis(n, d)
        g = np.zeros((len(basis), len(basis)), dtype=np.complex128)
        for a, p in enumerate(basis):
            q = n - p
            rows = [0] * p + [1] * q
            for b, s in enumerate(basis):
                t = n - s
                cols = [0] * s + [1] * t
                sub = u[np.ix_(rows, cols)] if n > 0 else np.ones((0, 0))
                perm = permanent_ryser(sub) if n > 0 else 1.0
                g[a, b] = perm / math.sqrt(math.factorial(p) * math.factorial(q)
                                           * math.factorial(s) * math.factorial(t))
        blocks.append(g)
    return blocks


def flatten_blocks(blocks) -> np.ndarray:
    """Blocks n = 0..2(d-1), each row-major, concatenated as complex128."""
    return np.concatenate([np.asarray(b, dtype=np.complex128).reshape(-1) for b in blocks])


# ---------------------------------------------------------------------------
# Z_n clock chain (the Z_n-symmetric example; n = 2 is the transverse-field Ising chain)
# ---------------------------------------------------------------------------

def clock_h_blocks(n: int, J: float, f: float, w_left: float, w_right: float):
    """h = -J (Z1 Z2^dag + Z1^dag Z2) - f (w1 (X1 + X1^dag) + w2 (X2 + X2^dag)) by Z_n charge.

    Local basis |k>, k = 0..n-1, is the Z_n charge: X|k> = w^k |k> (w = exp(2 pi i / n)),
    so X + X^dag = diag(2 cos(2 pi k / n)), and Z|k> = |k+1 mod n> shifts the charge, so
    Z1 Z2^dag conserves the pair's total (i + j) mod n.  Block q acts on (i, (q - i) mod n),
    i ascending.  w1, w2 count each on-site term once per step (as for Bose-Hubbard).
    """
    xs = 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
    blocks = []
    for q in range(n):
        basis = [(i, (q - i) % n) for i in range(n)]
        idx = {b: a for a, b in enumerate(basis)}
        h = np.zeros((n, n))
        for a, (i, j) in enumerate(basis):
            h[a, a] = -f * (w_left * xs[i] + w_right * xs[j])
            for di in (1, -1):           # Z1 Z2^dag: (i, j) -> (i+1, j-1); its adjoint the reverse
                b = idx[((i + di) % n, (j - di) % n)]
                h[b, a] += -J
        blocks.append(h)
    return blocks


def clock_gate(L: int, s: int, n: int, J: float, f: float, tau: float):
    """exp(-i h tau) per Z_n block for the bond (s, s+1), chain-end weights as bh_weights."""
    wl, wr = bh_weights(L, s)
    return [_expm_hermitian(h, tau) for h in clock_h_blocks(n, J, f, wl, wr)]
