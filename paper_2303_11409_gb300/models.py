"""Charge-block two-site gates of the models the library is benchmarked on.

Host-side model set-up (FP64, once per workload), not part of the update path.
A gate conserving the total charge n = i + j of a site pair is given by its
blocks G_n over the basis (i, n - i), i ascending (the layout of the C ABI).
Models: XXZ chain, Bose-Hubbard chain, boson-sampling beam splitter (the U(1)
examples of arXiv:2303.11409, Sec. I), and the Z_n clock chain for the cyclic-group
handles (mps_create_zn; n = 2 is the transverse-field Ising chain): its gates have the n
blocks q = (i + j) mod n over the pairs (i, (q - i) mod n), i ascending.  cyclic_blocks
regroups a U(1) gate for a Z_n handle with d < n (mps_create_cyclic).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def basis(n: int, d: int) -> range:
    return range(max(0, n - d + 1), min(d - 1, n) + 1)


def xxz_gate(delta: float, tau: float, J: float = 1.0) -> list[np.ndarray]:
    """exp(-i tau h), h = J (S+S- + S-S+)/2 + Delta SzSz, in closed form per block.

    n = 0 and n = 2 (both spins equal) carry Delta/4; n = 1 is
    -Delta/4 + (J/2) sigma_x on (down-up, up-down).
    """
    e_diag = np.exp(-1j * tau * delta / 4.0)
    c, s = math.cos(0.5 * J * tau), math.sin(0.5 * J * tau)
    mid = np.exp(1j * tau * delta / 4.0) * np.array([[c, -1j * s], [-1j * s, c]])
    return [np.array([[e_diag]]), mid, np.array([[e_diag]])]


def bose_hubbard_gate(d: int, J: float, U: float, tau: float, w_left: float, w_right: float) -> list[np.ndarray]:
    """exp(-i tau h) per charge block, h = -J(b1^dag b2 + h.c.) + U/2 (w1 n1(n1-1) + w2 n2(n2-1))."""
    out = []
    for n in range(2 * d - 1):
        occ = list(basis(n, d))
        k = len(occ)
        h = np.zeros((k, k))
        for a, i in enumerate(occ):
            j = n - i
            h[a, a] = 0.5 * U * (w_left * i * (i - 1) + w_right * j * (j - 1))
            if a + 1 < k:     # |i, j> -> |i+1, j-1> by b1^dag b2, amplitude sqrt((i+1) j)
                amp = -J * math.sqrt((i + 1) * j)
                h[a + 1, a] = amp
                h[a, a + 1] = amp
        out.append(scipy.linalg.expm(-1j * tau * h))
    return out


def bose_hubbard_weights(L: int, s: int) -> tuple[float, float]:
    """Share of the on-site term given to each bond: a site inside the chain sits on two bonds."""
    return (1.0 if s == 0 else 0.5), (1.0 if s + 1 == L - 1 else 0.5)


def beam_splitter_gate(theta: float, phi: float, d: int) -> list[np.ndarray]:
    """Fock blocks of the beam splitter a_k^dag -> sum_j u_jk a_j^dag, truncated at d - 1.

    u = [[cos t, -e^{-i phi} sin t], [e^{i phi} sin t, cos t]].  By the binomial
    expansion of (u00 a0^dag + u10 a1^dag)^s (u01 a0^dag + u11 a1^dag)^t,
    <p,q|U|s,t> = sqrt(p! q! / (s! t!)) sum_{j+k=p} C(s,j) C(t,k) u00^j u10^(s-j) u01^k u11^(t-k).
    """
    ct, st = math.cos(theta), math.sin(theta)
    u00, u01 = ct, -np.exp(-1j * phi) * st
    u10, u11 = np.exp(1j * phi) * st, ct
    out = []
    for n in range(2 * d - 1):
        occ = list(basis(n, d))
        g = np.zeros((len(occ), len(occ)), dtype=np.complex128)
        for b, s_ in enumerate(occ):
            t_ = n - s_
            for a, p in enumerate(occ):
                q = n - p
                acc = 0j
                for j in range(0, min(s_, p) + 1):
                    k = p - j
                    if k > t_:
                        continue
                    acc += (math.comb(s_, j) * math.comb(t_, k) * u00 ** j * u10 ** (s_ - j)
                            * u01 ** k * u11 ** (t_ - k))
                g[a, b] = acc * math.sqrt(math.factorial(p) * math.factorial(q)
                                          / (math.factorial(s_) * math.factorial(t_)))
        out.append(g)
    return out


def clock_gate(n: int, J: float, f: float, tau: float, w_left: float, w_right: float) -> list[np.ndarray]:
    """exp(-i tau h) per Z_n block, h = -J (Z1 Z2^dag + Z1^dag Z2) - f (w1 (X1 + X1^dag) + w2 (X2 + X2^dag)).

    The local index k is the Z_n charge: X|k> = e^{2 pi i k / n}|k> (X + X^dag is diagonal,
    2 cos(2 pi k / n)) and Z|k> = |k + 1 mod n>, so Z1 Z2^dag moves (i, j) to (i + 1, j - 1)
    within the block of (i + j) mod n.
    """
    field = 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)
    out = []
    for q in range(n):
        h = np.zeros((n, n))
        for a in range(n):                 # basis pair a = (a, (q - a) mod n)
            j = (q - a) % n
            h[a, a] = -f * (w_left * field[a] + w_right * field[j])
            h[(a + 1) % n, a] += -J        # Z1 Z2^dag
            h[(a - 1) % n, a] += -J        # its adjoint
        out.append(scipy.linalg.expm(-1j * tau * h))
    return out


def cyclic_blocks(u1_blocks, d: int, n: int) -> list[np.ndarray]:
    """The gate of a U(1)-conserving model in the layout of a Z_n handle with local dimension
    d <= n (mps_create_cyclic): the particle number mod n is conserved too, so the Z_n block of
    residue q holds the U(1) blocks of the totals t = q, q + n, ... (zero between different t),
    over the pairs (i, (q - i) mod n) with both entries below d, i ascending; residues that no
    pair reaches are left out."""
    out = []
    for q in range(n):
        pairs = [(i, (q - i) % n) for i in range(d) if (q - i) % n < d]
        if not pairs:
            continue
        G = np.zeros((len(pairs), len(pairs)), dtype=np.complex128)
        for a, (i, j) in enumerate(pairs):
            for b, (k, l) in enumerate(pairs):
                t = i + j
                if k + l == t:
                    lo = max(0, t - d + 1)
                    G[a, b] = u1_blocks[t][i - lo, k - lo]
        out.append(G)
    return out


def xxz_bond_term(delta: float, J: float = 1.0) -> list[np.ndarray]:
    """Charge blocks of h = J (S+S- + S-S+)/2 + Delta SzSz (the generator of xxz_gate), for mps_dmrg."""
    return [np.array([[delta / 4.0]]), np.array([[-delta / 4.0, 0.5 * J], [0.5 * J, -delta / 4.0]]),
            np.array([[delta / 4.0]])]


def bose_hubbard_bond_term(d: int, J: float, U: float, w_left: float, w_right: float) -> list[np.ndarray]:
    """Charge blocks of h = -J(b1^dag b2 + h.c.) + U/2 (w1 n1(n1-1) + w2 n2(n2-1)), for mps_dmrg."""
    out = []
    for n in range(2 * d - 1):
        occ = list(basis(n, d))
        k = len(occ)
        h = np.zeros((k, k))
        for a, i in enumerate(occ):
            j = n - i
            h[a, a] = 0.5 * U * (w_left * i * (i - 1) + w_right * j * (j - 1))
            if a + 1 < k:
                amp = -J * math.sqrt((i + 1) * j)
                h[a + 1, a] = amp
                h[a, a + 1] = amp
        out.append(h)
    return out


def chain_bond_terms(model: str, L: int, d: int, **p) -> list[list[np.ndarray]]:
    """The L - 1 bond terms of an XXZ ("xxz": delta, J) or Bose-Hubbard ("bh": J, U) chain."""
    if model == "xxz":
        t = xxz_bond_term(p.get("delta", 1.0), p.get("J", 1.0))
        return [t for _ in range(L - 1)]
    return [bose_hubbard_bond_term(d, p.get("J", 1.0), p.get("U", 0.0), *bose_hubbard_weights(L, s))
            for s in range(L - 1)]


def flatten(blocks) -> np.ndarray:
    return np.concatenate([np.asarray(b, dtype=np.complex128).reshape(-1) for b in blocks])
