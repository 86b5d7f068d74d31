"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmarks.

This module only draws numbers and lays out inputs: initial occupations, Haar
angles and Haar-random unitaries, random blocks and weights, the request mix, and
the recipe of a synthetic saturated chain (sector sizes in proportion to a count of
occupation strings).  It holds none of the two-site update's arithmetic (no
contraction, no SVD, no truncation), so the CUDA path and the float64 oracle can
both take their inputs from it without sharing any of the method.

Workloads follow the model families the paper names for U(1)-symmetric tensor
networks (Sec. I: Bose-Hubbard chains, XXZ spin chains, boson-sampling
circuits).  The paper prints no benchmark inputs, so every input here is
synthetic and seeded (numpy PCG64).
"""
from __future__ import annotations

import functools

import numpy as np

__all__ = [
    "neel_occupations",
    "mott_occupations",
    "single_photon_occupations",
    "haar_beam_splitter_angles",
    "brickwork_pairs",
    "random_complex",
    "random_positive",
    "random_occupations",
    "serving_requests",
    "haar_unitary",
    "random_u1_gate",
    "saturated_sector_dims",
    "saturated_random_state",
    "entanglement_weights",
    "uniforms",
]


def neel_occupations(L: int) -> list[int]:
    """Neel product state of an XXZ chain: up (occupation 1) on even 0-based sites."""
    return [1 if s % 2 == 0 else 0 for s in range(L)]


def mott_occupations(L: int, filling: int = 1) -> list[int]:
    """Mott product state of a Bose-Hubbard chain: `filling` bosons on every site."""
    return [filling] * L


def single_photon_occupations(M: int, n_photons: int) -> list[int]:
    """Boson-sampling input: one photon in each of modes 0..n_photons-1."""
    return [1 if j < n_photons else 0 for j in range(M)]


def brickwork_pairs(M: int, depth: int) -> list[list[int]]:
    """Left-mode indices of the beam splitters of a brickwork interferometer.

    Layer l (0-based) acts on pairs (0,1),(2,3),... when l is even and on
    (1,2),(3,4),... when l is odd.
    """
    layers = []
    for layer in range(depth):
        start = layer % 2
        layers.append(list(range(start, M - 1, 2)))
    return layers


def haar_beam_splitter_angles(n_gates: int, seed: int = 0) -> np.ndarray:
    """(theta, phi) per beam splitter, Haar-distributed on U(2)/phases.

    sin^2(theta) ~ U[0,1] and phi ~ U[0, 2 pi), drawn from numpy PCG64(seed).
    Returns an (n_gates, 2) float64 array.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(n_gates)
    phi = rng.random(n_gates) * 2.0 * np.pi
    theta = np.arcsin(np.sqrt(u))
    return np.stack([theta, phi], axis=1)


def random_complex(shape, rng: np.random.Generator) -> np.ndarray:
    """Complex normal entries (real and imaginary parts standard normal)."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_positive(n: int, rng: np.random.Generator) -> np.ndarray:
    """Positive reals in (0.05, 1], sorted descending (stand-in Schmidt weights)."""
    v = 0.05 + 0.95 * rng.random(n)
    return np.sort(v)[::-1].copy()


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """An n x n unitary drawn from the Haar measure: Q of the QR decomposition of a
    complex Gaussian matrix, each column multiplied by the phase of R's diagonal entry
    (Mezzadri's recipe)."""
    z = random_complex((n, n), rng) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    dg = np.diag(r)
    return q * (dg / np.abs(dg))[None, :]


def random_u1_gate(d: int, rng: np.random.Generator) -> list[np.ndarray]:
    """A charge-conserving two-site gate with Haar-random charge blocks.

    Block n (n = 0..2(d-1)) acts on the states (i, n - i) of two sites of local
    dimension d, so its size is the number of such i in [0, d-1]."""
    blocks = []
    for n in range(2 * (d - 1) + 1):
        size = min(d - 1, n) - max(0, n - d + 1) + 1
        blocks.append(haar_unitary(size, rng))
    return blocks


def uniforms(n: int, L: int, seed: int = 0) -> np.ndarray:
    """n x L uniform numbers in [0, 1) (numpy PCG64(seed)): the random draws of pattern
    sampling, one per site per sample, handed to both the CUDA path and the oracle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, L))


def random_occupations(L: int, d: int, N: int, rng: np.random.Generator) -> list[int]:
    """A random product state of L sites, local dimension d, total charge N."""
    if N > L * (d - 1):
        raise ValueError("N too large for L sites of dimension d")
    occ = [0] * L
    left = N
    while left:
        s = int(rng.integers(L))
        if occ[s] < d - 1:
            occ[s] += 1
            left -= 1
    return occ


def serving_requests(n: int, seed: int = 0, rate_hz: float = 1.0, L_choices=(32, 64, 128),
                     chi_choices=(64, 256, 1024), steps_range=(50, 500)):
    """Seeded request mix for the serving workload.

    Each request is a dict: arrival time (Poisson process of `rate_hz`), model
    ('xxz' with Delta ~ U[0,2], or 'bh' with U/J ~ U[1,10]), chain length L from
    L_choices, chi from chi_choices and a Trotter step count in steps_range
    (inclusive).  The defaults are the full serving configuration.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps)
    out = []
    for k in range(n):
        model = "xxz" if rng.random() < 0.5 else "bh"
        L = int(rng.choice(list(L_choices)))
        chi = int(rng.choice(list(chi_choices)))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        param = float(rng.uniform(0.0, 2.0)) if model == "xxz" else float(rng.uniform(1.0, 10.0))
        out.append(dict(id=k, arrival=float(t[k]), model=model, L=L, chi=chi, steps=steps, param=param))
    return out


@functools.lru_cache(maxsize=None)
def _string_table(n_sites: int, d: int) -> tuple:
    """Row n of the table is the count of occupation strings of n sites (0..d-1 each)
    for every total q = 0..n (d-1); built once per (n_sites, d) by adding one site at a
    time (exact integers)."""
    rows = [(1,)]
    for n in range(1, n_sites + 1):
        prev = rows[-1]
        qmax = n * (d - 1)
        rows.append(tuple(sum(prev[q - i] for i in range(d) if 0 <= q - i < len(prev))
                          for q in range(qmax + 1)))
    return tuple(rows)


def _strings(n_sites: int, d: int, q: int) -> int:
    """Number of occupation strings of n_sites sites (0..d-1 each) summing to q."""
    if q < 0 or q > n_sites * (d - 1):
        return 0
    return _string_table(max(n_sites, 1), d)[n_sites][q]


def saturated_sector_dims(L: int, d: int, N: int, b: int, chi: int) -> dict:
    """Sector dimensions {charge: dim} of bond b of a chain at saturation: chi spread over
    the charges c the bond can carry in proportion to min(#strings of the left part with
    N - c particles, #strings of the right part with c), each capped by that bound."""
    lo, hi = max(0, N - (d - 1) * b), min(N, (d - 1) * (L - b))
    bound = {c: min(_strings(b, d, N - c), _strings(L - b, d, c)) for c in range(lo, hi + 1)}
    bound = {c: v for c, v in bound.items() if v > 0}
    tot = sum(bound.values())
    if tot <= chi:
        return bound
    dims = {c: min(v, int(chi * v / tot)) for c, v in bound.items()}
    dims = {c: v for c, v in dims.items() if v > 0}
    return dims or {max(bound, key=bound.get): 1}


def entanglement_weights(n: int, beta: float, rng: np.random.Generator) -> np.ndarray:
    """n positive weights w_k = exp(-beta (ln k)^2), k = 1..n, in a random order (stand-in
    Schmidt values with the decay of an evolved chain's entanglement spectrum)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.exp(-beta * np.log(k) ** 2)[rng.permutation(n)]


def saturated_random_state(L: int, d: int, N: int, chi: int, seed: int, beta: float | None = None):
    """A synthetic saturated chain: every inner bond at saturated_sector_dims, positive
    Schmidt-like weights (unit norm per bond, descending per sector) and complex normal
    blocks for every allowed (l, m) pair (0 <= l - m <= d - 1) scaled by 1/sqrt(max dim).
    Weights: beta None draws them flat (random_positive, within a factor 20 of each other);
    a number draws entanglement_weights(., beta) and deals them to the sectors at random.
    Not canonical; it gives an update the sector sizes and the cost of a saturated one.
    Returns (lam, blocks): lam[b] = {c: weights} for b = 1..L-1 (index 0 and L unused),
    blocks[s] = {(l, m): array}."""
    rng = np.random.default_rng(seed)
    bonds = [None] * (L + 1)
    bonds[0], bonds[L] = {N: 1}, {0: 1}
    lam = [None] * (L + 1)
    for b in range(1, L):
        bonds[b] = dict(sorted(saturated_sector_dims(L, d, N, b, chi).items()))
        n_b = sum(bonds[b].values())
        w = random_positive(n_b, rng) if beta is None else entanglement_weights(n_b, beta, rng)
        w /= np.linalg.norm(w)
        lam[b], off = {}, 0
        for c, D in bonds[b].items():
            lam[b][c] = np.sort(w[off:off + D])[::-1].copy()
            off += D
    blocks = []
    for s in range(L):
        blk = {}
        for l, Dl in bonds[s].items():
            for m, Dm in bonds[s + 1].items():
                if 0 <= l - m <= d - 1:
                    blk[(l, m)] = random_complex((Dl, Dm), rng) / np.sqrt(max(Dl, Dm))
        blocks.append(blk)
    return lam, blocks
