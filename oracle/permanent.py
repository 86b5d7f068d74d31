"""Matrix permanents for the oracle (TEST INFRASTRUCTURE ONLY).

Boson-sampling amplitudes are permanents of submatrices of the interferometer
(the paper's boson-sampling example of U(1) symmetry, Sec. I).
"""
from __future__ import annotations

import itertools

import numpy as np


def permanent_bruteforce(a: np.ndarray) -> complex:
    """Perm(A) = sum over permutations sigma of prod_i A[i, sigma(i)]."""
    n = a.shape[0]
    if n == 0:
        return 1.0 + 0j
    tot = 0j
    for perm in itertools.permutations(range(n)):
        p = 1.0 + 0j
        for i in range(n):
            p *= a[i, perm[i]]
        tot += p
    return tot


def permanent_ryser(a: np.ndarray) -> complex:
    """Ryser's inclusion-exclusion formula, O(2^n n^2)."""
    n = a.shape[0]
    if n == 0:
        return 1.0 + 0j
    tot = 0j
    for mask in range(1, 1 << n):
        cols = [j for j in range(n) if mask >> j & 1]
        rowsums = a[:, cols].sum(axis=1)
        term = np.prod(rowsums)
        tot += (-1) ** len(cols) * term
    return (-1) ** n * tot
