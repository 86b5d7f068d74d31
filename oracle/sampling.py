"""Sequential sampling of occupation patterns from the U(1) MPS (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
import this module; the library never does.

What it computes.  The amplitude of a pattern i_0..i_{L-1} is the product of the one
block per site its right-charges select (Sec. II, U(1) amplitude formula).  In the
right-canonical form the state keeps (B = Gamma lambda), the sites right of bond s form
an isometry, so the probability of a prefix i_0..i_{s-1} is the squared norm of the row
vector v_s = B^[0][c_0, c_1] ... B^[s-1][c_{s-1}, c_s].  The pattern is drawn site by
site: at site s every occupation i with a block (c_s, c_s - i) gets the weight
w_i = |v_s B^[s][c_s, c_s - i]|^2, the conditional probability is w_i / sum_j w_j (the
normalisation absorbs any drift from exact canonical form that truncation leaves), and i
is the first occupation, in ascending order, whose cumulative probability exceeds the
caller's uniform number u_s in [0, 1).  The row vector is then advanced to v_s B and
rescaled to unit norm (the conditionals are ratios).  The probability of the drawn
pattern is the product of its conditionals; on an exactly canonical, untruncated state
it equals |<pattern|psi>|^2 (for boson sampling |Perm(U_{t,s})|^2 / prod t!).

Reading (the paper describes no sampling): the uniform numbers are inputs, one per site
per sample, so the CUDA path and this oracle draw from the same numbers.
"""
from __future__ import annotations

import numpy as np

from .u1mps import U1MPS


def sample_patterns(st: U1MPS, uniforms: np.ndarray):
    """Patterns drawn with uniforms[k, s] at site s of sample k.

    Returns (patterns: int32 array (n, L), probs: float64 array (n,)), the probability
    being the product of the conditionals taken.
    """
    u = np.asarray(uniforms, dtype=np.float64)
    n, L = u.shape
    if L != st.L:
        raise ValueError("one uniform per site")
    pats = np.zeros((n, L), dtype=np.int32)
    probs = np.ones(n)
    for k in range(n):
        c = st.N
        v = np.ones((1, 1), dtype=np.complex128)
        p = 1.0
        for s in range(L):
            cands = []
            for i in range(st.d):
                blk = st.B[s].get((c, c - i))
                if blk is None:
                    continue
                w = v @ blk
                cands.append((i, w, float(np.vdot(w, w).real)))
            tot = sum(x[2] for x in cands)
            if not cands or tot <= 0.0:
                raise FloatingPointError("no continuation with nonzero weight")
            acc = 0.0
            pick = cands[-1]
            for cand in cands:
                acc += cand[2] / tot
                if u[k, s] < acc:
                    pick = cand
                    break
            i, w, wi = pick
            pats[k, s] = i
            p *= wi / tot
            v = w / np.sqrt(wi)
            c -= i
        probs[k] = p
    return pats, probs


def pattern_probability(st: U1MPS, pattern) -> float:
    """Product of the sequential conditionals along a given pattern (0 if it is not allowed)."""
    c = st.N
    v = np.ones((1, 1), dtype=np.complex128)
    p = 1.0
    for s, i in enumerate(int(x) for x in pattern):
        ws = {}
        for j in range(st.d):
            blk = st.B[s].get((c, c - j))
            if blk is not None:
                w = v @ blk
                ws[j] = (w, float(np.vdot(w, w).real))
        tot = sum(x[1] for x in ws.values())
        if i not in ws or tot <= 0.0 or ws[i][1] == 0.0:
            return 0.0
        w, wi = ws[i]
        p *= wi / tot
        v = w / np.sqrt(wi)
        c -= i
    return p if c == 0 else 0.0
