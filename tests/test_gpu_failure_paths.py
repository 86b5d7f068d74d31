"""Failure detection on the GPU without faulting it.

Non-convergence: a Jacobi sweep limit of 1 leaves graded sectors unconverged; the
update reports MPS_ENOCONV (a JacobiNotConverged warning in Python), still updates the
state with valid charge structure, and a later update with the normal limit works.

Bounded waits: with stall injection on, the tensor-core GEMM kernels issue no MMA, so
their mbarrier waits run out after ~50 ms and the calls report MPS_ETIMEOUT; an update
on a TF32 handle leaves its state unchanged; with injection off again the same context
computes correct products and updates.
"""
import numpy as np
import pytest

import workloads as W
from oracle import gates
from tests.helpers import compare_update, load_state, random_state

pytestmark = pytest.mark.gpu


def test_sweep_limit_reports_non_convergence_and_the_handle_recovers(gpu_lib):
    m = gpu_lib
    L, d, N = 8, 3, 8
    st = random_state(L, d, N, 60, seed=9)
    g = m.MPS(d, [1] * L, 80)
    load_state(g, st)
    G = gates.bh_gate(L, 3, d, 1.0, 2.0, 0.4)
    with pytest.raises(m.MPSError):
        g.set_sweep_limit(0)
    g.set_sweep_limit(1)
    with pytest.warns(m.JacobiNotConverged):
        g.apply_gate2(3, G, 40, 1e-10)
    # the charge structure is still valid: every kept charge is one the update can produce
    plan_charges = {c for c in g.bond_dims(4)}
    assert plan_charges and all(0 <= c <= N for c in plan_charges)
    lam = np.concatenate(list(g.bond(4).values()))
    assert abs(np.sum(lam ** 2) - 1.0) < 1e-12
    # back to the normal limit: a fresh load and update match the oracle again
    g.set_sweep_limit(40)
    load_state(g, st)
    g.apply_gate2(3, G, 40, 1e-10)
    st.apply_gate2(3, G, 40, 1e-10)
    compare_update(g, st, 3)
    g.close()


def test_tensor_core_wait_expiry_is_reported_and_the_context_survives(gpu_lib):
    m = gpu_lib
    rng = np.random.default_rng(0)
    A = W.random_complex((150, 70), rng)
    B = W.random_complex((70, 90), rng)
    L, d, N = 8, 3, 8
    st = random_state(L, d, N, 40, seed=4)
    g = m.MPS(d, [1] * L, 60, precision=m.MPS_TF32)
    load_state(g, st)
    G = gates.bh_gate(L, 2, d, 1.0, 2.0, 0.3)
    before = g.site(2)
    m.tc_inject_stall(True)
    try:
        with pytest.raises(m.MPSError) as e:
            m.zgemm_tc(A, B, precision=m.MPS_TF32)
        assert e.value.code == m.MPS_ETIMEOUT
        with pytest.raises(m.MPSError) as e:
            g.apply_gate2(2, G, 40, 1e-10)
        assert e.value.code == m.MPS_ETIMEOUT
    finally:
        m.tc_inject_stall(False)
    after = g.site(2)                                  # the failed update changed nothing
    assert before.keys() == after.keys()
    for k in before:
        assert np.array_equal(before[k], after[k])
    C = m.zgemm_tc(A, B, precision=m.MPS_TF32)        # the context is still usable
    assert np.max(np.abs(C - A @ B)) <= 2e-3 * np.max(np.abs(A @ B))
    g.apply_gate2(2, G, 40, 1e-10)
    assert abs(sum(float(np.sum(v ** 2)) for v in g.bond(3).values()) - 1.0) < 1e-12
    g.close()
