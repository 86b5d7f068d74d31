"""Serving: continuous batching of independent TEBD requests on one GPU.

A request's result must not depend on what it shares launches with: every
request is served in a mix (staggered arrivals, slots freed and refilled
mid-run, XXZ and Bose-Hubbard together) and again alone, and the observables
must agree within 1e-12.
"""
import numpy as np
import pytest

from oracle import U1MPS, tebd

pytestmark = pytest.mark.gpu


def _requests(m):
    R = m.serve.Request
    return [
        R(0, "xxz", 12, 32, 6, 0.5, arrival=0.00),
        R(1, "bh", 10, 24, 4, 2.0, arrival=0.00),
        R(2, "xxz", 16, 40, 3, 1.3, arrival=0.02),
        R(3, "bh", 8, 30, 5, 6.5, arrival=0.05),
        R(4, "xxz", 10, 16, 8, 0.0, arrival=0.05),
        R(5, "bh", 12, 20, 3, 9.0, arrival=0.10),
    ]


@pytest.mark.parametrize("lanes", [1, 2])
def test_mix_equals_alone(gpu_lib, lanes):
    """With one executor, and with two executor lanes on their own streams running each tick's
    calls from two host threads at once."""
    m = gpu_lib
    reqs = _requests(m)
    srv = m.serve.Server(budget_bytes=8 << 30, max_slots=3, lanes=lanes)
    mixed = {r.id: r for r in srv.run(reqs)}
    assert srv.max_active_seen <= 3
    for req in reqs:
        solo = m.serve.Server(budget_bytes=8 << 30, max_slots=1)
        alone = solo.run([m.serve.Request(**{**req.__dict__, "arrival": 0.0})])[0]
        solo.close()
        a, b = mixed[req.id], alone
        assert a.updates == b.updates
        scale = max(1.0, np.max(np.abs(b.observables)))
        assert np.max(np.abs(a.observables - b.observables)) <= 1e-12 * scale, req.id
    srv.close()


def test_served_request_matches_oracle(gpu_lib):
    m = gpu_lib
    req = m.serve.Request(7, "bh", 8, 24, 4, 2.0)
    srv = m.serve.Server(budget_bytes=4 << 30)
    res = srv.run([req])[0]
    srv.close()
    st = U1MPS.product(5, [1] * 8)
    tebd.run_tebd(st, tebd.bh_gates(8, 5, 1.0, 2.0, 0.02), 4, 24, 1e-10)
    ref = np.array([st.expect_local(s, np.arange(5)) for s in range(8)])
    assert np.max(np.abs(res.observables - ref)) <= 1e-9 * 4


def test_admission_respects_the_memory_budget(gpu_lib):
    m = gpu_lib
    reqs = _requests(m)
    sizes = sorted(m.serve.footprint(r) for r in reqs)
    budget = sizes[-1] + sizes[-2]            # room for the two largest at once, no more
    srv = m.serve.Server(budget_bytes=budget, max_slots=16)
    res = srv.run(reqs)
    srv.close()
    assert len(res) == len(reqs)
    assert srv.max_bytes_seen <= budget
    s = m.serve.summarize(res, max(r.finished for r in res))
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
