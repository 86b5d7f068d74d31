"""Float64 CPU oracle of the U(1)-symmetric two-site TEBD update.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the cpu_baseline / reference leg of bench.py, never by the library.  It shares
no code with the CUDA path.  Functions whose parity has no independent pin say
"parity unpinned" in their docstring; every function here is pinned by the
-m "not gpu" tests (dense evolution, free fermions, permanents, invariants).
"""
from .u1mps import (TIE_REL, U1MPS, SectorPlan, bond_charge_range, count_configs,  # noqa: F401
                    gate_basis, hilbert_dim, plan_update, select_kept)
from . import gates, tebd, dense, freefermion, permanent, sampling, synth, dmrg, multiu1  # noqa: F401
