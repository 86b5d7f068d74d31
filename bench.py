#!/usr/bin/env python
"""Two-site TEBD update throughput of the U(1) block-sparse MPS on one GB300.

Default workload (the largest single-GPU configuration): Bose-Hubbard chain L=128,
local cutoff n_max=4 (d=5), N=128 bosons, J=1, U=2, second-order Trotter layers of
dt=0.02, chi<=2048, cutoff 1e-10, sector GEMMs (the Theta' build and the reassembly
product) in TF32 on the tensor cores with FP32 accumulation, SVD, truncation and
renormalisation in FP64.  The chain starts saturated: every inner bond at chi spread
over its charges in proportion to the Hilbert-space bound of each charge, random
complex blocks (seeded), Schmidt weights exp(-0.3 (ln k)^2) for k = 1..chi dealt to the
sectors at random (the decay of an evolved Bose-Hubbard middle-bond spectrum; evolving
the Mott state to saturation at chi=2048 would take hours).  A "step" is one whole Strang layer of
that chain: the odd bonds with dt/2, the even bonds with dt, the odd bonds with dt/2,
in turn (64, 63, 64 two-site updates), each update running the whole path (planner,
Theta' build, per-sector SVD, global top-chi, reassembly, renormalisation).  The
chain's 17 GB of site tensors exceed the 129 MB L2 many times over; the L2 is also
flushed (256 MiB write) between timed steps, outside the timed events.

Prints one JSON line (rank 0).  --impl reference times the float64 oracle on the host
cores instead (a bounded sample of the same chain's updates per step).  --serve runs
the serving workload (continuous batching) instead.  --case selects the other
configurations (bh64: L=64, chi<=512, FP64, evolved from the Mott state; small:
L=32 for profiler captures; small_tf32: a saturated L=24, chi<=1024 chain in TF32 for
captures of the tensor-core kernels; boson: boson sampling M=100, chi<=1024; dmrg: two-site
DMRG sweeps on the L=64 Bose-Hubbard chain at chi<=256).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

D, J, U, DT, CUTOFF = 5, 1.0, 2.0, 0.02, 1e-10
METRIC = "two-site updates/s"
CASES = {
    # the configuration of record: L=128, chi<=2048, mixed-precision sector GEMMs
    "bh128": dict(L=128, N=128, CHI=2048, precision="tf32", start="saturated", beta=0.3,
                  workload="bose_hubbard_L128_nmax4_N128_J1_U2_dt0.02_chi2048_cutoff1e-10"),
    # L=64, chi<=512, FP64, evolved from the Mott state until the middle bond reaches chi
    "bh64": dict(L=64, N=64, CHI=512, precision="fp64", start="evolved",
                 workload="bose_hubbard_L64_nmax4_N64_J1_U2_dt0.02_chi512_cutoff1e-10"),
    # half the L=64 chain at the same chi and sector sizes, for profiler captures
    "small": dict(L=32, N=32, CHI=512, precision="fp64", start="evolved",
                  workload="bose_hubbard_L32_nmax4_N32_J1_U2_dt0.02_chi512_cutoff1e-10"),
    # a short saturated chain at chi<=1024 with TF32 sector GEMMs (about 1.5 GB), for profiler
    # captures of the tensor-core kernels
    "small_tf32": dict(L=24, N=24, CHI=1024, precision="tf32", start="saturated", beta=0.3,
                       workload="bose_hubbard_L24_nmax4_N24_J1_U2_dt0.02_chi1024_cutoff1e-10"),
    # two-site DMRG ground state of the Bose-Hubbard chain (L=64, N=64, U=2), chi<=256: one step
    # is one sweep (126 two-site updates) through mps_dmrg, after warm-up sweeps from the Mott state
    "dmrg": dict(L=64, N=64, CHI=256, precision="fp64", start="dmrg",
                 workload="dmrg_bose_hubbard_L64_nmax4_N64_J1_U2_chi256_cutoff1e-10"),
    # two-site TDVP quench: the chi<=256 DMRG ground state of U=2 evolved with U=4, dt=0.02; one
    # step is one TDVP time step (two passes, 126 two-site updates and 124 one-site backward steps)
    "tdvp": dict(L=64, N=64, CHI=256, precision="fp64", start="dmrg",
                 workload="tdvp_bose_hubbard_L64_nmax4_N64_J1_U2to4_dt0.02_chi256_cutoff1e-10"),
    # a short chain whose bonds saturate at chi<=256 within three sweeps, for profiler captures of
    # the H_eff products at the benchmark's sector sizes
    "dmrg_mid": dict(L=12, N=12, CHI=256, precision="fp64", start="dmrg",
                     workload="dmrg_bose_hubbard_L12_nmax4_N12_J1_U2_chi256_cutoff1e-10"),
    # the same at L=24, chi<=128, for profiler captures
    "dmrg_small": dict(L=24, N=24, CHI=128, precision="fp64", start="dmrg",
                       workload="dmrg_bose_hubbard_L24_nmax4_N24_J1_U2_chi128_cutoff1e-10"),
    # boson sampling: M=100 modes, photons in modes 0..49, per-mode cutoff 4, Haar brickwork
    "boson": dict(L=100, N=50, CHI=1024, precision="fp64", start="brickwork", depth=100,
                  workload="boson_sampling_M100_photons50_d5_brickwork100_chi1024_cutoff1e-10"),
}
# FP64 peak of the GB300 CUDA cores: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (unit counts and
# the maximum clock; an FMA-chain probe, run by every bench, measures 1.19-1.26 TFLOP/s)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# fallback of the measured peaks when MEASURED_PEAKS.json is absent (one earlier GB300 measurement)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
KERNEL_BOUND = {"theta": "alu", "svd": "alu", "gemm": "alu", "select": "hbm", "lambda": "hbm",
                "tcgemm": "tensor", "shadow": "hbm",
                "scatter": "hbm", "expect": "hbm", "amplitude": "alu", "sample": "alu"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return {k: float(p[k]) for k in FALLBACK_PEAKS}, "MEASURED_PEAKS.json (measured on this pool's GB300)"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback peaks (MEASURED_PEAKS.json absent)"


def tensor_peak_tflops(precision: str, peaks: dict) -> tuple[float, str]:
    """Peak of a sector GEMM timed inside the long step: the sustained BF16 rate times the
    nominal ratio of the format (TF32 1.1 / BF16 2.25 PFLOP/s dense); BF16x3 issues three
    BF16 MMAs per product."""
    bf = peaks["bf16_tflops_sustained"]
    if precision == "tf32":
        return bf * 1.1 / 2.25, "sustained bf16 x 1.1/2.25 (nominal TF32/BF16 ratio)"
    return bf / 3.0, "sustained bf16 / 3 (three BF16 MMAs per product)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--case", default="bh128", choices=sorted(CASES))
    p.add_argument("--precision", default=None,
                   help="sector GEMMs in fp64, tf32 or bf16x3 (tensor cores); SVD and truncation stay FP64; "
                        "default: the case's (tf32 for bh128, fp64 otherwise); a comma-separated list runs each")
    p.add_argument("--max-prep", type=int, default=120)
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=1, help="steps of the end-to-end measurement (at most --steps)")
    p.add_argument("--serve", action="store_true",
                   help="serving workload instead: continuous batching vs the plain one-request-at-a-time form")
    p.add_argument("--serve-requests", type=int, default=48)
    p.add_argument("--serve-mix", default="scaled", choices=("scaled", "full"),
                   help="full: the 512-request configuration (L in {32,64,128}, chi in {64,256,1024}, 50-500 steps) "
                        "at --serve-rate requests/s, served for --serve-seconds of wall time")
    p.add_argument("--serve-rate", type=float, default=4.0)
    p.add_argument("--serve-lanes", type=int, default=2, choices=(1, 2),
                   help="serving executors run concurrently from two host threads, each on its own stream")
    p.add_argument("--serve-seconds", type=float, default=25.0,
                   help="wall-time bound of the serving sub-measurement of the main line (0: none)")
    p.add_argument("--graphs", type=int, default=1, help="capture each update call's launch phases in CUDA graphs")
    p.add_argument("--autotune", type=int, default=0,
                   help="SVD tile shape chosen per sector-size histogram (tuning runs happen before the timed steps)")
    p.add_argument("--chi-deflation", type=float, default=3e-4,
                   help="second SVD deflation level: values below this fraction of a bond's previous chi cut are "
                        "left unresolved (level / 30 when the cut is older than the previous layer; the update is redone if its cut "
                        "falls below that level / 6e-4 of it); 0: off")
    p.add_argument("--svd-mixed-min-k", type=int, default=192,
                   help="cluster SVD sectors with min(m, n) >= this start with FP32 Jacobi sweeps (0: FP64 only)")
    p.add_argument("--svd-candidate", type=int, default=-1,
                   help="force one SVD tile-shape candidate (0..11) for every update call (-1: the default rule)")
    a = p.parse_args()
    a.cfg = CASES[a.case]
    if a.precision is None:
        a.precision = a.cfg["precision"]
    if a.case != "bh128":
        a.serve_seconds = 0.0
    return a


def config_of(a, extra=None):
    c = a.cfg
    if a.case == "boson":
        out = {"workload": c["workload"] + "_" + a.precision, "model": "boson_sampling", "M": c["L"], "d": D,
               "photons": c["N"], "depth": c["depth"], "chi": c["CHI"], "cutoff": CUTOFF,
               "step": "one brickwork layer of Haar beam splitters (49 or 50 two-site updates)",
               "regime": "the brickwork from the input state; timed layers follow the layers that bring "
                         "the largest bond to chi"}
    else:
        out = {"workload": c["workload"] + "_" + a.precision, "model": "bose_hubbard", "L": c["L"], "d": D,
               "N": c["N"], "J": J, "U": U, "dt": DT, "chi": c["CHI"], "cutoff": CUTOFF,
               "step": "one Strang layer (odd dt/2, even dt, odd dt/2 in turn): all of its two-site updates",
               "regime": ("synthetic saturated chain (every inner bond at chi spread over its charges in proportion "
                          "to the Hilbert bound; seeded random complex blocks; Schmidt weights exp(-0.3 (ln k)^2), "
                          "k = 1..chi, dealt to the sectors at random, the decay of an evolved Bose-Hubbard "
                          "spectrum; not canonical)" if c["start"] == "saturated" else
                          "saturated (timed layers follow untimed Trotter steps from the Mott state until the "
                          "middle bond reaches chi)")}
    out["sector_gemms"] = a.precision
    out["svd_truncation_renorm"] = "fp64"
    out["l2"] = "inputs (site tensors) larger than L2; also flushed between timed steps (256 MiB write)"
    if extra:
        out.update(extra)
    return out


# ---------------------------------------------------------------------------
# distributed plumbing (timing only: barrier and max over ranks; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region (samples go to a temporary file)
# ---------------------------------------------------------------------------
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.fh = None

    def __enter__(self):
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", prefix="clocks_", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.fh is not None:
            self.fh.close()

    def summary(self):
        if self.proc is None or self.fh is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.fh.name) as fh:
            lines = fh.readlines()
        try:
            os.unlink(self.fh.name)
        except OSError:
            pass
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the saturated chain, and the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
_STATE = {}


def saturated_chain(cfg):
    """(lam, blocks) of the seeded synthetic saturated chain (built once per process)."""
    import workloads as W
    key = (cfg["L"], cfg["N"], cfg["CHI"], cfg.get("beta"))
    if key not in _STATE:
        _STATE[key] = W.saturated_random_state(cfg["L"], D, cfg["N"], cfg["CHI"], seed=0, beta=cfg.get("beta"))
    return _STATE[key]


def oracle_state(cfg):
    """The oracle's copy of the same chain (the generated inputs, no arithmetic)."""
    import numpy as np
    from oracle import U1MPS
    L, N = cfg["L"], cfg["N"]
    lam, blocks = saturated_chain(cfg)
    st = U1MPS(L, D, N)
    st.bond = [None] * (L + 1)
    st.lam = [None] * (L + 1)
    st.bond[0], st.bond[L] = {N: 1}, {0: 1}
    st.lam[0], st.lam[L] = {N: np.ones(1)}, {0: np.ones(1)}
    for b in range(1, L):
        st.lam[b] = {c: np.array(v) for c, v in lam[b].items()}
        st.bond[b] = {c: len(v) for c, v in lam[b].items()}
    st.B = [dict(bl) for bl in blocks]
    return st


def oracle_updates(cfg, seconds: float, max_updates: int | None = None):
    """Oracle updates of the chain's odd layer (middle bonds first, dt/2 gates) for about
    `seconds`; each update starts from the chain as generated (the sites are restored)."""
    from oracle import tebd as otebd
    L, chi = cfg["L"], cfg["CHI"]
    st = oracle_state(cfg)
    gate_of = otebd.bh_gates(L, D, J, U, DT)
    order = sorted(range(0, L - 1, 2), key=lambda s: (abs(s - (L // 2 - 1)), s))
    n, el = 0, 0.0
    for s in order * 4:
        keep = (dict(st.bond[s + 1]), dict(st.lam[s + 1]), dict(st.B[s]), dict(st.B[s + 1]))
        t0 = time.perf_counter()
        st.apply_gate2(s, gate_of(s, 0.5), chi, CUTOFF)
        el += time.perf_counter() - t0
        st.bond[s + 1], st.lam[s + 1], st.B[s], st.B[s + 1] = keep
        n += 1
        if (max_updates is not None and n >= max_updates) or el >= seconds:
            break
    return n, el


def blas_threads() -> int:
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count() or 1


def oracle_single_thread(case: str, seconds: float):
    """The same sample in a fresh process with one BLAS thread (the thread count is fixed
    when numpy loads, so it needs a process of its own)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "n, el = bench.oracle_updates(bench.CASES[%r], %r); print(json.dumps([n, el]))" % (ROOT, case, seconds))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        n, el = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": n / el, "unit": "updates/s", "cores": 1, "sample": f"{n} oracle updates ({el:.1f} s)"}
    except Exception as e:  # pragma: no cover - reported, not fatal
        return {"value": None, "error": str(e)[:200]}


def run_reference(args, world, rank):
    """The float64 oracle on the host cores, on the same chain and metric: each step is a
    bounded sample of the configuration's updates (two updates of the odd layer)."""
    if rank != 0:
        return
    if args.case != "bh128":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the default configuration"}))
        return
    per_step = 2
    times = []
    for i in range(args.warmup + args.steps):
        n, el = oracle_updates(args.cfg, 1e9, max_updates=per_step)
        if i >= args.warmup:
            times.append(el)
    tot = sum(times)
    value = per_step * len(times) / tot
    cores = blas_threads()
    sample = (f"{per_step} oracle updates per step on the odd layer (middle bonds first) of the saturated "
              f"synthetic chi={args.cfg['CHI']} chain")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, {"oracle": "float64 numpy/scipy (zgesvd)"}),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
def build_workload(args, m, W, stream, prec):
    """The state on the device and a step function (returns the updates it made)."""
    import numpy as np
    cfg = args.cfg
    L, CHI = cfg["L"], cfg["CHI"]

    def new_psi(occ, precision):
        p = m.MPS(D, occ, CHI, precision=precision, stream=stream.cuda_stream)
        p.set_graphs(bool(args.graphs))
        p.set_autotune(bool(args.autotune))
        p.set_chi_deflation(args.chi_deflation)
        return p

    prep = 0
    if cfg["start"] == "brickwork":
        layers = W.brickwork_pairs(L, cfg["depth"])
        ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=0)
        first = np.cumsum([0] + [len(x) for x in layers])
        psi = new_psi(W.single_photon_occupations(L, cfg["N"]), prec)
        pos = [0]

        def step():                      # the next brickwork layer (wrapping round after the last)
            li = pos[0] % len(layers)
            sites = layers[li]
            gs = [m.models.flatten(m.models.beam_splitter_gate(*ang[first[li] + k], D)) for k in range(len(sites))]
            psi.apply_layer(sites, gs, CHI, CUTOFF)
            pos[0] += 1
            return len(sites)

        while prep < args.max_prep and max(sum(psi.bond_dims(b).values()) for b in range(L + 1)) < CHI:
            step()
            prep += 1
        return psi, step, prep

    gates = m.tebd.GateTable("bh", L, D, DT, J=J, U=U)
    if cfg["start"] == "saturated":
        psi = new_psi(W.mott_occupations(L), prec)
        lam, blocks = saturated_chain(cfg)
        for b in range(1, L):
            psi.set_bond(b, lam[b])
        for s_ in range(L):
            psi.set_site(s_, blocks[s_])
    else:
        psi = new_psi(W.mott_occupations(L), m.MPS_FP64)
        while prep < args.max_prep and sum(psi.bond_dims(L // 2).values()) < CHI:
            m.tebd.trotter_step(psi, gates, CHI, CUTOFF)
            prep += 1
        if prec != m.MPS_FP64:
            # the same saturated state, continued with the sector GEMMs on the tensor cores
            low = new_psi(W.mott_occupations(L), prec)
            for b in range(1, L):
                low.set_bond(b, psi.bond(b))
            for s_ in range(L):
                low.set_site(s_, psi.site(s_))
            psi.close()
            psi = low
    layers = m.tebd.strang_layers(L)
    pos = [0]

    def step():                          # the next Strang layer: odd dt/2, even dt, odd dt/2, ...
        sites, f = layers[pos[0] % 3]
        psi.apply_layer(sites, [gates(s_, f) for s_ in sites], CHI, CUTOFF)
        pos[0] += 1
        return len(sites)

    return psi, step, prep


def oracle_dmrg_sample(cfg, seconds: float, tdvp: bool = False):
    """The oracle's DMRG on the same chain and schedule from the Mott state, timed for about
    `seconds` of local steps.  Its bonds are still below chi during the sample, so the rate is
    an upper bound on the oracle's rate at saturation.  For TDVP the sample is the oracle's TDVP
    (forward steps and the backward site steps between them) on the same quench, from the Mott
    state."""
    from oracle import U1MPS, dmrg as odmrg
    import workloads as W
    L, CHI = cfg["L"], cfg["CHI"]
    dm = odmrg.DMRG(U1MPS.product(D, W.mott_occupations(L)), odmrg.bh_bonds(L, D, J, 2.0 * U if tdvp else U))
    order = [(s_, True) for s_ in range(L - 1)] + [(s_, False) for s_ in range(L - 2, -1, -1)]
    t0 = time.perf_counter()
    n = 0
    half = 0.5 * DT

    def forward(s_, lay, dim, X0):
        v0 = dm._flat(lay, X0)
        return None, dm._expm_apply(lambda x: dm._flat(lay, dm._apply(s_, lay, dm._unflat(lay, x))), v0, -1j * half)
    while time.perf_counter() - t0 < seconds:
        s_, right = order[n % len(order)]
        if tdvp:
            dm.step(s_, CHI, CUTOFF, right, local=forward)
            if right and s_ < L - 2:
                dm._backward(s_ + 1, half)
            elif not right and s_ > 0:
                dm._backward(s_, half)
        else:
            dm.step(s_, CHI, CUTOFF, right)
        n += 1
    el = time.perf_counter() - t0
    largest = max(sum(b.values()) for b in dm.st.bond)
    return {"value": n / el, "unit": "updates/s", "cores": blas_threads(), "kind": "oracle",
            "sample": (f"the first {n} local steps ({el:.1f} s) of the oracle's {'TDVP' if tdvp else 'DMRG'} on the same "
                       f"chain from the Mott state (largest bond reached {largest} < chi: an upper bound on its rate "
                       f"at saturation)")}


def run_dmrg_case(args, world, rank, local):
    """Two-site DMRG sweeps (mps_dmrg) on the Bose-Hubbard chain: each timed step is one call of
    one sweep (2 (L-1) two-site updates, then the canonical form), after warm-up sweeps from
    the Mott state at the same chi.  The oracle's DMRG gives the CPU baseline on the same
    chain (a bounded number of local steps)."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import paper_2303_11409_gb300 as m
    import workloads as W
    cfg = args.cfg
    L, CHI = cfg["L"], cfg["CHI"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    fp64_measured = m.fp64_peak_probe(stream.cuda_stream)
    terms = m.models.chain_bond_terms("bh", L, D, J=J, U=U)
    tdvp = args.case == "tdvp"
    quench = m.models.chain_bond_terms("bh", L, D, J=J, U=2.0 * U) if tdvp else None
    psi = m.MPS(D, W.mott_occupations(L), CHI, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        psi.dmrg(terms, 1, CHI, CUTOFF)
    print(f"[bench] {args.warmup} warm-up sweeps in {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
    psi.set_profiling(True)
    torch.cuda.synchronize()
    launches0 = m.launch_count()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kinds = {}
    energies = []
    n_upd = 0
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            e = psi.tdvp(quench, 1, DT, CHI, CUTOFF) if tdvp else psi.dmrg(terms, 1, CHI, CUTOFF)
            ev[k][1].record(stream)
            n_upd += 2 * (L - 1)
            energies.append(float(e[-1]))
            for name, v in psi.dmrg_stats().items():
                if isinstance(v, dict):
                    a = kinds.setdefault(name, {"launches": 0, "ms": 0.0, "flops": 0.0})
                    for kk in a:
                        a[kk] += v[kk]
        torch.cuda.synchronize()
    barrier(world)
    launches = m.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * n_upd / (total_ms / 1000.0)
    largest = max(sum(psi.bond_dims(b).values()) for b in range(L + 1))
    tot = max(sum(v["ms"] for v in kinds.values()), 1e-12)
    hv = kinds["heff"]
    achieved = hv["flops"] / (hv["ms"] / 1000.0) / 1e9 if hv["ms"] > 0 else None
    roofline = {"kernel": "heff (sumprod_kernel: H_eff products)", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS if achieved else None, "traffic": None,
                "traffic_note": "null: no ncu DRAM capture of this kernel at this configuration",
                "per_launch": {"flops": hv["flops"] / max(hv["launches"], 1), "ms": hv["ms"] / max(hv["launches"], 1)},
                "peak_source": "FP64 CUDA-core peak from unit counts and the 2070 MHz max clock",
                "fp64_peak_measured_gflops": fp64_measured,
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": v["ms"] / tot,
                                "gflops": v["flops"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] > 0 else None}
                            for k, v in kinds.items()}}
    # e2e: the same call with host-resident bond terms and energies (mps_dmrg is host-in,
    # host-out), timed on the host clock
    t0 = time.perf_counter()
    if tdvp:
        psi.tdvp(quench, 1, DT, CHI, CUTOFF)
    else:
        psi.dmrg(terms, 1, CHI, CUTOFF)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    glen = m.gate_length(D)
    e2e = {"value": world * 2 * (L - 1) / e2e_s, "unit": "updates/s", "steps": 1,
           "h2d_bytes_per_step": int((L - 1) * glen * 16), "d2h_bytes_per_step": int(2 * (L - 1) * 8),
           "what": ("one time step through MPS.tdvp (mps_tdvp)" if tdvp else "one sweep through MPS.dmrg (mps_dmrg)")
                   + " with host bond terms, energies read back"}
    psi.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_dmrg_sample(cfg, args.cpu_seconds, tdvp)
    if rank == 0:
        line = {"metric": "two-site TDVP updates/s" if tdvp else "two-site DMRG updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": cfg["workload"], "model": "bose_hubbard", "L": L, "d": D, "N": cfg["N"],
                           "J": J, "U": U, "chi": CHI, "cutoff": CUTOFF,
                           "step": (f"one mps_tdvp call of one time step dt={DT} of the U={2.0 * U} quench ({2 * (L - 1)} "
                                    f"two-site and {2 * (L - 2)} one-site updates, then the canonical form)" if tdvp else
                                    f"one mps_dmrg call of one sweep ({2 * (L - 1)} two-site updates, then the canonical form)"),
                           "lanczos": ("Krylov 24, exponential error estimate 1e-12" if tdvp else
                                       "Krylov 24, residual tolerance 1e-12 |E|"),
                           "largest_bond_dim": largest,
                           "l2": "no flush (one sweep streams the environments and Krylov vectors of 63 bonds)"},
                "energy_per_site": energies[-1] / L, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(), "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import paper_2303_11409_gb300 as m
    import workloads as W

    peaks, peak_src = measured_peaks()
    # a stream of its own: the legacy default stream cannot be captured into CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    fp64_measured = m.fp64_peak_probe(stream.cuda_stream)
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[args.precision]
    if args.svd_candidate >= 0:
        m.autotune_force(args.svd_candidate)
    m.svd_mixed_min_k(args.svd_mixed_min_k)
    t_prep = time.perf_counter()
    psi, step, prep = build_workload(args, m, W, stream, prec)
    L = args.cfg["L"]
    print(f"[bench] workload ready in {time.perf_counter() - t_prep:.1f} s", file=sys.stderr, flush=True)

    for _ in range(args.warmup):
        step()
    # tile shapes are tuned during the preparation and the warm-up steps; a sector-size
    # histogram first seen inside the timed steps keeps the default shape
    m.autotune_freeze(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    psi.reset_kernel_stats()
    psi.set_profiling(True)
    launches0 = m.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n_upd = 0
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.random_(0, 255)
            ev[k][0].record(stream)
            n_upd += step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = m.launch_count() - launches0
    graph_stats = psi.graph_stats()
    deflation = psi.deflation_stats()
    psi.set_profiling(False)
    ks = psi.kernel_stats()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * n_upd / (total_ms / 1000.0)
    largest = max(sum(psi.bond_dims(b).values()) for b in range(L + 1))

    # roofline of the dominant kernel (largest device time in the timed region)
    tot_ms = max(sum(v["ms"] for v in ks.values()), 1e-12)
    dom = max(ks, key=lambda k: ks[k]["ms"])
    kd = ks[dom]
    per_launch_ms = kd["ms"] / max(kd["launches"], 1)
    if KERNEL_BOUND[dom] == "hbm":
        achieved = kd["bytes"] / (kd["ms"] / 1000.0) / 1e9
        peak, unit = peaks["hbm_gbs"], "GB/s"
        src = peak_src + " hbm_gbs"
    else:
        achieved = kd["flops"] / (kd["ms"] / 1000.0) / 1e9
        peak, unit = FP64_PEAK_GFLOPS, "GFLOP/s"
        src = "FP64 CUDA-core peak from unit counts and the 2070 MHz max clock (152 SMs x 2 FMA/clk x 2 flop)"
    roofline = {"kernel": dom, "bound": KERNEL_BOUND[dom], "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None,
                "traffic_note": "null: no ncu DRAM capture of this kernel at this configuration's current build",
                "traffic_small_case": None,
                "per_launch": {"flops" if unit == "GFLOP/s" else "bytes":
                               (kd["flops"] if unit == "GFLOP/s" else kd["bytes"]) / max(kd["launches"], 1),
                               "ms": per_launch_ms},
                "peak_source": src, "fp64_peak_measured_gflops": fp64_measured,
                "frac_of_measured_fp64": achieved / fp64_measured if unit == "GFLOP/s" else None,
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": v["ms"] / tot_ms}
                            for k, v in ks.items() if v["launches"]}}
    if dom == "svd":
        # ncu DRAM bytes of the cluster SVD on the saturated L=24, chi<=1024 chain (bench.py --case
        # small_tf32, the first cluster-SVD launch of the layer): 9.05 + 28.21 GB for a launch of
        # 3.21e11 nominal flops.  The write-back of staged column blocks grows with the sweep work,
        # so the figure is scaled to this launch by its nominal flops.
        small_bytes, small_flops = 9.05e9 + 28.21e9, 3.2139e11
        flops_launch = kd["flops"] / max(kd["launches"], 1)
        roofline["traffic"] = small_bytes * flops_launch / small_flops
        roofline["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of the small-case capture "
                                    "(L=24, chi<=1024), scaled to this launch by nominal flops; the column "
                                    "blocks written back after every block round, about 1% of the DRAM bandwidth")
        roofline["traffic_small_case"] = {"bytes": small_bytes, "nominal_flops": small_flops}
    if args.precision != "fp64":
        # the tensor-core sector GEMMs (the products of the Theta' build and of the reassembly,
        # one TMA-fed kernel) against the format's peak, and against the HBM roofline of their
        # algorithmic bytes (shadow operands read, products written)
        tpk, tsrc = tensor_peak_tflops(args.precision, peaks)
        v = ks["tcgemm"]
        tc = {}
        if v["launches"] and v["ms"] > 0:
            sec = v["ms"] / 1000.0
            tf = v["flops"] / sec / 1e12
            ai = v["flops"] / max(v["bytes"], 1.0)
            attainable = min(tpk, ai * peaks["hbm_gbs"] / 1000.0)
            tc = {"kernel": "tma_zgemm_kernel", "achieved": tf, "unit": "TFLOP/s", "peak": tpk, "frac": tf / tpk,
                  "flops_per_launch": v["flops"] / v["launches"], "ms_per_launch": v["ms"] / v["launches"],
                  "launches": v["launches"], "bytes_per_launch": v["bytes"] / v["launches"],
                  "arithmetic_intensity_flop_per_byte": ai, "attainable_tflops": attainable,
                  "frac_of_attainable": tf / attainable, "achieved_gbs": v["bytes"] / sec / 1e9,
                  "share_of_device_time": v["ms"] / tot_ms}
        roofline["tensor_gemms"] = tc
        roofline["tensor_peak_source"] = peak_src + ": " + tsrc

    # e2e: the public API with host buffers (gate blocks and descriptors go up, kept counts and
    # one <n_i> come back), host wall clock
    glen = m.gate_length(D)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_upd = 0
    for _ in range(e2e_steps):
        e2e_upd += step()
        psi.expect(L // 2, np.arange(D, dtype=np.float64))
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, world)
    per_step = e2e_upd / e2e_steps
    e2e = {"value": world * e2e_upd / e2e_s, "unit": "updates/s", "steps": e2e_steps,
           "h2d_bytes_per_step": int(per_step * glen * 16),
           "d2h_bytes_per_step": int(per_step * 8 + 8),
           "what": "Strang layers through MPS.apply_layer (mps_apply_layer) with host gate buffers, "
                   "plus one <n_i> read back per step"}
    psi.close()
    del flush

    serving = None
    if args.serve_seconds > 0:
        serving = serving_sample(args, m, W, stream, prec)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.case == "bh128":
        n, el = oracle_updates(args.cfg, args.cpu_seconds)
        cpu = {"value": n / el, "unit": "updates/s", "cores": blas_threads(), "kind": "oracle",
               "sample": (f"{n} oracle updates ({el:.1f} s) of the odd layer, middle bonds first, on the same "
                          f"saturated chi={args.cfg['CHI']} chain"),
               "single_thread": oracle_single_thread(args.case, max(5.0, args.cpu_seconds / 2))}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else f"{args.precision}+f64", "data": "synthetic",
                "config": config_of(args, {"prep_steps": prep, "largest_bond_dim": largest, "updates_timed": n_upd,
                                           "parallelism": "replicas" if world > 1 else "single",
                                           "cuda_graphs": bool(args.graphs), "autotune": bool(args.autotune)}),
                "graphs": graph_stats, "autotune": {**m.autotune_stats(), "table": m.autotune_table()},
                "svd_deflation": deflation, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "serving": serving, "gpu_launches": launches, "clocks": clk.summary(),
                "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
SERVE_MIX = dict(L_choices=(16, 32), chi_choices=(32, 64, 128), steps_range=(5, 40))


def serving_sample(args, m, W, stream, prec):
    """Bounded p50/p99 measurement for the main line: requests of the scaled serving mix
    through the continuous-batching server at --precision, Poisson arrivals at 0.8 x the
    capacity measured on the same requests queued at once, stopped after --serve-seconds
    of arrivals (requests arriving later are not sent)."""
    n = 24
    raw = W.serving_requests(n, seed=1, rate_hz=1.0, **SERVE_MIX)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=0.0)
            for r in raw]
    srv = m.serve.Server(budget_bytes=64 << 30, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=bool(args.graphs), lanes=args.serve_lanes)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    cap_s = time.perf_counter() - t0
    srv.close()
    capacity = sum(r.updates for r in res) / cap_s
    rate = 0.8 * len(reqs) / cap_s
    raw = W.serving_requests(n, seed=1, rate_hz=rate, **SERVE_MIX)
    raw = [r for r in raw if r["arrival"] <= args.serve_seconds]
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=r["arrival"])
            for r in raw]
    srv = m.serve.Server(budget_bytes=64 << 30, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=bool(args.graphs), lanes=args.serve_lanes)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    srv.close()
    s = m.serve.summarize(res, wall)
    return {"p50_latency_s": s["p50_latency_s"], "p99_latency_s": s["p99_latency_s"], "requests": s["requests"],
            "updates_per_s_under_load": s["updates_per_s"], "capacity_updates_per_s": capacity,
            "arrival_rate_hz": rate, "lanes": args.serve_lanes,
            "mix": {k: list(v) for k, v in SERVE_MIX.items()}, "precision": args.precision,
            "what": "scaled serving mix (xxz / bose-hubbard quenches), Poisson arrivals at 0.8 x capacity"}


def run_serving_full(args, world, rank, local):
    """The full serving configuration, bounded in wall time: 512 requests (XXZ or Bose-Hubbard
    quenches, L in {32, 64, 128}, chi in {64, 256, 1024}, 50-500 Trotter steps) arriving as a
    Poisson process of --serve-rate requests/s, served by continuous batching (two lanes) for
    --serve-seconds.  Completed requests give p50 / p99 latency (the short ones complete first,
    so these describe the completed part of the mix); all requests' updates give the served
    throughput under load."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import paper_2303_11409_gb300 as m
    import workloads as W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec_name = args.precision.split(",")[0]
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[prec_name]
    raw = W.serving_requests(512, seed=rank, rate_hz=args.serve_rate)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=r["arrival"])
            for r in raw]
    budget = 120 << 30
    srv = m.serve.Server(budget_bytes=budget, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=bool(args.graphs), lanes=args.serve_lanes)
    launches0 = m.launch_count()
    t0 = time.perf_counter()
    res = srv.run(reqs, deadline=args.serve_seconds)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    srv.close()
    ups = sum(r.updates for r in res) + srv.unfinished_updates
    lat = np.array([r.latency for r in res]) if res else np.zeros(1)
    if rank == 0:
        line = {"metric": "serving two-site updates/s (full request mix, bounded run)", "value": ups / wall,
                "unit": "updates/s", "n_gpus": world, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec_name == "fp64" else f"{prec_name}+f64",
                "data": "synthetic", "wall_s": wall, "requests_arrived": sum(1 for r in raw if r["arrival"] <= wall),
                "requests_completed": len(res), "requests_unfinished": srv.unfinished,
                "p50_latency_completed_s": float(np.percentile(lat, 50)),
                "p99_latency_completed_s": float(np.percentile(lat, 99)),
                "max_active": srv.max_active_seen, "max_bytes": srv.max_bytes_seen,
                "gpu_launches": m.launch_count() - launches0,
                "config": {"workload": "serving_mix_full_512", "rate_hz": args.serve_rate,
                           "seconds": args.serve_seconds, "lanes": args.serve_lanes, "budget_bytes": budget,
                           "max_slots": 64, "served_precision": prec_name, "cuda_graphs": bool(args.graphs),
                           "latency": "arrival to result, requests completed within the bounded run"}}
        print(json.dumps(line), flush=True)


def run_serving(args, world, rank, local):
    """Serving: Poisson arrivals of mixed XXZ / Bose-Hubbard quenches through the
    continuous-batching server, next to the plain form (each request alone, in turn).

    Reported: the served capacity (all requests queued at once) against the plain
    form's, and p50/p99 latency under Poisson arrivals at 0.8 x the served capacity.
    The request mix is the serving configuration scaled down so that the whole run
    takes minutes: L in {16, 32}, chi in {32, 64, 128}, 5..40 Trotter steps (the full
    mix has L up to 128, chi up to 1024 and up to 500 steps per request).  The plain
    form is FP64 with direct launches; the served form runs at --precision (sector GEMMs
    on the tensor cores for tf32 / bf16x3, SVD and truncation FP64) with CUDA graphs
    (--graphs), and the largest deviation of its <n_i> from the plain FP64 results is
    reported beside the speed-up.
    """
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import paper_2303_11409_gb300 as m
    import workloads as W
    stream = torch.cuda.Stream()          # capturable (the legacy default stream is not)
    torch.cuda.set_stream(stream)
    prec_name = args.precision.split(",")[0]
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[prec_name]
    graphs = bool(args.graphs)
    raw = W.serving_requests(args.serve_requests, seed=rank, rate_hz=1.0, **SERVE_MIX)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=0.0)
            for r in raw]
    budget = 64 << 30
    t0 = time.perf_counter()
    plain_updates = 0
    plain_obs = {}
    for q in reqs:
        srv = m.serve.Server(budget_bytes=budget, max_slots=1, stream=stream.cuda_stream)
        res = srv.run([q])
        srv.close()
        plain_updates += res[0].updates
        plain_obs[q.id] = res[0].observables
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_rate = plain_updates / plain_s
    srv = m.serve.Server(budget_bytes=budget, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=graphs, lanes=args.serve_lanes)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    cap_s = time.perf_counter() - t0
    srv.close()
    served_cap = sum(r.updates for r in res) / cap_s
    obs_err = max(float(np.max(np.abs(r.observables - plain_obs[r.id]))) for r in res)
    req_rate = 0.8 * len(reqs) / cap_s
    raw = W.serving_requests(args.serve_requests, seed=rank, rate_hz=req_rate, **SERVE_MIX)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=r["arrival"])
            for r in raw]
    srv = m.serve.Server(budget_bytes=budget, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=graphs, lanes=args.serve_lanes)
    launches0 = m.launch_count()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    gstats = srv.executor.graph_stats()
    srv.close()
    summ = m.serve.summarize(res, wall)
    if rank == 0:
        line = {"metric": "serving two-site updates/s (p50/p99 request latency)", "value": served_cap,
                "unit": "updates/s", "n_gpus": world, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec_name == "fp64" else f"{prec_name}+f64",
                "data": "synthetic",
                "p50_latency_s": summ["p50_latency_s"], "p99_latency_s": summ["p99_latency_s"],
                "requests": len(res), "updates": summ["updates"], "loaded_wall_s": wall,
                "loaded_updates_per_s": summ["updates_per_s"],
                "plain_updates_per_s": plain_rate, "served_over_plain": served_cap / plain_rate,
                "max_observable_error_vs_plain_fp64": obs_err,
                "arrival_rate_hz": req_rate, "max_active_under_load": srv.max_active_seen,
                "gpu_launches": m.launch_count() - launches0, "graphs": gstats,
                "config": {"workload": "serving_mix_scaled", "requests": len(reqs),
                           **{k: list(v) for k, v in SERVE_MIX.items()},
                           "models": "xxz Delta~U[0,2] (Neel) / bh U~U[1,10] J=1 (Mott), 50/50",
                           "value": "served capacity (all requests queued at t=0, merged launches)",
                           "latency": "Poisson arrivals at 0.8 x the served capacity",
                           "plain": "FP64, each request alone, one after another, direct launches",
                           "served_precision": prec_name, "cuda_graphs": graphs, "budget_bytes": budget,
                           "lanes": args.serve_lanes,
                           "max_slots": 64}}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.serve and args.serve_mix == "full":
        run_serving_full(args, world, rank, local)
    elif args.serve:
        run_serving(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    elif args.case in ("dmrg", "dmrg_small", "dmrg_mid", "tdvp"):
        run_dmrg_case(args, world, rank, local)
    else:
        precisions = args.precision.split(",")
        for p_ in precisions:
            if p_ not in ("fp64", "tf32", "bf16x3"):
                raise SystemExit(f"unknown precision {p_}")
        for p_ in precisions:
            args.precision = p_
            run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
