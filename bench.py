#!/usr/bin/env python
"""Two-site TEBD update throughput of the U(1) block-sparse MPS on one GB300.

Workload: Bose-Hubbard chain L=64, local cutoff n_max=4 (d=5), N=64 bosons
(unit filling), J=1, U=2, Mott initial state, second-order Trotter steps of
dt=0.02, chi<=512, cutoff 1e-10, FP64.  A "step" is one Trotter step: three
layers (odd dt/2, even dt, odd dt/2), 95 two-site updates, each running the
whole update path (planner, Theta build, per-sector SVD, global top-chi,
reassembly, renormalisation).  The timed steps are taken in the saturated
regime: the chain is first evolved from the Mott state by the same Trotter
steps until its middle bond reaches chi (untimed), then W warm-up and K timed
steps follow.  The L2 cache is flushed (256 MiB write) between timed steps,
outside the timed events.

Prints one JSON line (rank 0).  --impl reference times the float64 oracle on the
host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L, D, N_PART, J, U, DT, CHI, CUTOFF = 64, 5, 64, 1.0, 2.0, 0.02, 512, 1e-10
UPDATES_PER_STEP = 32 + 31 + 32
METRIC = "two-site updates/s"
WORKLOAD = "bose_hubbard_L64_nmax4_N64_J1_U2_dt0.02_chi512_cutoff1e-10_fp64"
# --case small: the same model on L=32, chi=512 (half the chain, same sector sizes), for profiler captures
SMALL = dict(L=32, N=32, CHI=512, WORKLOAD="bose_hubbard_L32_nmax4_N32_J1_U2_dt0.02_chi512_cutoff1e-10_fp64")
# --case bh128: Bose-Hubbard L=128, N=128, chi<=2048 (the mixed-precision configuration), timed on
# Strang layers of Bose-Hubbard gates applied to a synthetic saturated chain (evolving the Mott
# state to saturation at chi=2048 would take far longer than a benchmark run)
BH128 = dict(L=128, N=128, CHI=2048, SAMPLE=8,
             WORKLOAD="bose_hubbard_L128_nmax4_N128_J1_U2_dt0.02_chi2048_cutoff1e-10_fp64")
_BH128_STATE = None
# --case boson: boson sampling, M=100 modes, single photons in modes 0..49, per-mode cutoff 4
# (d=5), brickwork of seeded Haar beam splitters, chi<=1024; a step is one brickwork layer
BOSON = dict(L=100, N=50, CHI=1024, DEPTH=100,
             WORKLOAD="boson_sampling_M100_photons50_d5_brickwork100_chi1024_cutoff1e-10_fp64")
# FP64 peak of the GB300 CUDA cores: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz.
# (An FMA-chain probe measured 1.195 TFLOP/s, i.e. 2 FMA/clk/SM at the clock it ran.)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# DRAM bytes per launch of the SVD phase of a saturated layer of this workload (all SVD kernels
# of one layer), from an ncu capture of dram__bytes_read.sum + dram__bytes_write.sum with the
# default tile shape; emptied whenever those kernels change.
NCU_TRAFFIC = {"svd": 22.57e9}
# Tensor peaks of the reduced-precision GEMMs, from the measured dense BF16 rate times the nominal
# ratio of the format (TF32 1.1 / BF16 2.25 PFLOP/s dense); BF16x3 issues three BF16 MMAs per product.
BF16_MEASURED_TFLOPS = 1913.8
TENSOR_PEAK_TFLOPS = {"tf32": BF16_MEASURED_TFLOPS * 1.1 / 2.25, "bf16x3": BF16_MEASURED_TFLOPS / 3.0}
KERNEL_BOUND = {"theta": "alu", "svd": "alu", "gemm": "alu", "select": "hbm", "lambda": "hbm",
                "scatter": "hbm", "expect": "hbm", "amplitude": "alu"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--max-prep", type=int, default=120)
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--serve", action="store_true",
                   help="serving workload instead: continuous batching vs the plain one-request-at-a-time form")
    p.add_argument("--serve-requests", type=int, default=48)
    p.add_argument("--case", default="full", choices=["full", "small", "bh128", "boson"],
                   help="full: the benchmark workload; small: L=32, chi=512 (for profiler captures); "
                        "bh128: L=128, chi=2048; boson: boson sampling M=100, chi=1024")
    p.add_argument("--precision", default="fp64",
                   help="sector GEMMs in fp64 (default), tf32 or bf16x3 (tensor cores); SVD and truncation stay "
                        "FP64; a comma-separated list runs each in turn from the same start state")
    p.add_argument("--graphs", type=int, default=1, help="capture each update call's launch phases in CUDA graphs")
    p.add_argument("--autotune", type=int, default=0,
                   help="SVD tile shape chosen per sector-size histogram (tuning runs happen before the timed steps)")
    a = p.parse_args()
    global L, N_PART, CHI, WORKLOAD, UPDATES_PER_STEP
    if a.case != "full":
        c = {"small": SMALL, "bh128": BH128, "boson": BOSON}[a.case]
        L, N_PART, CHI, WORKLOAD = c["L"], c["N"], c["CHI"], c["WORKLOAD"]
        UPDATES_PER_STEP = (L // 2) + (L - 1) // 2 + (L // 2)
        a.no_cpu_baseline = True
    if a.case == "bh128":
        UPDATES_PER_STEP = BH128["SAMPLE"]
    return a


def config(extra=None, case="full"):
    if case == "boson":
        c = {"workload": WORKLOAD, "model": "boson_sampling", "M": L, "d": D, "photons": N_PART,
             "depth": BOSON["DEPTH"], "chi": CHI, "cutoff": CUTOFF,
             "step": "one brickwork layer of Haar beam splitters (49 or 50 two-site updates)",
             "regime": "the brickwork from the input state; timed layers follow the layers that bring the largest bond to chi"}
    else:
        c = {"workload": WORKLOAD, "model": "bose_hubbard", "L": L, "d": D, "N": N_PART, "J": J, "U": U,
             "dt": DT, "chi": CHI, "cutoff": CUTOFF, "updates_per_step": UPDATES_PER_STEP,
             "regime": ("synthetic saturated chain (every inner bond at chi spread over its charges in proportion "
                        "to the Hilbert bound, random blocks, not canonical); a timed step is the 8 central updates "
                        "of the odd (dt/2) layer, a bounded sample of the 127 updates of a Strang layer"
                        if case == "bh128" else
                        "saturated (timed steps follow untimed Trotter steps from the Mott state until the middle "
                        "bond reaches chi)")}
    c["l2"] = "flushed between timed steps (256 MiB device write outside the timed events)"
    if extra:
        c.update(extra)
        if extra.get("precision", "fp64") != "fp64":
            c["workload"] = WORKLOAD.replace("_fp64", "_" + extra["precision"])
    return c


# ---------------------------------------------------------------------------
# distributed plumbing (timing only: barrier and max over ranks; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
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
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
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
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
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
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(seconds: float, max_updates: int | None = None):
    """Oracle updates of the odd layer on a saturated synthetic chain, for about `seconds`."""
    from oracle import synth, tebd as otebd
    import workloads as W
    st = synth.random_state(L, D, N_PART, CHI, seed=0, occ=W.mott_occupations(L))
    gate_of = otebd.bh_gates(L, D, J, U, DT)
    odd = list(range(0, L - 1, 2))
    order = sorted(odd, key=lambda s: (abs(s - (L // 2 - 1)), s))     # middle bonds first
    n, t0 = 0, time.perf_counter()
    for s in order * 4:
        st.apply_gate2(s, gate_of(s, 0.5), CHI, CUTOFF)
        n += 1
        el = time.perf_counter() - t0
        if (max_updates is not None and n >= max_updates) or el >= seconds:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))
    return n, el, cores


def run_reference(args, world, rank):
    if rank != 0:
        return
    per_step = 4
    times = []
    for i in range(args.warmup + args.steps):
        n, el, cores = oracle_sample(1e9, max_updates=per_step)
        if i >= args.warmup:
            times.append(el)
    tot = sum(times)
    value = per_step * len(times) / tot
    sample = (f"{per_step} oracle updates per step on the odd layer (middle bonds first) of a saturated "
              f"synthetic chi={CHI} chain (random blocks at Hilbert-proportional sector dims)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config({"oracle": "float64 numpy/scipy (zgesvd)"}),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    global _BH128_STATE
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import paper_2303_11409_gb300 as m
    import workloads as W

    # a stream of its own: the legacy default stream cannot be captured into CUDA graphs
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    fp64_measured = m.fp64_peak_probe(stream.cuda_stream)
    prec = {"fp64": m.MPS_FP64, "tf32": m.MPS_TF32, "bf16x3": m.MPS_BF16X3}[args.precision]

    def new_psi(occ, precision):
        p = m.MPS(D, occ, CHI, precision=precision, stream=stream.cuda_stream)
        p.set_graphs(bool(args.graphs))
        p.set_autotune(bool(args.autotune))
        return p

    prep = 0
    if args.case == "boson":
        layers = W.brickwork_pairs(L, BOSON["DEPTH"])
        ang = W.haar_beam_splitter_angles(sum(map(len, layers)), seed=0)
        first = np.cumsum([0] + [len(x) for x in layers])
        psi = new_psi(W.single_photon_occupations(L, N_PART), prec)
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
    else:
        gates = m.tebd.GateTable("bh", L, D, DT, J=J, U=U)
        if args.case == "bh128":
            # a synthetic saturated chain (Hilbert-proportional sector sizes, random blocks) loaded
            # through mps_set_bond / mps_set_site, at the run's precision
            psi = new_psi(W.mott_occupations(L), prec)
            if _BH128_STATE is None:
                _BH128_STATE = W.saturated_random_state(L, D, N_PART, CHI, seed=0)
            lam, blocks = _BH128_STATE
            for b in range(1, L):
                psi.set_bond(b, lam[b])
            for s_ in range(L):
                psi.set_site(s_, blocks[s_])
        else:
            psi = new_psi(W.mott_occupations(L), m.MPS_FP64)
            while prep < args.max_prep and sum(psi.bond_dims(L // 2).values()) < CHI:
                m.tebd.trotter_step(psi, gates, CHI, CUTOFF)
                prep += 1
            if args.precision != "fp64":
                # the same saturated state, continued with the sector GEMMs on the tensor cores
                low = new_psi(W.mott_occupations(L), prec)
                for b in range(1, L):
                    low.set_bond(b, psi.bond(b))
                for s_ in range(L):
                    low.set_site(s_, psi.site(s_))
                psi.close()
                psi = low

        if args.case == "bh128":
            sample = list(range(L // 2 - BH128["SAMPLE"], L // 2 + BH128["SAMPLE"], 2))

            def step():                  # the central updates of the odd (dt/2) layer
                t0 = time.perf_counter()
                psi.apply_layer(sample, [gates(s_, 0.5) for s_ in sample], CHI, CUTOFF)
                print(f"{len(sample)} updates: {time.perf_counter() - t0:.2f} s", file=sys.stderr, flush=True)
                return len(sample)
        else:
            def step():
                m.tebd.trotter_step(psi, gates, CHI, CUTOFF)
                return UPDATES_PER_STEP

    for _ in range(args.warmup):
        step()
    # tile shapes are tuned during the evolution to saturation and the warm-up steps; a
    # sector-size histogram first seen inside the timed steps keeps the default shape
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
    mid_dims = max(sum(psi.bond_dims(b).values()) for b in range(L + 1))

    # roofline of the dominant kernel (largest device time in the timed region)
    dom = max(ks, key=lambda k: ks[k]["ms"])
    kd = ks[dom]
    if KERNEL_BOUND[dom] == "hbm":
        achieved = kd["bytes"] / (kd["ms"] / 1000.0) / 1e9
        peak, unit, traffic_unit = 6790.3, "GB/s", kd["bytes"] / max(kd["launches"], 1)
    else:
        achieved = kd["flops"] / (kd["ms"] / 1000.0) / 1e9
        peak, unit = FP64_PEAK_GFLOPS, "GFLOP/s"
    roofline = {"kernel": dom, "bound": KERNEL_BOUND[dom], "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak,
                "traffic": (NCU_TRAFFIC.get(dom) if args.case == "full" and args.precision == "fp64"
                            and not args.autotune else None),
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the phase",
                "per_launch": {"flops" if unit == "GFLOP/s" else "bytes":
                               (kd["flops"] if unit == "GFLOP/s" else kd["bytes"]) / max(kd["launches"], 1),
                               "ms": kd["ms"] / max(kd["launches"], 1)},
                "peak_source": ("FP64 CUDA-core peak from unit counts and the 2070 MHz max clock "
                                "(152 SMs x 2 FMA/clk x 2 flop)")
                if unit == "GFLOP/s" else "MEASURED_PEAKS.json hbm_gbs (measured copy)",
                "fp64_peak_measured_gflops": fp64_measured,
                "precision": args.precision,
                "frac_of_measured_fp64": achieved / fp64_measured if unit == "GFLOP/s" else None,
                "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                "share": v["ms"] / max(sum(x["ms"] for x in ks.values()), 1e-12)}
                            for k, v in ks.items() if v["launches"]}}
    if args.precision != "fp64":
        # the tensor-core sector GEMMs (Theta' build and reassembly) against the format's peak
        tc = {}
        for k in ("theta", "gemm"):
            v = ks[k]
            if v["launches"] and v["ms"] > 0:
                tf = v["flops"] / (v["ms"] / 1000.0) / 1e12
                tc[k] = {"achieved": tf, "unit": "TFLOP/s", "peak": TENSOR_PEAK_TFLOPS[args.precision],
                         "frac": tf / TENSOR_PEAK_TFLOPS[args.precision],
                         "bytes_per_s_gb": v["bytes"] / (v["ms"] / 1000.0) / 1e9}
        roofline["tensor_gemms"] = tc
        roofline["tensor_peak_source"] = ("MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio (1.1/2.25)"
                                          if args.precision == "tf32" else
                                          "MEASURED_PEAKS.json bf16_tflops / 3 (three BF16 MMAs per product)")

    # e2e: the public API with host buffers, host wall clock, one observable read back per step
    glen = m.gate_length(D)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_upd = 0
    for _ in range(args.steps):
        e2e_upd += step()
        psi.expect(L // 2, np.arange(D, dtype=np.float64))
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, world)
    per_step = e2e_upd / args.steps
    e2e = {"value": world * e2e_upd / e2e_s, "unit": "updates/s",
           "h2d_bytes_per_step": int(per_step * glen * 16),
           "d2h_bytes_per_step": int(per_step * 8 + 8),
           "what": "steps through MPS.apply_layer with host gate buffers, plus one <n_i> read back per step"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, el, cores = oracle_sample(args.cpu_seconds)
        cpu = {"value": n / el, "unit": "updates/s", "cores": cores, "kind": "oracle",
               "sample": (f"{n} oracle updates ({el:.1f} s) of the odd layer, middle bonds first, on a saturated "
                          f"synthetic chi={CHI} chain (random blocks at Hilbert-proportional sector dims)")}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else f"{args.precision}+f64", "data": "synthetic",
                "config": config({"prep_steps": prep, "largest_bond_dim": mid_dims, "updates_timed": n_upd,
                                  "parallelism": "replicas" if world > 1 else "single",
                                  "precision": args.precision, "cuda_graphs": bool(args.graphs),
                                  "autotune": bool(args.autotune)}, case=args.case),
                "graphs": graph_stats, "autotune": {**m.autotune_stats(), "table": m.autotune_table()},
                "svd_deflation": deflation,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line), flush=True)
    psi.close()


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
    mix = dict(L_choices=(16, 32), chi_choices=(32, 64, 128), steps_range=(5, 40))
    raw = W.serving_requests(args.serve_requests, seed=rank, rate_hz=1.0, **mix)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=0.0)
            for r in raw]
    budget = 64 << 30
    # plain form: FP64, one request at a time, no merging, direct launches
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
    plain_rate = plain_updates / plain_s                    # updates/s
    # served capacity: every request queued at t = 0, merged launches across requests
    srv = m.serve.Server(budget_bytes=budget, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=graphs)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    cap_s = time.perf_counter() - t0
    srv.close()
    served_cap = sum(r.updates for r in res) / cap_s
    # accuracy of the served form against the plain FP64 form, per observable <n_i>
    obs_err = max(float(np.max(np.abs(r.observables - plain_obs[r.id]))) for r in res)
    # latency under load: Poisson arrivals at 0.8 x the served capacity (in requests/s)
    req_rate = 0.8 * len(reqs) / cap_s
    raw = W.serving_requests(args.serve_requests, seed=rank, rate_hz=req_rate, **mix)
    reqs = [m.serve.Request(r["id"], r["model"], r["L"], r["chi"], r["steps"], r["param"], arrival=r["arrival"])
            for r in raw]
    srv = m.serve.Server(budget_bytes=budget, max_slots=64, stream=stream.cuda_stream, precision=prec,
                         graphs=graphs)
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
                "config": {"workload": "serving_mix_scaled", "requests": len(reqs), **{k: list(v) for k, v in mix.items()},
                           "models": "xxz Delta~U[0,2] (Neel) / bh U~U[1,10] J=1 (Mott), 50/50",
                           "value": "served capacity (all requests queued at t=0, merged launches)",
                           "latency": "Poisson arrivals at 0.8 x the served capacity",
                           "plain": "FP64, each request alone, one after another, direct launches",
                           "served_precision": prec_name, "cuda_graphs": graphs, "budget_bytes": budget,
                           "max_slots": 64}}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.serve:
        run_serving(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
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
