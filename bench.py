#!/usr/bin/env python
"""Benchmark of the short-range nonbonded path on one GB300 (or N replicas).

Workload (the production-size configuration): a 96,000-atom rigid 3-site
water box (32,000 waters, L = 9.858 nm), rc = 1.0 nm, rlist = 1.1 nm,
r_inner = 1.04 nm, rolling prune every 10 evaluations. One step = one
trajectory of 100 force + energy evaluations on a Gaussian random walk
(sigma = 0.001 nm per component per frame), with the pair search and the
prunes the schedule calls for. All frames are resident in HBM before the
timed region; L2 is flushed (256 MiB write) between steps.

Metric: in-range pairs per second (pairs within rc counted by the force
kernel, summed over the 100 evaluations, divided by the step time) and
microseconds per force evaluation.

``--impl reference`` times the CPU FP64 oracle (all host cores) on the same
workload instead: each step is one full force + energy evaluation of one
frame.

Under torchrun each rank runs an independent replica (its own box seed);
there is no data-path collective.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "nonbonded pairs/s & µs/force-eval at 96k atoms; batched & backward vs plain"
UNIT = "pairs/s"
N_WATERS = 32000
RC, RLIST, R_INNER = 1.0, 1.1, 1.04
PRUNE_INTERVAL = 10
SIGMA = 0.001
KERNEL_SAMPLE = 10  # the force kernel is timed on 1 evaluation in KERNEL_SAMPLE
# FP32 operations per in-range pair in the force + energy formula as the
# kernel evaluates it (FMA = 2): d 3, r^2 5, rsqrt 1, 1/r^2 and 1/r^6 3, C6/r^6 and
# C12/r^12 3, LJ force scalar 4, r 1, beta r 1, exp 2, erfcx P/Q 18,
# erfc/r 2, f qi qj 1, force scalar 5, the 6 force FMAs 12, energies 5. The
# Newton steps of rsqrt and rcp and the exp polynomial's range reduction are
# not counted (they refine, they add no work to the formula).
FLOPS_PER_PAIR = 66
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


def workload_desc(evals: int) -> dict:
    L = synth.box_edge(N_WATERS)
    return {
        "workload": (f"water96k: 96,000-atom rigid 3-site water box ({N_WATERS} waters, L={L:.3f} nm), "
                     f"rc {RC} / rlist {RLIST} / r_inner {R_INNER} nm, prune every {PRUNE_INTERVAL} evals, "
                     f"{evals} force+energy evals per step on a sigma={SIGMA} nm random walk"),
        "n_atoms": 3 * N_WATERS,
        "evals_per_step": evals,
        "cache": "L2 flushed (256 MiB write) between timed steps",
    }


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--evals", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip every extra leg (see --legs)")
    ap.add_argument("--legs", default="peak,small,pme,backward,batched,halo,million",
                    help="comma-separated extra legs to run after the 96,000-atom one (default: all)")
    ap.add_argument("--no-tune", action="store_true",
                    help="default force launch shape and gathered tiles instead of autotuning them (for profiler "
                         "runs: under a profiler the tuner's timings, and so its choices, are not the bench's)")
    args = ap.parse_args()
    args.leg_set = set() if args.no_extras else {leg.strip() for leg in args.legs.split(",") if leg.strip()}
    unknown = args.leg_set - {"peak", "small", "pme", "backward", "batched", "halo", "million"}
    if unknown:
        ap.error(f"unknown legs: {sorted(unknown)}")
    return args


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def dist_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units_local: float, seconds_local: float, world: int) -> float:
    """Whole-job throughput of independent replicas: the units of all ranks
    divided by the slowest rank's time (max over ranks)."""
    return dist_sum(units_local, world) / dist_max(seconds_local, world)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- oracle timing

def time_oracle(box, frames, evals_budget_s: float = 15.0, max_evals: int = 20):
    """Oracle (FP64, all host cores) pairs/s on whole frames of the workload."""
    import oracle
    beta = synth.ewald_beta(RC)
    oracle.energy_forces(frames[0], box.q, box.type, box.ljparams, box.box, RC, beta, box.excl_off,
                         box.excl_idx)  # warm: builds/loads the library
    pairs = 0
    n = 0
    t0 = time.perf_counter()
    while n < max_evals and (time.perf_counter() - t0) < evals_budget_s:
        _, _, _, p = oracle.energy_forces(frames[n % len(frames)], box.q, box.type, box.ljparams, box.box, RC,
                                          beta, box.excl_off, box.excl_idx)
        pairs += p
        n += 1
    dt = time.perf_counter() - t0
    return pairs / dt, n, dt, oracle.threads()


def run_reference(args, rank, world):
    """The oracle on the host cores (rank 0 only), same metric and config."""
    if rank != 0:
        return
    import oracle
    box = synth.water_box(N_WATERS, 2)
    frames = synth.random_walk_frames(box, max(args.steps + args.warmup, 1), SIGMA, seed=2)
    beta = synth.ewald_beta(RC)
    times, pairs = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, _, p = oracle.energy_forces(frames[s % len(frames)], box.q, box.type, box.ljparams, box.box, RC,
                                          beta, box.excl_off, box.excl_idx)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pairs.append(p)
    value = sum(pairs) / sum(times)
    cores = oracle.threads()
    sample = "one full force+energy evaluation of one 96,000-atom frame per step (cell list, FP64)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(args.evals), parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm

def load_traffic(name: str = "force_kernel_traffic.json"):
    """DRAM bytes per launch from a committed ncu record under profiles/, if it matches the kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec.get("source_files", []):  # the kernel's sources, relative to the repository root
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec.get("bytes_per_launch_96k")


def _median_ms(fn, reps: int, stream):
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def measure_fp32_peak(dev, reps: int = 12, iters: int = 8192) -> dict:
    """FP32 rate of independent fused multiply-add chains on every SM (nb_fp32_peak_probe).

    Scalar FFMA and packed FFMA2 forms, 8 blocks of 256 threads per SM, each
    launch about 15 ms; three untimed launches, then ``reps`` launches timed
    with events on the launching stream while nvidia-smi samples the clocks.
    A fused multiply-add counts as 2 flops.
    """
    import torch

    from paper_2405_01420_gb300 import nb
    stream = torch.cuda.current_stream(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.empty(sms * 8 * 256, dtype=torch.float32, device=dev)
    res = {}
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    for packed in (False, True):
        flops = 0.0
        for _ in range(3):
            flops = nb.nb_fp32_peak_probe(out, packed=packed, iters=iters, stream=stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nb.nb_fp32_peak_probe(out, packed=packed, iters=iters, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        ts.sort()
        res["ffma2" if packed else "ffma"] = {"tflops_best": flops / ts[0] / 1e12,
                                              "tflops_median": flops / ts[len(ts) // 2] / 1e12,
                                              "ms_per_launch": 1e3 * ts[len(ts) // 2]}
    clocks = sampler.stop()
    best = max(v["tflops_median"] for v in res.values())
    return {"tflops": best, "forms": res, "clocks": clocks, "iters": iters, "reps": reps,
            "how": f"{sms} SMs x 8 blocks x 256 threads, 8 independent FMA chains per thread, "
                   f"{iters} x 16 steps per chain; median of {reps} event-timed launches; FMA = 2 flops"}


def bench_small(dev, reps: int = 200, with_oracle: bool = True) -> dict:
    """The smallest configuration: 1,536 atoms (512 waters), rc = rlist = 0.9 nm.

    One call sequence = nb_search + nb_forces (forces and energies). Timed
    two ways with events on the launching stream: as issued from Python one
    call after the other, and as one replay of a CUDA graph that captured the
    two calls; and the force call alone (gather, force kernel, permute-back
    on the searched list) as a graph replay. The oracle (FP64, all host
    cores) computes the same evaluation, timed beside it. Median and p99 of
    ``reps`` sequences.
    """
    import torch

    from paper_2405_01420_gb300 import nb
    import oracle
    rc = 0.9
    beta = synth.ewald_beta(rc)
    b = synth.water_box(512, 1)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x, q, t, lj, eo, ei = d(b.coords), d(b.q), d(b.type), d(b.ljparams), d(b.excl_off), d(b.excl_idx)
    stream = torch.cuda.current_stream(dev)
    counter = nb.Pairlist(b.n_atoms, count_pairs=True)
    counter.search(x, b.box, rc, eo, ei)
    counter.forces(x, q, t, lj, rc, beta)
    pairs = counter.stats()["pairs_last"]
    assert counter.status() == 0
    counter.close()

    pl = nb.Pairlist(b.n_atoms)
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)

    def seq(s=None):
        pl.search(x, b.box, rc, eo, ei, stream=s)
        pl.forces(x, q, t, lj, rc, beta, F, E, stream=s)

    def timed(fn):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            torch.cuda.synchronize()
            ts.append(1e3 * a.elapsed_time(e))
        return _percentile(ts, 50), _percentile(ts, 99)

    plain50, plain99 = timed(seq)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            seq(side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph50, graph99 = timed(g.replay)
    # the force call alone (gather, force kernel, permute-back) on the searched list, as a graph
    gf = torch.cuda.CUDAGraph()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(gf, stream=side):
            pl.forces(x, q, t, lj, rc, beta, F, E, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    forces50, forces99 = timed(gf.replay)
    # the host's view of one replay: launch, then wait for the result
    host = []
    for _ in range(reps):
        t0 = time.perf_counter()
        g.replay()
        torch.cuda.synchronize()
        host.append(1e6 * (time.perf_counter() - t0))
    assert pl.status() == 0
    e = E.cpu().numpy()
    # the force call on the pruned list (gathered tiles): what each evaluation costs once the list has
    # been pruned, as in a run that searches and prunes once for several evaluations
    pl.prune(x, rc)
    gp = torch.cuda.CUDAGraph()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(gp, stream=side):
            pl.forces(x, q, t, lj, rc, beta, F, E, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    pruned50, pruned99 = timed(gp.replay)
    assert pl.status() == 0
    Fo, elj, ec, _ = oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off,
                                          b.excl_idx)
    assert abs(e[0] - elj) <= 1e-6 * abs(elj) and abs(e[1] - ec) <= 1e-6 * abs(ec)
    pl.close()
    out = {"workload": "water1.5k: 1,536-atom water box (512 waters, L 2.484 nm), rc = rlist = 0.9 nm; "
                       "one nb_search + one nb_forces (forces and energies)",
           "pairs": pairs, "plain_p50_us": plain50, "plain_p99_us": plain99, "graph_p50_us": graph50,
           "graph_p99_us": graph99, "graph_host_wall_p50_us": _percentile(host, 50),
           "forces_only_graph_p50_us": forces50, "forces_only_graph_p99_us": forces99,
           "forces_after_prune_graph_p50_us": pruned50, "forces_after_prune_graph_p99_us": pruned99, "reps": reps,
           "paper_context": "19.2 us: the paper's minimum NBNXM walltime, smallest Grappa input (about 1.5k "
                            "atoms) on one MI250X GCD (Sec. III-A, Fig. 2); the force kernel alone on a pruned "
                            "list, not a search: compare forces_after_prune_graph (gather, kernel, permute-back)"}
    if with_oracle:
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            oracle.pairs_f64(b.coords, b.box, rc, b.excl_off, b.excl_idx)
            oracle.energy_forces(b.coords, b.q, b.type, b.ljparams, b.box, rc, beta, b.excl_off, b.excl_idx)
            ts.append(1e6 * (time.perf_counter() - t0))
        out["oracle_us"] = statistics.median(ts)
        out["oracle_cores"] = oracle.threads()
        out["oracle_sample"] = "pair set (FP64 brute force) + one FP64 force+energy evaluation, median of 5"
    return out


def pme_mesh(box, spacing: float = 0.12) -> tuple:
    """Mesh with at most ``spacing`` nm between points; sizes with no prime factor above 7."""
    def fft_size(n):
        while True:
            m = n
            for p in (2, 3, 5, 7):
                while m % p == 0:
                    m //= p
            if m == 1:
                return n
            n += 1
    return tuple(fft_size(int(np.ceil(float(L) / spacing))) for L in box)


def bench_pme(dev, reps: int = 50) -> dict:
    """PME charge spreading and force gathering on the 96,000-atom box (84^3 mesh, order 4).

    Ten calls of one kind are captured in a CUDA graph; a replay is timed
    with events on the launching stream (median of ``reps``) and divided by
    ten, so the device time per call excludes the host's launch overhead.
    Inputs are resident; the mesh (2.4 MB) and the atoms (1.9 MB) stay in L2
    between calls. The gather reads a random mesh potential (its cost does
    not depend on the values).
    """
    import torch

    from paper_2405_01420_gb300 import nb
    b = synth.water_box(N_WATERS, 2)
    K = pme_mesh(b.box)
    x = torch.from_numpy(b.coords).to(dev)
    q = torch.from_numpy(b.q).to(dev)
    grid = torch.empty(K, dtype=torch.float32, device=dev)
    phi = torch.randn(K, generator=torch.Generator(device=dev).manual_seed(1), device=dev)
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(5):
        nb.nb_pme_spread(x, q, b.box, K, grid)
        nb.nb_pme_gather(x, q, b.box, K, phi, F, energy=E)
    torch.cuda.synchronize()

    def per_call_ms(call, calls=10):
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for _ in range(calls):
                    call(side)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        return _median_ms(g.replay, reps, stream) / calls

    spread_ms = per_call_ms(lambda st: nb.nb_pme_spread(x, q, b.box, K, grid, stream=st))
    gather_ms = per_call_ms(lambda st: nb.nb_pme_gather(x, q, b.box, K, phi, F, energy=E, stream=st))
    n = b.n_atoms
    cells = int(np.prod(K))
    # algorithmic bytes: spread reads x, q (16 B per atom) and writes the mesh once; gather reads x, q and
    # the mesh once and writes the forces (12 B per atom)
    spread_bytes = 16 * n + 4 * cells
    gather_bytes = 16 * n + 4 * cells + 12 * n
    hbm_peak = 6780.0  # GB/s, the measured copy bandwidth of the GB300s
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    spread_gbs = spread_bytes / (spread_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_pme_spread (the larger of the two by DRAM-model time per call)",
            "achieved": spread_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": spread_gbs / hbm_peak,
            "traffic": load_traffic("pme_spread_traffic.json"),
            "note": "algorithmic bytes: 16 B per atom read and the mesh written once; the mesh stays in L2 and "
                    "the kernel is bound by the L1TEX queue of its 6.1M atomic additions, not by DRAM "
                    "(traffic: ncu DRAM read + write of one spread, cold)"}
    return {"workload": f"96,000-atom water box, {K[0]}x{K[1]}x{K[2]} mesh (0.117 nm), B-spline order 4; "
                        "spread = mesh cleared + charges spread; gather = forces + energy from a mesh potential",
            "roofline": roof,
            "mesh": list(K), "spread_us": 1e3 * spread_ms, "gather_us": 1e3 * gather_ms,
            "spread_atoms_per_s": n / (spread_ms / 1e3), "gather_atoms_per_s": n / (gather_ms / 1e3),
            "spread_mesh_updates_per_s": 64 * n / (spread_ms / 1e3),
            "spread_algorithmic_gbs": spread_bytes / (spread_ms / 1e3) / 1e9,
            "gather_algorithmic_gbs": gather_bytes / (gather_ms / 1e3) / 1e9, "reps": reps}


def bench_backward(dev, reps: int = 30):
    """Force-matching workload: 24,000 atoms, N(0, 0.4) charges, 4 LJ types.

    Times one forward call (forces + energies) and one forward plus the
    hand-written adjoint (nb_backward), each through the C ABI on resident
    inputs, median of ``reps``.
    """
    import torch
    from paper_2405_01420_gb300 import nb
    b = synth.water_box(8000, 4)
    p = synth.diff_params(b, seed=4)
    lj = torch.from_numpy(synth.combine_geometric(p["c6"], p["c12"]).astype(np.float32)).to(dev)
    x = torch.from_numpy(b.coords).to(dev)
    q = torch.from_numpy(p["q"].astype(np.float32)).to(dev)
    t = torch.from_numpy(p["type"]).to(dev)
    eo = torch.from_numpy(b.excl_off).to(dev)
    ei = torch.from_numpy(b.excl_idx).to(dev)
    beta = synth.ewald_beta(RC)
    pl = nb.Pairlist(b.n_atoms)
    pl.search(x, b.box, RLIST, eo, ei)
    pl.prune(x, R_INNER)
    F = torch.empty((b.n_atoms, 3), dtype=torch.float32, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)
    g = torch.randn((b.n_atoms, 3), dtype=torch.float32, device=dev)
    gx = torch.empty_like(F)
    gq = torch.empty_like(q)
    glj = torch.empty((4, 4, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def fwd():
        nb.nb_forces(pl.handle, x, q, t, lj, RC, beta, F, E)

    def fwd_bwd():
        nb.nb_forces(pl.handle, x, q, t, lj, RC, beta, F, E)
        nb.nb_backward(pl.handle, x, q, t, lj, RC, beta, g, gx, gq, glj)

    for _ in range(5):
        fwd_bwd()
    t_f = _median_ms(fwd, reps, stream)
    t_fb = _median_ms(fwd_bwd, reps, stream)
    assert pl.status() == 0
    pl.close()
    return {"workload": "24,000-atom box (8,000 waters), charges N(0,0.4) neutralised, 4 LJ types, rc 1.0 / "
                        "rlist 1.1 / r_inner 1.04 nm; forces+energies vs forces+energies then nb_backward "
                        "(dL/dx, dL/dq, dL/dC); median of 30 calls, inputs resident",
            "us_forward": 1e3 * t_f, "us_forward_backward": 1e3 * t_fb, "ratio_to_plain": t_fb / t_f}


def bench_million(dev, n_evals: int = 50, with_oracle: bool = True):
    """1,000,002 atoms (333,334 waters): 1 search + 50 evaluations with the rolling prune.

    Times each force kernel with events (inputs resident; the 50 frames of a
    sigma = 0.001 nm walk are in HBM), counts the in-range pairs of every
    evaluation on a separate counting list, and times one FP64 oracle
    evaluation of the first frame on the host cores.
    """
    import torch
    from paper_2405_01420_gb300 import nb
    from paper_2405_01420_gb300.engine import NonbondedEngine
    box = synth.water_box(333334, 3)
    frames = synth.random_walk_frames(box, n_evals, SIGMA, seed=3)
    N = box.n_atoms
    beta = synth.ewald_beta(RC)
    frames_d = torch.from_numpy(frames).to(dev)
    q = torch.from_numpy(box.q).to(dev)
    typ = torch.from_numpy(box.type).to(dev)
    lj = torch.from_numpy(box.ljparams).to(dev)
    eo = torch.from_numpy(box.excl_off).to(dev)
    ei = torch.from_numpy(box.excl_idx).to(dev)
    forces = torch.empty((N, 3), dtype=torch.float32, device=dev)
    energies = torch.zeros((n_evals, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    counter = NonbondedEngine(N, box.box, RC, beta, RLIST, R_INNER, PRUNE_INTERVAL, eo, ei, count_pairs=True)
    pairs = []
    for i in range(n_evals):
        counter.compute(frames_d[i], q, typ, lj, forces, energies[i])
        pairs.append(counter.pl.stats()["pairs_last"])
    assert counter.check() == 0
    counter.close()

    eng = NonbondedEngine(N, box.box, RC, beta, RLIST, R_INNER, PRUNE_INTERVAL, eo, ei)
    for i in range(3):  # warm-up
        eng.compute(frames_d[i], q, typ, lj, forces, energies[i])
    eng.evals_since_search = None
    eng.n_search = eng.n_prune = 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_evals)]
    for a, b in ev:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(n_evals):
        nb.nb_set_timing_events(eng.pl.handle, *ev[i])
        eng.compute(frames_d[i], q, typ, lj, forces, energies[i])
    t1.record(stream)
    torch.cuda.synchronize()
    nb.nb_set_timing_events(eng.pl.handle, None, None)
    assert eng.check() == 0
    total_ms = t0.elapsed_time(t1)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    n_search, n_prune = eng.n_search, eng.n_prune
    eng.close()
    total_pairs = float(sum(pairs))
    kern_mean = statistics.mean(kern_ms)
    out = {"workload": "1,000,002-atom water box (333,334 waters, L=21.53 nm), rc 1.0 / rlist 1.1 / r_inner 1.04 nm, "
                       f"1 search + {n_evals} force+energy evals with the rolling prune, sigma=0.001 nm walk, "
                       "frames resident",
           "pairs_per_eval": total_pairs / n_evals,
           "pairs_per_s": total_pairs / (total_ms / 1e3),
           "us_per_eval": 1e3 * total_ms / n_evals,
           "kernel_us_per_launch": 1e3 * kern_mean,
           "kernel_pairs_per_s": total_pairs / n_evals / (kern_mean / 1e3),
           "searches": n_search, "prunes": n_prune}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out["fp32_frac"] = FLOPS_PER_PAIR * out["kernel_pairs_per_s"] / (sms * FP32_LANES_PER_SM * 2 * 2070e6)
    if with_oracle:
        import oracle
        t = time.perf_counter()
        oracle.energy_forces(frames[0], box.q, box.type, box.ljparams, box.box, RC, beta, box.excl_off,
                             box.excl_idx)
        dt = time.perf_counter() - t
        out["cpu_oracle_s_per_eval"] = dt
        out["cpu_oracle_pairs_per_s"] = pairs[0] / dt
    return out


def bench_halo(dev, reps: int = 30) -> dict:
    """Local / non-local split with a synthetic halo exchange (96,000 atoms).

    Two halo shapes of a domain decomposition with a halo of width rlist:
    ``slab`` (the waters whose oxygen lies within rlist of the upper x face,
    one neighbour domain) and ``shell`` (within rlist of any of the three
    upper faces, as in an eighth-shell decomposition). Halo atoms are
    numbered last. Each evaluation copies the halo atoms' coordinates from
    pinned host memory (the receive of a halo exchange), then computes
    forces and energies. Sequential: copy, then nb_forces. Overlapped: the
    local part runs on the compute stream while the copy runs on a second
    stream; the non-local part waits for the copy. Also timed on their own:
    the copy, the unsplit forces, the local part and the non-local part.
    Each schedule is captured in a CUDA graph (the copy a memcpy node, the
    wait a graph edge) and replayed: medians over ``reps`` replays, events on
    the compute stream, so host launch overhead is not counted.
    """
    out = {}
    for shape in ("slab", "shell"):
        out[shape] = _halo_case(dev, shape, reps)
    return out


def _halo_case(dev, shape: str, reps: int) -> dict:
    import torch
    from paper_2405_01420_gb300 import nb
    b = synth.water_box(N_WATERS, 2)
    L = b.box.astype(np.float64)
    o = b.coords[0::3].astype(np.float64)
    if shape == "slab":
        is_halo = o[:, 0] >= L[0] - RLIST
    else:
        is_halo = (o >= L - RLIST).any(axis=1)
    home = np.flatnonzero(~is_halo)
    halo = np.flatnonzero(is_halo)
    atoms = (3 * np.concatenate([home, halo])[:, None] + np.arange(3)[None, :]).reshape(-1)
    x = np.ascontiguousarray(b.coords[atoms])
    n_home = 3 * len(home)
    N = b.n_atoms
    base = 3 * (np.arange(N) // 3)
    k = np.arange(N) % 3
    ei = np.empty(2 * N, np.int32)
    ei[0::2] = base + (k + 1) % 3
    ei[1::2] = base + (k + 2) % 3
    eo = (2 * np.arange(N + 1)).astype(np.int32)
    beta = synth.ewald_beta(RC)
    xd = torch.from_numpy(x).to(dev)
    q = torch.from_numpy(np.ascontiguousarray(b.q[atoms])).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(b.type[atoms])).to(dev)
    lj = torch.from_numpy(b.ljparams).to(dev)
    halo_host = torch.from_numpy(np.ascontiguousarray(x[n_home:])).pin_memory()
    pl = nb.Pairlist(N)
    pl.set_home(n_home)
    pl.search(xd, b.box, RLIST, torch.from_numpy(eo).to(dev), torch.from_numpy(ei).to(dev))
    pl.prune(xd, R_INNER)
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)
    main = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    halo_dev = xd[n_home:]

    def copy():
        halo_dev.copy_(halo_host, non_blocking=True)

    def forces():
        nb.nb_forces(pl.handle, xd, q, t, lj, RC, beta, F, E)

    def local():
        nb.nb_forces_part(pl.handle, nb.NB_PART_LOCAL, xd, q, t, lj, RC, beta, None, E)

    def nonlocal_():
        nb.nb_forces_part(pl.handle, nb.NB_PART_NONLOCAL, xd, q, t, lj, RC, beta, F, E)

    def sequential():
        copy()
        forces()

    def overlapped():
        cur = torch.cuda.current_stream(dev)  # the compute stream (the capturing one inside a graph)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            copy()
        local()
        cur.wait_stream(side)
        nonlocal_()

    for _ in range(5):
        sequential()
        overlapped()
    torch.cuda.synchronize()

    def graph_ms(fn):
        # captured once and replayed: the device time without the host's launch overhead
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(main)
        with torch.cuda.graph(g, stream=cap):
            fn()
        main.wait_stream(cap)
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        return _median_ms(g.replay, reps, main)

    t_copy = graph_ms(copy)
    t_forces = graph_ms(forces)
    t_local = graph_ms(local)
    t_nonlocal = graph_ms(lambda: (local(), nonlocal_())) - t_local
    t_seq = graph_ms(sequential)
    t_ovl = graph_ms(overlapped)
    assert pl.status() == 0
    pl.close()
    desc = ("waters with O within rlist of the upper x face" if shape == "slab"
            else "waters with O within rlist of any upper face (eighth shell)")
    return {"workload": f"96,000-atom water box, {desc} as halo atoms ({N - n_home} atoms, "
                        f"{12 * (N - n_home)} B of coordinates copied from pinned host memory per evaluation), "
                        "rc 1.0 / r_inner 1.04 nm, after a prune",
            "halo_atoms": N - n_home, "us_copy": 1e3 * t_copy, "us_forces": 1e3 * t_forces,
            "us_local": 1e3 * t_local, "us_nonlocal": 1e3 * t_nonlocal,
            "us_split_cost": 1e3 * (t_local + t_nonlocal - t_forces),
            "us_sequential": 1e3 * t_seq, "us_overlapped": 1e3 * t_ovl, "saving": 1.0 - t_ovl / t_seq}


def _concat_systems(boxes):
    off = np.zeros(len(boxes) + 1, np.int32)
    for k, b in enumerate(boxes):
        off[k + 1] = off[k] + b.n_atoms
    eo = [np.zeros(1, np.int32)]
    ei = []
    base = 0
    for k, b in enumerate(boxes):
        eo.append(b.excl_off[1:] + base)
        ei.append(b.excl_idx + off[k])
        base += b.excl_off[-1]
    return (off, np.concatenate([b.coords for b in boxes]), np.concatenate([b.q for b in boxes]),
            np.concatenate([b.type for b in boxes]), np.concatenate(eo), np.concatenate(ei),
            np.stack([b.box for b in boxes]))


def _percentile(ts, p):
    ts = sorted(ts)
    return ts[min(len(ts) - 1, int(round(p / 100.0 * (len(ts) - 1))))]


def bench_batch(dev, n_boxes: int = 256, reps: int = 30, plain_reps: int = 5):
    """Batched form: 256 independent water boxes of 1,536..24,000 atoms.

    One batch = search (rlist 1.0) + forces and energies (rc 0.9) of every box.
    Batched: one pair list over all boxes, the whole batch captured in one
    CUDA graph and replayed. Plain: one pair list per box, nb_search +
    nb_forces launched box after box. Per-batch latency from CUDA events.
    """
    import torch
    from paper_2405_01420_gb300 import nb
    rc, rlist = 0.9, 1.0
    beta = synth.ewald_beta(rc)
    boxes = synth.batch_boxes(n_boxes, 1536, 24000, seed=5)
    off, x, q, t, eo, ei, bx = _concat_systems(boxes)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    xd, qd, td, eod, eid = d(x), d(q), d(t), d(eo), d(ei)
    lj = d(boxes[0].ljparams)
    stream = torch.cuda.current_stream(dev)
    counter = nb.Pairlist.batch(off, bx, count_pairs=True)
    counter.search(xd, None, rlist, eod, eid)
    counter.forces(xd, qd, td, lj, rc, beta)
    pairs = counter.stats()["pairs_last"]
    assert counter.status() == 0
    counter.close()

    from paper_2405_01420_gb300.tune import tune_batch_prune, tune_force_shape, tune_tile_form
    pl = nb.Pairlist.batch(off, bx)
    F = torch.empty((pl.n_atoms, 3), dtype=torch.float32, device=dev)
    E = torch.empty(2 * pl.n_systems, dtype=torch.float64, device=dev)
    pl.search(xd, None, rlist, eod, eid)
    pl.forces(xd, qd, td, lj, rc, beta, F, E)
    torch.cuda.synchronize()
    # autotune (untimed), each step at the default launch shape: whether to prune to rc before the
    # forces, then the tile form; last the force launch shape, on the list the batch will use (one
    # shape serves both force kernels, and they favour different ones)
    use_prune, prune_times = tune_batch_prune(lambda: pl.search(xd, None, rlist, eod, eid),
                                              lambda: pl.prune(xd, rc),
                                              lambda: pl.forces(xd, qd, td, lj, rc, beta, F, E), reps=3)
    tile_form, tile_times = "cluster", None
    pl.search(xd, None, rlist, eod, eid)
    if use_prune:  # the tile form matters only after a prune
        pl.prune(xd, rc)
        tile_form, tile_times = tune_tile_form(pl, lambda: pl.forces(xd, qd, td, lj, rc, beta, F, E), reps=3)
    shape, _ = tune_force_shape(pl, lambda: pl.forces(xd, qd, td, lj, rc, beta, F, E), reps=3)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            pl.search(xd, None, rlist, eod, eid, stream=side)
            if use_prune:
                pl.prune(xd, rc, stream=side)
            pl.forces(xd, qd, td, lj, rc, beta, F, E, stream=side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    graph_ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        graph_ms.append(a.elapsed_time(b))
    assert pl.status() == 0
    pl.close()

    plain = []
    for k, bxk in enumerate(boxes):
        p1 = nb.Pairlist(bxk.n_atoms)
        plain.append((p1, int(off[k]), int(off[k + 1]), bxk))
    Fp = torch.empty_like(F)
    Ep = torch.empty(2 * n_boxes, dtype=torch.float64, device=dev)

    # per-system exclusion slices are rebuilt outside the timed region
    excl = [((eod[a0:a1 + 1] - eod[a0]).contiguous(), (eid[int(eo[a0]):int(eo[a1])] - a0).contiguous())
            for (_, a0, a1, _) in plain]

    def plain_batch_pre():
        for k, (p1, a0, a1, bxk) in enumerate(plain):
            nb.nb_search(p1.handle, xd[a0:a1], bxk.box, rlist, excl[k][0], excl[k][1])
            nb.nb_forces(p1.handle, xd[a0:a1], qd[a0:a1], td[a0:a1], lj, rc, beta, Fp[a0:a1], Ep[2 * k:2 * k + 2])

    plain_batch_pre()
    torch.cuda.synchronize()
    plain_ms = []
    for _ in range(plain_reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain_batch_pre()
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b))
    for p1, _, _, _ in plain:
        assert p1.status() == 0
        p1.close()
    torch.testing.assert_close(Fp, F, rtol=0, atol=1e-4 * F.abs().max().item())
    g50, g99 = _percentile(graph_ms, 50), _percentile(graph_ms, 99)
    p50, p99 = _percentile(plain_ms, 50), _percentile(plain_ms, 99)
    return {"workload": f"{n_boxes} independent water boxes, {int(off[-1])} atoms in total (1,536..24,000 each, "
                        "whole waters), rc 0.9 / rlist 1.0 nm; one batch = search + forces + energies of every box",
            "pairs_per_batch": pairs,
            "graph_p50_ms": g50, "graph_p99_ms": g99, "graph_pairs_per_s": pairs / (g50 / 1e3),
            "plain_launches_p50_ms": p50, "plain_launches_p99_ms": p99, "plain_pairs_per_s": pairs / (p50 / 1e3),
            "speedup_p50": p50 / g50, "graph_reps": reps, "plain_reps": plain_reps,
            "tuned": {"force_shape": list(shape), "prune_before_forces": bool(use_prune),
                      "prune_choice_ms": prune_times, "tile_form": tile_form, "tile_form_ms": tile_times}}


def run_ours(args, rank, world, local):
    import torch

    from paper_2405_01420_gb300 import nb
    from paper_2405_01420_gb300.engine import NonbondedEngine

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nb.load_library()
    box = synth.water_box(N_WATERS, 2 + rank)
    frames = synth.random_walk_frames(box, args.evals, SIGMA, seed=2 + rank)
    N = box.n_atoms
    beta = synth.ewald_beta(RC)
    frames_d = torch.from_numpy(frames).to(dev)
    q = torch.from_numpy(box.q).to(dev)
    typ = torch.from_numpy(box.type).to(dev)
    lj = torch.from_numpy(box.ljparams).to(dev)
    eo = torch.from_numpy(box.excl_off).to(dev)
    ei = torch.from_numpy(box.excl_idx).to(dev)
    forces = torch.empty((N, 3), dtype=torch.float32, device=dev)
    energies = torch.zeros((args.evals, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    eng = NonbondedEngine(N, box.box, RC, beta, RLIST, R_INNER, PRUNE_INTERVAL, eo, ei)

    def restart():
        eng.evals_since_search = None
        eng.interval = PRUNE_INTERVAL
        eng.n_search = eng.n_prune = 0

    def one_step(frame_src, kernel_events=None, out_forces=None):
        restart()
        for i in range(args.evals):
            if kernel_events is not None:
                nb.nb_set_timing_events(eng.pl.handle, *kernel_events.get(i, (None, None)))
            x = frame_src(i)
            eng.compute(x, q, typ, lj, forces, energies[i])
            if out_forces is not None:
                out_forces(i)
        if kernel_events is not None:
            nb.nb_set_timing_events(eng.pl.handle, None, None)

    # untimed pass on a counting pair list: in-range pairs of each evaluation
    # (the count is exact, so it does not depend on which list found them)
    counter = NonbondedEngine(N, box.box, RC, beta, RLIST, R_INNER, PRUNE_INTERVAL, eo, ei, count_pairs=True)
    pairs = []
    for i in range(args.evals):
        counter.compute(frames_d[i], q, typ, lj, forces, energies[i])
        pairs.append(counter.pl.stats()["pairs_last"])
    assert counter.check() == 0, "device error word set in the counting pass"
    counter.close()
    pairs_per_step = float(sum(pairs))

    # autotune the force kernel's launch shape and tile form on this workload (untimed)
    from paper_2405_01420_gb300.tune import tune_force_shape, tune_tile_form
    restart()
    eng.compute(frames_d[0], q, typ, lj, forces, energies[0])
    force_call = lambda: nb.nb_forces(eng.pl.handle, frames_d[0], q, typ, lj, RC, beta, forces, energies[0])
    if args.no_tune:
        shape, shape_times, tile_form, tile_times = (256, 16, 0), None, "gathered", None
    else:
        shape, shape_times = tune_force_shape(eng.pl, force_call)
        tile_form, tile_times = tune_tile_form(eng.pl, force_call)

    for _ in range(args.warmup):
        one_step(lambda i: frames_d[i])
    torch.cuda.synchronize()

    # the force kernel is timed with an event pair on a sample of the evaluations (an event record costs
    # about a microsecond of stream time), whose positions cycle through the prune interval
    ev = {i: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for i in range(args.evals) if i % KERNEL_SAMPLE == (i // KERNEL_SAMPLE) % KERNEL_SAMPLE}
    for a, b in ev.values():  # torch only times events it has recorded once; libnb re-records them at the kernel
        a.record(stream)
        b.record(stream)
    sampler = ClockSampler(local) if rank == 0 else None
    step_ms, kern_ms = [], []
    searches = prunes = 0
    if sampler:
        sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier(world)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        one_step(lambda i: frames_d[i], kernel_events=ev)
        t1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(t0.elapsed_time(t1))
        kern_ms.append(statistics.mean(a.elapsed_time(b) for a, b in ev.values()))
        searches, prunes = eng.n_search, eng.n_prune
    clocks = sampler.stop() if sampler else None
    err = eng.check()
    assert err == 0, f"device error word 0x{err:x} in the timed steps"

    ms_step = dist_max(statistics.mean(step_ms), world)
    value = replica_throughput(pairs_per_step * args.steps, sum(step_ms) / 1e3, world)
    kern_ms_per_launch = statistics.mean(kern_ms)
    pairs_per_eval = pairs_per_step / args.evals

    # end to end through the public API: each evaluation's frame comes from pinned host memory and its
    # forces and energies go back to pinned host memory, all inside the timed region. The copies run on
    # a second stream, double-buffered, as an MD driver would overlap them: frame i + 1 comes in and the
    # results of i - 1 go out while evaluation i computes.
    e2e = None
    if not args.no_e2e:
        frames_h = torch.from_numpy(frames).pin_memory()
        f_out = torch.empty((args.evals, N, 3), dtype=torch.float32).pin_memory()
        e_out = torch.empty((args.evals, 2), dtype=torch.float64).pin_memory()
        x_buf = [torch.empty((N, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        f_buf = [torch.empty((N, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        copy_s = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]    # frame copied into buffer b
        ev_done = [torch.cuda.Event() for _ in range(2)]  # evaluation on buffer b computed
        ev_out = [torch.cuda.Event() for _ in range(2)]   # results of buffer b copied out

        def e2e_step():
            restart()
            copy_s.wait_stream(stream)  # no copy starts before the timed region does
            with torch.cuda.stream(copy_s):
                x_buf[0].copy_(frames_h[0], non_blocking=True)
                ev_in[0].record(copy_s)
            for i in range(args.evals):
                b = i % 2
                if i + 1 < args.evals:  # the next frame, once the evaluation that used its buffer has run
                    nb_ = (i + 1) % 2
                    with torch.cuda.stream(copy_s):
                        if i >= 1:
                            copy_s.wait_event(ev_done[nb_])
                        x_buf[nb_].copy_(frames_h[i + 1], non_blocking=True)
                        ev_in[nb_].record(copy_s)
                stream.wait_event(ev_in[b])
                if i >= 2:
                    stream.wait_event(ev_out[b])  # buffer b's forces of evaluation i - 2 are out
                eng.compute(x_buf[b], q, typ, lj, f_buf[b], energies[i])
                ev_done[b].record(stream)
                with torch.cuda.stream(copy_s):
                    copy_s.wait_event(ev_done[b])
                    f_out[i].copy_(f_buf[b], non_blocking=True)
                    e_out[i].copy_(energies[i], non_blocking=True)
                    ev_out[b].record(copy_s)
            stream.wait_stream(copy_s)  # the step ends with the last results on the host

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier(world)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        # the last step's results reached the host: spot-check them against the device copies
        assert torch.equal(f_out[args.evals - 1], f_buf[(args.evals - 1) % 2].cpu())
        assert torch.equal(e_out[args.evals - 1], energies[args.evals - 1].cpu())
        e2e_value = replica_throughput(pairs_per_step * args.steps, sum(e2e_ms) / 1e3, world)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": args.evals * N * 12,
               "d2h_bytes_per_step": args.evals * (N * 12 + 16),
               "copies": "second stream, double-buffered: overlapped with the evaluations"}
        assert eng.check() == 0

    # the list's side of an evaluation: search and prune calls timed on their own (events, median of 5),
    # and the pair slots the force kernel computes (32 per gathered tile of the current list)
    slots = 32 * eng.pl.stats()["gathered_tiles"]
    x_last = frames_d[args.evals - 1]

    def _call_us(fn):
        ts = []
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(1e3 * a.elapsed_time(b))
        return statistics.median(ts)

    # the same force call without energies (what an MD step that does not report energies runs):
    # the force kernel alone, events around it on 20 calls
    ev_f = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e_ in ev_f:
        e_.record(stream)
    nb.nb_set_timing_events(eng.pl.handle, *ev_f)
    f_only = []
    for _ in range(20):
        nb.nb_forces(eng.pl.handle, x_last, q, typ, lj, RC, beta, forces, None)
        torch.cuda.synchronize()
        f_only.append(ev_f[0].elapsed_time(ev_f[1]))
    nb.nb_set_timing_events(eng.pl.handle, None, None)
    forces_only_us = 1e3 * statistics.median(f_only)
    search_us = _call_us(lambda: eng.pl.search(x_last, box.box, RLIST, eo, ei))
    prune_us = _call_us(lambda: eng.pl.prune(x_last, R_INNER))
    list_side = {"search_us_per_call": search_us, "prune_us_per_call": prune_us,
                 "force_kernel_no_energy_us": forces_only_us,
                 "list_us_per_eval": (search_us * searches + prune_us * prunes) / args.evals,
                 "pair_slots_per_eval": slots, "slot_efficiency": pairs_per_eval / slots if slots else None}
    assert eng.check() == 0

    legs = args.leg_set
    fp32_peak = measure_fp32_peak(dev) if "peak" in legs else None
    small = bench_small(dev, with_oracle=(rank == 0 and world == 1 and not args.no_cpu_baseline)) \
        if "small" in legs else None
    pme = bench_pme(dev) if "pme" in legs else None
    backward = bench_backward(dev) if "backward" in legs else None
    batched = bench_batch(dev) if "batched" in legs else None
    halo = bench_halo(dev) if "halo" in legs else None
    million = bench_million(dev, with_oracle=(rank == 0 and world == 1 and not args.no_cpu_baseline)) \
        if "million" in legs else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n_ev, dt, cores = time_oracle(box, frames)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_ev} full force+energy evaluations of frames of the same 96,000-atom trajectory "
                         f"(cell list, FP64), {dt:.1f} s"}

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak_nominal = sms * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    achieved = FLOPS_PER_PAIR * pairs_per_eval / (kern_ms_per_launch / 1e3) / 1e12
    nominal_basis = f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop/FMA x 2070 MHz (max SM clock)"
    if fp32_peak is not None:
        peak, basis = fp32_peak["tflops"], ("measured: FP32 FMA-chain probe (nb_fp32_peak_probe), the faster of "
                                            "FFMA and FFMA2, in this run; see fp32_peak")
    else:
        peak, basis = peak_nominal, nominal_basis
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": load_traffic(),
            "kernel": "k_force_vt (gathered 4x8 tiles after the prune; LJ + Ewald real-space, energies on)",
            "peak_basis": basis, "peak_nominal": peak_nominal, "peak_nominal_basis": nominal_basis,
            "frac_nominal": achieved / peak_nominal,
            "peak_measured": None if fp32_peak is None else fp32_peak["tflops"],
            "kernel_us_per_launch": 1e3 * kern_ms_per_launch}
    if clocks and clocks.get("sm_mhz"):
        peak_clk = sms * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e6 / 1e12
        roof["frac_nominal_at_measured_clock"] = achieved / peak_clk
    # our kernels per call: a search 6 (system table, 4 grid-sort kernels, search; the exclusion list only
    # with the excluded-pair correction, which this workload leaves off), a prune 4 (its gather, prune,
    # length offsets, length scatter), an evaluation 3 (gather, force, scatter)
    n_launch_search, n_launch_prune, n_launch_force = 6, 4, 3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_desc(args.evals), parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "us_per_eval": 1e3 * ms_step / args.evals,
        "pairs_per_eval": pairs_per_eval,
        "list": list_side,
        "searches_per_step": searches, "prunes_per_step": prunes,
        "force_shape": {"threads": shape[0], "chunk": shape[1], "blocks_per_sm": shape[2], "tuned_ms": shape_times,
                        "tile_form": tile_form, "tile_form_ms": tile_times},
        "roofline": roof,
        "fp32_peak": fp32_peak,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": n_launch_search * searches + n_launch_prune * prunes + n_launch_force * args.evals,
        "small": small,
        "pme": pme,
        "backward": backward,
        "batched": batched,
        "million": million,
        "halo": halo,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
