#!/usr/bin/env python
"""Benchmark: converged collision solves per second on one GB300.

Headline workload (one step = one collision_solve over every node, inputs
resident in HBM): the perturbed collapse profile (+-10% seeded perturbations of
rho, T and Ye), 2^20 nodes, 4 species (nu_e, anti-nu_e, nu_x, anti-nu_x),
Grid F with linear elements (32 x 2 = 64 energies), emission/absorption +
isoenergetic + NES + pair, Anderson depth 3, solved by the mixed-precision
persistent kernel at tol 1e-10 (inner; the tolerance at which the mixed path
stays within 1e-5 of the FP64 solve on this batch) and 1e-9 (outer).  On the same
inputs the line also times the FP64 persistent kernel and the plain FP64
per-iteration launches (NMC_MODE_PLAIN), both at tol 1e-10, and reports the
mixed path's error against the FP64 solve (every node) and against the CPU
oracle (the nodes of the CPU-baseline sample).  Inputs (J, H: 8.6 GB) are
larger than L2, so every step reads them from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nmc|reference]

The roofline denominators are measured by nmc_fma_probe (FP64 and FP32 FMA
chains at full occupancy, CUDA events) once the GPU is warm, before the
headline's timed steps.
Further objects on the same line, each timed the same way on its own
workload:
  "batching"        the uneven core/tail mix of 2^22 nodes (half rho > 1e13,
                    half rho < 1e10, dt log-uniform 1e-7..1e-5 s, Grid C
                    16x2): persistent FP64 kernel replayed from a CUDA graph,
                    mixed persistent kernel, and plain FP64 launches
                    (one timed step each, --batching-steps);
  "adjoint"         collision_adjoint over 2^18 profile nodes (Grid C 16x2);
  "velocity"        collision_solve_v (the O(v/c) solve) over 2^16 nodes;
  "c2p"             conserved_to_primitive over every bin of 2^16 nodes;
  "opacity_interp"  tetralinear interpolation at 2^23 scattered points;
  "relaxation"      the relaxation problem of Sec. 6.1, 4096 problems.
The side objects time min(K, 5) steps after min(W, 2) warm-up steps.

Prints one JSON line.  --impl reference times the CPU oracle (the plain FP64
restatement of the algorithm) on a bounded sample of the headline workload.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# headline workload: Grid F with linear elements, perturbed profile, 2^20 nodes
N_NODES = 1 << 20
H_ELEM, H_DE1 = 32, 1.0
NQ, NS = 2, 4
MEM = 3
TOL = 1e-10   # FP64 paths
# inner, outer tolerances of the mixed path: where dtau chi ~ 1e4 the heavy flavours' number-conserving
# mode keeps an error ~ tol_inner (1 + dtau chi), so the stated <= 1e-5 error on the perturbed
# 64-energy batch needs tol_inner 1e-10 (1.04e-5 at 3e-10); the outer test at 1e-9, because between
# outer iterations the FP32 rounding of the converged moments moves the matter map by ~1e-10
# relative (at 1e-10, 142 of the 2^20 nodes cycled to the outer cap; none at 1e-9)
MIXED_TOL = (1e-10, 1e-9)
# side workloads: Grid C with linear elements (32 energies)
N_ELEM, DE1 = 16, 1.875
SIDE_NODES = 1 << 16
METRIC = "converged collision solves/s (nodes*steps/s), mixed vs FP64 at stated error"
WORKLOAD = ("perturbed collapse profile (+-10% seeded perturbations of rho, T, Ye), 2^20 nodes, 4 species, "
            "Grid F 32x2 = 64 energies, EmAb+Iso+NES+pair, Anderson depth 3, mixed precision at tol 1e-10 "
            "(inner) and 1e-9 (outer); FP64 at tol 1e-10 on the same inputs")
# DRAM bytes (read + write) per node of one launch, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum); traffic grows with the node count.  None where the kernel has changed since its
# counters were taken.
TRAFFIC_PER_NODE = {"fused_kernel<double>": 15540.0, "fused_kernel<float>": 14506.0,
                    "adjoint_kernel": 12079.0, "velocity_kernel": 6029.0,
                    "c2p_kernel": 530723584 / 65536, "opacity_interp_kernel": 159e6 / (1 << 22),
                    "opacity_interp_mixed_kernel": 162e6 / (1 << 22)}


def _traffic(kernel, n):
    t = TRAFFIC_PER_NODE[kernel]
    return None if t is None else t * n


CPU_SAMPLE = 24           # oracle sample (nodes) for the CPU baseline, one thread
CPU_PER_CORE = 6          # oracle nodes per core for the all-cores CPU baseline
ADJ_NODES = 1 << 18
BATCH_NODES = 1 << 22
REL_WORKLOAD = ("relaxation problem of Sec. 6.1 (six species, Grid C 16x2, v = 0.1 c, Gaussian forward-peaked "
                "initial neutrinos), +-10% seeded perturbations of rho = 1e12, T = 7.6 MeV, Ye = 0.135 per problem, "
                "backward Euler with dt from 1e-4 ms x1.04 per step to t = 100 ms, tol 1e-8, Anderson depth 2")
C2P_WORKLOAD = ("conserved-to-primitive recovery of every bin (collapse profile, 2^16 nodes x 4 species x 32 "
                "energies, conserved moments of the profile's occupations, infall velocity up to 0.15 c), FP64, "
                "tol 1e-8, Anderson memory 3")
C2P_BYTES_PER_BIN = 68    # N, G in; D, I, iteration count out (8 + 24 + 8 + 24 + 4 bytes)
INTERP_WORKLOAD = ("opacity_interp: chi_EmAb and sigma_Iso of each of 4 species (8 launches per step) at 2^23 "
                   "scattered points, (rho, T, Ye) uniform in (log10 rho, log10 T, Ye) over the tables and E "
                   "log-uniform over Grid C 16x2's node energies, FP64, inputs larger than L2")
INTERP_BYTES_PER_POINT = 40   # rho, T, Ye, E in and the interpolated value out, f64, per launch
VEL_WORKLOAD = ("O(v/c) solve (collapse profile, 2^16 nodes, 4 species, Grid C 16x2 energies, all processes, "
                "infall velocity field up to 0.15 c, Minerbo closure, FP64, tol 1e-10, Anderson depth 3)")
ADJ_WORKLOAD = ("gradient of the FP64 solve (collapse profile, 2^18 nodes, 4 species, Grid C 16x2 energies, "
                "all processes, forward tol 1e-10) w.r.t. J, H, Ye, T and the 4 opacity scales, "
                "cotangents on J, H, Ye, eps, T")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nmc", choices=["nmc", "reference"])
    ap.add_argument("--nodes", type=int, default=N_NODES)
    ap.add_argument("--compare-steps", type=int, default=1,
                    help="timed steps of the FP64 persistent and plain FP64 arms on the headline inputs (0 skips)")
    ap.add_argument("--adjoint-nodes", type=int, default=ADJ_NODES, help="0 skips the adjoint measurement")
    ap.add_argument("--batching-nodes", type=int, default=BATCH_NODES,
                    help="nodes of the persistent-vs-plain comparison (0 skips it)")
    ap.add_argument("--batching-steps", type=int, default=1, help="timed steps of each batching arm")
    ap.add_argument("--velocity-nodes", type=int, default=SIDE_NODES,
                    help="nodes of the O(v/c) solve measurement (0 skips it)")
    ap.add_argument("--c2p-nodes", type=int, default=SIDE_NODES,
                    help="nodes of the conserved-to-primitive measurement (0 skips it)")
    ap.add_argument("--interp-points", type=int, default=1 << 23,
                    help="points of the opacity_interp measurement (0 skips it)")
    ap.add_argument("--relaxation-problems", type=int, default=4096,
                    help="problems in the relaxation-driver measurement (0 skips it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    return ap.parse_args()


def _grid(n_elem=H_ELEM, de1=H_DE1):
    """Interfaces and node energies of a geometric grid with linear elements, from the library."""
    from paper_2601_00976_gb300 import nmc
    edges, _ = nmc.geometric_edges(n_elem, de1)
    eps, _, _ = nmc.grid_nodes(edges, NQ)
    return edges, eps


def _workload(seed, nodes, oracle_grid=False, kind="perturbed", n_elem=H_ELEM, de1=H_DE1):
    """Grid, synthetic tables and seeded node inputs of a workload (the headline's by default)."""
    from paper_2601_00976_gb300 import synthetic
    if oracle_grid:      # the reference arm builds its grid with the oracle's own code
        from oracle import grid as ogrid
        edges, _ = ogrid.geometric_edges(n_elem, de1)
        eps = ogrid.EnergyGrid(edges, NQ).eps
    else:
        edges, eps = _grid(n_elem, de1)
    tables = synthetic.make_tables(eps, NS, seed=0)
    inp = synthetic.make_inputs(kind, nodes, eps, NS, seed=seed)
    return edges, eps, tables, inp


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    from paper_2601_00976_gb300.dist import world
    return world()


def run_reference(args):
    """Time the CPU oracle on a bounded sample of the headline workload (the reference arm)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import grid as ogrid, solver as osolver
    edges, _, tables, inp = _workload(0, CPU_SAMPLE, oracle_grid=True)
    g = ogrid.EnergyGrid(edges, NQ)
    prm = osolver.Params(tol_inner=TOL, tol_outer=TOL, M_inner=MEM, M_outer=MEM)
    per = max(2, CPU_SAMPLE // 8)
    for w in range(args.warmup):
        osolver.solve(g, tables, prm, inp, nodes=range(w % CPU_SAMPLE, w % CPU_SAMPLE + 1))
    t_all = time.perf_counter()
    for k in range(args.steps):
        lo = (k * per) % CPU_SAMPLE
        osolver.solve(g, tables, prm, inp, nodes=range(lo, lo + per))
    total = time.perf_counter() - t_all
    value = per * args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (the CPU oracle, tol 1e-10)",
                   "sample_nodes_per_step": per},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per} nodes of the headline workload per step, numpy FP64 oracle, one thread"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


_CPU_STATE = None


def _cpu_worker_init():
    """Oracle grid, tables and parameters of the headline workload in a worker process (built once)."""
    global _CPU_STATE
    from oracle import grid as ogrid, solver as osolver
    from paper_2601_00976_gb300 import synthetic
    edges, _ = ogrid.geometric_edges(H_ELEM, H_DE1)
    g = ogrid.EnergyGrid(edges, NQ)
    _CPU_STATE = (g, synthetic.make_tables(g.eps, NS, seed=0),
                  osolver.Params(tol_inner=TOL, tol_outer=TOL, M_inner=MEM, M_outer=MEM))


def _cpu_worker_solve(chunk):
    from oracle import solver as osolver
    g, tables, prm = _CPU_STATE
    osolver.solve(g, tables, prm, chunk)
    return len(chunk["rho"])


def cpu_baseline(edges, tables, inp, gpu_out=None):
    """The oracle on the host cores, on the headline workload: one thread on its first CPU_SAMPLE
    nodes, then one single-threaded worker per core (spawned processes, nodes split evenly) on
    CPU_PER_CORE nodes per core.  With gpu_out (the mixed path's outputs for those nodes, numpy) the
    mixed path's error against the oracle on the one-thread sample is returned too."""
    from oracle import grid as ogrid, solver as osolver
    g = ogrid.EnergyGrid(edges, NQ)
    prm = osolver.Params(tol_inner=TOL, tol_outer=TOL, M_inner=MEM, M_outer=MEM)
    t0 = time.perf_counter()
    refs = osolver.solve(g, tables, prm, inp, nodes=range(CPU_SAMPLE))
    dt = time.perf_counter() - t0
    out = {"value": CPU_SAMPLE / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": f"first {CPU_SAMPLE} nodes of the headline workload, numpy FP64 oracle at tol 1e-10, "
                     f"one thread, {dt:.1f} s"}
    err = None
    if gpu_out is not None:
        ok = [n for n, r in enumerate(refs) if r["status"] == 0 and gpu_out["status"][n] == 0]
        eD = np.zeros(NS)
        eB = np.zeros(NS)
        ex = {"Ye": 0.0, "eps": 0.0, "T": 0.0}
        for n in ok:
            r = refs[n]
            ref = np.sqrt(np.sum(g.W2 * r["D"] ** 2, axis=-1))
            eD = np.maximum(eD, np.sqrt(np.sum(g.W2 * (gpu_out["J"][n] - r["D"]) ** 2, axis=-1)) / ref)
            fl = 1e-4 * np.max(np.abs(r["D"]), axis=-1, keepdims=True)
            eB = np.maximum(eB, np.max(np.abs(gpu_out["J"][n] - r["D"]) / np.maximum(np.abs(r["D"]), fl), axis=-1))
            for k in ex:
                ex[k] = max(ex[k], abs(gpu_out[k][n] - r[k]) / abs(r[k]))
        err = {"nodes": len(ok), "oracle_tol": TOL, "D_wnorm_by_species": eD.tolist(),
               "D_per_bin_by_species_floor_1e-4": eB.tolist(), **ex}
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cores = os.cpu_count() or 1
    nodes = min(cores * CPU_PER_CORE, len(inp["rho"]))
    chunks = [{k: v[i:nodes:cores] for k, v in inp.items()} for i in range(cores)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                 initializer=_cpu_worker_init) as ex:
            list(ex.map(_cpu_worker_solve, [{k: v[i:i + 1] for k, v in inp.items()} for i in range(cores)]))
            t0 = time.perf_counter()
            done = sum(ex.map(_cpu_worker_solve, chunks))
            dtp = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out["all_cores"] = {"value": done / dtp, "unit": "solves/s", "cores": cores, "kind": "oracle",
                        "sample": f"first {done} nodes of the headline workload, numpy FP64 oracle, one "
                                  f"single-threaded process per core, {dtp:.1f} s after a warm-up task per worker"}
    return out, err


def _measured_hbm_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json beside this file), else 6800 GB/s."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _measured_hbm_gbs()
# FMA-pipe peaks (TFLOP/s), measured by measure_peaks() at the start of a run
PEAKS = {"fp64": None, "fp32": None, "smem_gbs": None, "smem_relative_cost": None}
PEAK_NOTE = "measured: nmc_fma_probe (16 independent FMA chains per thread, full occupancy, CUDA events)"


def measure_peaks(stream, reps=5, warm=10):
    """FP64 and FP32 FMA-pipe peaks of this GPU (TFLOP/s): the best of `reps` timed launches of
    nmc_fma_probe after `warm` untimed ones (the clocks settle at their load value), each between
    CUDA events on `stream`."""
    import torch
    from paper_2601_00976_gb300 import nmc
    out = {}
    for name, prec, iters, dt in (("fp64", nmc.FP64, 2000, torch.float64), ("fp32", nmc.MIXED, 100000, torch.float32)):
        sink = torch.zeros(1, dtype=dt, device="cuda")
        for _ in range(warm):
            nmc.fma_probe(prec, iters, sink, stream=stream)
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = nmc.fma_probe(prec, iters, sink, stream=stream)
            e1.record(stream)
            e1.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    # shared-memory pipe: lane-consecutive 4-byte loads (128 bytes per warp load), GB/s, and the cost of
    # the other load kinds per warp load relative to it
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    per_load = {}
    for mode in range(5):
        for _ in range(3):
            nmc.smem_probe(mode, 200, sink, stream=stream)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            loads = nmc.smem_probe(mode, 200, sink, stream=stream)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3 / loads)
        per_load[mode] = best
    out["smem_gbs"] = 128.0 / per_load[nmc.SMEM_B32_CONSECUTIVE] / 1e9
    base = per_load[nmc.SMEM_B32_CONSECUTIVE]
    out["smem_relative_cost"] = {"b32_broadcast": per_load[nmc.SMEM_B32_BROADCAST] / base,
                                 "b64_broadcast": per_load[nmc.SMEM_B64_BROADCAST] / base,
                                 "b128_broadcast": per_load[nmc.SMEM_B128_BROADCAST] / base,
                                 "b128_consecutive": per_load[nmc.SMEM_B128_CONSECUTIVE] / base}
    return out


def _side(args):
    """(steps, warm-up steps) of the side measurements."""
    return max(1, min(args.steps, 5)), min(args.warmup, 2)


def _time_path(ctx, prm, t, out, steps, warmup, barrier, stream):
    import torch

    def step():
        ctx.collision_solve(prm, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], out=out)

    for _ in range(warmup):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    barrier()
    per_step = [a.elapsed_time(b) for a, b in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][1])
    return per_step, total_ms


def _fp64_roof(ach, kernel, n, fl, kern_ms):
    return {"bound": "alu", "achieved": ach, "peak": PEAKS["fp64"], "unit": "TFLOP/s",
            "frac": ach / PEAKS["fp64"], "traffic": _traffic(kernel, n), "kernel": kernel,
            "peak_source": "FP64 FMA pipe, " + PEAK_NOTE, "algorithmic_flops_per_launch": fl, "kernel_ms": kern_ms}


def time_velocity(args, ctx, eps, dev, rank, barrier, allmax, stream):
    """Time collision_solve_v (the O(v/c) solve, FP64) over the profile with an infall velocity field."""
    import torch
    from paper_2601_00976_gb300 import nmc, synthetic, flops
    from paper_2601_00976_gb300.dist import workload_seed, weak_scaling_value
    n = args.velocity_nodes
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    inp = synthetic.make_inputs("profile", n, eps, NS, seed=workload_seed(rank, 3))
    t = {k: torch.tensor(v, device=dev) for k, v in inp.items()}
    v = torch.tensor(synthetic.make_velocities("profile", n, seed=workload_seed(rank, 3)), device=dev)
    p = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM)
    out = ctx.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"])

    def step():
        ctx.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"], out=out)

    steps, warmup = _side(args)
    for _ in range(warmup):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    barrier()
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    total_ms = allmax(evs[0][0].elapsed_time(evs[-1][1]))
    n_in = out["n_inner"].cpu().numpy().astype(np.int64)
    n_out = out["n_outer"].cpu().numpy().astype(np.int64)
    fl = float(np.sum(flops.velocity_node_flops(NS, len(eps), N_ELEM, NQ, MEM, n_in, n_out)))
    ach = fl / (kern_ms * 1e-3) / 1e12
    vmag = torch.sqrt((v * v).sum(1))
    # the same solve with linear-order (Phi_1) NES and pair kernels in the tables
    edges, _ = _grid(N_ELEM, DE1)
    tl = synthetic.make_tables(ctx.energies, NS, seed=0, linear=True)
    ctx_l = nmc.Context(edges, NQ, NS, tl)
    out_l = ctx_l.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"])
    for _ in range(warmup):
        ctx_l.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"], out=out_l)
    barrier()
    evl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evl[k][0].record(stream)
        ctx_l.collision_solve_v(p, t["rho"], t["T"], t["Ye"], v, t["D"], t["I"], t["dt"], t["scale"], out=out_l)
        evl[k][1].record(stream)
    barrier()
    total_l = allmax(evl[0][0].elapsed_time(evl[-1][1]))
    linear = {"value": weak_scaling_value(ws * n, steps, total_l), "unit": "solves/s",
              "ms_per_step": total_l / steps,
              "converged_fraction": float((out_l["status"] == 0).float().mean().item()),
              "mean_inner_iters": float(out_l["n_inner"].float().mean().item()),
              "note": "tables with linear-order (Phi_1) NES and pair kernels; the kernel holds their matrices "
                      "next to the isotropic ones (one block per SM)"}
    ctx_l.close()
    return {"metric": "converged O(v/c) collision solves/s (nodes*steps/s)",
            "value": weak_scaling_value(ws * n, steps, total_ms), "unit": "solves/s",
            "ms_per_step": total_ms / steps, "dtype": "f64",
            "config": {"workload": VEL_WORKLOAD, "nodes_per_gpu": n, "max_speed_c": float(vmag.max().item()),
                       "converged_fraction": float((out["status"] == 0).float().mean().item()),
                       "mean_inner_iters": float(n_in.mean()), "mean_outer_iters": float(n_out.mean())},
            "roofline": _fp64_roof(ach, "velocity_kernel", n, fl, kern_ms),
            "linear_phi1": linear}


def time_relaxation(args, dev, rank, barrier, allmax):
    """The relaxation problem of Sec. 6.1 (six species, v = 0.1 c, dt x1.04 per step to 100 ms: 271 steps),
    batched over problems with seeded +-10% perturbations of (rho, T, Ye), through the backward-Euler driver."""
    import torch
    from paper_2601_00976_gb300 import nmc, synthetic, relaxation
    from paper_2601_00976_gb300.dist import workload_seed
    n = args.relaxation_problems
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    edges, eps = _grid(N_ELEM, DE1)
    tables = synthetic.make_tables(eps, 6, seed=81)
    ctx = nmc.Context(edges, NQ, 6, tables)
    rng = np.random.default_rng(workload_seed(rank, 5))
    f64 = dict(dtype=torch.float64, device=dev)
    rho = torch.tensor(1e12 * rng.uniform(0.9, 1.1, n), **f64)
    T = torch.tensor(7.6 * rng.uniform(0.9, 1.1, n), **f64)
    Ye = torch.tensor(0.135 * rng.uniform(0.9, 1.1, n), **f64)
    v = torch.zeros((n, 3), **f64)
    v[:, 0] = 0.1
    D0, I0 = relaxation.initial_moments(ctx.energies, 6, 7.6)
    D = torch.tensor(np.broadcast_to(D0, (n,) + D0.shape).copy(), **f64)
    I = torch.tensor(np.broadcast_to(I0, (n,) + I0.shape).copy(), **f64)
    p = nmc.default_params(tol_inner=1e-8, tol_outer=1e-8, m_inner=2, m_outer=2, max_inner=1000, max_outer=200)
    steps = relaxation.schedule()
    rel = relaxation.Relaxation(ctx, p, rho, T, Ye, v, D, I)
    L0, E0 = rel.totals()
    barrier()
    t0 = time.perf_counter()
    rel.run(steps)
    torch.cuda.synchronize()
    barrier()
    wall = allmax(time.perf_counter() - t0)
    L1, E1 = rel.totals()
    ok = rel.state["status"] == 0
    out = {"metric": "relaxation problem-steps/s (problems*steps/s)", "value": ws * n * len(steps) / wall,
           "unit": "problem-steps/s", "s_per_run": wall, "dtype": "f64",
           "config": {"workload": REL_WORKLOAD, "problems_per_gpu": n, "steps": len(steps),
                      "converged_fraction_last_step": float(ok.float().mean().item()),
                      "max_rel_change_total_lepton_number": float((torch.abs(L1 - L0) / torch.abs(L0)).max().item()),
                      "max_rel_change_total_energy": float((torch.abs(E1 - E0) / torch.abs(E0)).max().item())}}
    ctx.close()
    return out


def time_c2p(args, ctx, eps, dev, rank, barrier, allmax, stream):
    """Time conserved_to_primitive (FP64) on every bin of the profile with an infall velocity field."""
    import torch
    from paper_2601_00976_gb300 import synthetic, flops
    from paper_2601_00976_gb300.dist import workload_seed, weak_scaling_value
    n = args.c2p_nodes
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    inp = synthetic.make_inputs("profile", n, eps, NS, seed=workload_seed(rank, 4))
    # conserved moments of the same shape and realizability as the profile's primitive ones
    N = torch.tensor(inp["D"], device=dev)
    G = torch.tensor(inp["I"], device=dev)
    v = torch.tensor(synthetic.make_velocities("profile", n, seed=workload_seed(rank, 4)), device=dev)
    out = ctx.conserved_to_primitive(N, G, v)

    def step():
        ctx.conserved_to_primitive(N, G, v, out=out)

    steps, warmup = _side(args)
    for _ in range(warmup):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    barrier()
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    total_ms = allmax(evs[0][0].elapsed_time(evs[-1][1]))
    it = out["iters"].cpu().numpy().astype(np.int64)
    bins = it.size
    fl = float(np.sum(flops.c2p_bin_flops(it)))
    ach = fl / (kern_ms * 1e-3) / 1e12
    byts = bins * C2P_BYTES_PER_BIN + n * 24
    return {"metric": "conserved-to-primitive recoveries/s (bins*steps/s)",
            "value": weak_scaling_value(ws * bins, steps, total_ms), "unit": "bins/s",
            "ms_per_step": total_ms / steps, "dtype": "f64",
            "config": {"workload": C2P_WORKLOAD, "nodes_per_gpu": n, "bins_per_gpu": bins,
                       "mean_iters": float(it.mean()), "max_iters": int(it.max()),
                       "converged_fraction": float((out["status"] == 0).float().mean().item()),
                       "hbm_gbs_algorithmic": byts / (kern_ms * 1e-3) / 1e9},
            "roofline": _fp64_roof(ach, "c2p_kernel", n, fl, kern_ms)}


def time_interp(args, ctx, eps, dev, rank, barrier, allmax, stream):
    """Time opacity_interp (FP64): chi_EmAb and sigma_Iso of every species at scattered points."""
    import torch
    from paper_2601_00976_gb300 import synthetic, flops
    from paper_2601_00976_gb300.dist import workload_seed, weak_scaling_value
    P = args.interp_points
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    pts = {k: torch.tensor(v, device=dev) for k, v in synthetic.make_interp_points(P, eps, seed=workload_seed(rank, 5)).items()}
    outs = [torch.empty(P, dtype=torch.float64, device=dev) for _ in range(2 * NS)]
    launches = [(which, sp) for which in (0, 1) for sp in range(NS)]

    def step():
        for k, (which, sp) in enumerate(launches):
            ctx.opacity_interp(which, sp, pts["rho"], pts["T"], pts["Ye"], pts["E"], out=outs[k])

    steps, warmup = _side(args)
    for _ in range(warmup):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    barrier()
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in evs) / len(launches)
    total_ms = allmax(evs[0][0].elapsed_time(evs[-1][1]))
    finite = all(bool(torch.isfinite(o).all().item()) and bool((o > 0).all().item()) for o in outs)
    # the FP32 entry point on the same points: bound by the bytes it moves (HBM)
    outm = [torch.empty(P, dtype=torch.float64, device=dev) for _ in range(2 * NS)]

    def step_m():
        for k, (which, sp) in enumerate(launches):
            ctx.opacity_interp(which, sp, pts["rho"], pts["T"], pts["Ye"], pts["E"], out=outm[k], mixed=True)

    for _ in range(warmup):
        step_m()
    barrier()
    evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evm[k][0].record(stream)
        step_m()
        evm[k][1].record(stream)
    barrier()
    launch_mm = statistics.mean(a.elapsed_time(b) for a, b in evm) / len(launches)
    total_mm = allmax(evm[0][0].elapsed_time(evm[-1][1]))
    rel = max(float((torch.abs(a - b) / b).max().item()) for a, b in zip(outm, outs))
    gbs_m = INTERP_BYTES_PER_POINT * P / (launch_mm * 1e-3) / 1e9
    mixed = {"value": weak_scaling_value(ws * P * len(launches), steps, total_mm), "unit": "points/s",
             "ms_per_step": total_mm / steps, "launch_ms": launch_mm, "max_rel_diff_vs_fp64_entry": rel,
             "roofline": {"bound": "hbm", "achieved": gbs_m, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                          "frac": gbs_m / HBM_PEAK_GBS, "traffic": _traffic("opacity_interp_mixed_kernel", P),
                          "kernel": "opacity_interp_mixed_kernel",
                          "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
                          "algorithmic_bytes_per_launch": INTERP_BYTES_PER_POINT * P, "kernel_ms": launch_mm}}
    fl = flops.interp_point_flops() * P
    ach = fl / (launch_ms * 1e-3) / 1e12
    gbs = INTERP_BYTES_PER_POINT * P / (launch_ms * 1e-3) / 1e9
    return {"metric": "interpolated opacities/s (points*launches*steps/s)",
            "value": weak_scaling_value(ws * P * len(launches), steps, total_ms), "unit": "points/s",
            "ms_per_step": total_ms / steps, "dtype": "f64",
            "config": {"workload": INTERP_WORKLOAD, "points_per_gpu": P, "launches_per_step": len(launches),
                       "all_values_finite_positive": finite,
                       "hbm_gbs_algorithmic": gbs, "hbm_frac_of_measured": gbs / HBM_PEAK_GBS},
            "roofline": _fp64_roof(ach, "opacity_interp_kernel", P, fl, launch_ms),
            "mixed": mixed}


def time_adjoint(args, ctx, eps, dev, rank, barrier, allmax, stream):
    """Time collision_adjoint over the adjoint workload (inputs and cotangents resident in HBM)."""
    import torch
    from paper_2601_00976_gb300 import nmc, synthetic, flops
    n = args.adjoint_nodes
    from paper_2601_00976_gb300.dist import workload_seed, weak_scaling_value
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    inp = synthetic.make_inputs("profile", n, eps, NS, seed=workload_seed(rank, 1))
    t = {k: torch.tensor(v, device=dev) for k, v in inp.items()}
    p = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM)
    fw = ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    gen = torch.Generator(device=dev).manual_seed(77 + rank)
    f64 = dict(dtype=torch.float64, device=dev, generator=gen)
    ct = dict(gJ=torch.randn(t["D"].shape, **f64), gH=torch.randn(t["I"].shape, **f64),
              gYe=torch.randn(n, **f64), geps=torch.randn(n, **f64) * 1e-19, gT=torch.randn(n, **f64))
    out = ctx.collision_adjoint(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], fw["J"], fw["T"],
                                **ct)

    def step():
        ctx.collision_adjoint(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], fw["J"], fw["T"],
                              out=out, **ct)

    steps, warmup = _side(args)
    for _ in range(warmup):
        step()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    barrier()
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    total_ms = allmax(evs[0][0].elapsed_time(evs[-1][1]))
    clean = int(torch.count_nonzero((out["status"] & ~nmc.TABLE_CLAMP) == 0).item())
    fl = flops.adjoint_flops(NS, len(eps), N_ELEM, NQ) * n
    ach = fl / (kern_ms * 1e-3) / 1e12
    return {"metric": "node gradients/s (nodes*steps/s)", "value": weak_scaling_value(ws * n, steps, total_ms),
            "unit": "nodes/s", "ms_per_step": total_ms / steps, "dtype": "f64",
            "config": {"workload": ADJ_WORKLOAD, "nodes_per_gpu": n, "clean_fraction": clean / n},
            "roofline": _fp64_roof(ach, "adjoint_kernel", n, fl, kern_ms)}


def time_batching(args, ctx, eps, dev, rank, barrier, allmax, stream):
    """The uneven core/tail batch: persistent FP64 kernel (autotuned, CUDA-graph replay), mixed persistent
    kernel and plain FP64 per-iteration launches on the same inputs, `--batching-steps` timed steps each."""
    import torch
    from paper_2601_00976_gb300 import nmc, synthetic
    from paper_2601_00976_gb300.dist import workload_seed
    n = args.batching_nodes
    K = max(1, args.batching_steps)
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    inp = synthetic.make_inputs("core_tail", n, eps, NS, seed=workload_seed(rank, 2))
    t = {k: torch.tensor(v, device=dev) for k, v in inp.items()}
    del inp
    sub = {k: v[: min(n, 1 << 16)].contiguous() for k, v in t.items()}
    p = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM)
    pm = nmc.default_params(tol_inner=MIXED_TOL[0], tol_outer=MIXED_TOL[1], m_inner=MEM, m_outer=MEM,
                            precision=nmc.MIXED)
    pp = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM, mode=nmc.MODE_PLAIN)
    minb, pct, _ = ctx.autotune(p, sub["rho"], sub["T"], sub["Ye"], sub["D"], sub["I"], sub["dt"], sub["scale"])
    minbm, pctm, _ = ctx.autotune(pm, sub["rho"], sub["T"], sub["Ye"], sub["D"], sub["I"], sub["dt"], sub["scale"])
    ctx.collision_solve(pp, sub["rho"], sub["T"], sub["Ye"], sub["D"], sub["I"], sub["dt"], sub["scale"])
    f64 = dict(dtype=torch.float64, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)

    def outputs():
        return dict(J=torch.empty_like(t["D"]), H=torch.empty_like(t["I"]), Ye=torch.empty(n, **f64),
                    eps=torch.empty(n, **f64), T=torch.empty(n, **f64), n_outer=torch.empty(n, **i32),
                    n_inner=torch.empty(n, **i32), status=torch.empty(n, **i32))
    out, outm, outp = outputs(), outputs(), outputs()
    barrier()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            ctx.collision_solve(p, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"], out=out)
    barrier()
    res = {}
    arms = (("persistent", lambda: graph.replay()),
            ("mixed", lambda: ctx.collision_solve(pm, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"],
                                                  out=outm)),
            ("plain", lambda: ctx.collision_solve(pp, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"],
                                                  t["scale"], out=outp)))
    for name, step in arms:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        barrier()
        res[name] = allmax(e0.elapsed_time(e1)) / K
    ni = out["n_inner"].cpu().numpy()
    st = {k: o["status"].cpu().numpy() for k, o in (("persistent", out), ("mixed", outm), ("plain", outp))}
    counts = {k: {str(int(u)): int(c) for u, c in zip(*np.unique(v, return_counts=True))} for k, v in st.items()}
    same_status = float(np.mean(st["persistent"] == st["plain"]))
    w2 = torch.tensor(ctx.w2, device=dev)
    ok = (out["status"] == 0) & (outm["status"] == 0)
    refn = torch.sqrt(torch.sum(w2 * out["J"][ok] ** 2, dim=-1))
    dmax = float(torch.max(torch.sqrt(torch.sum(w2 * (out["J"] - outp["J"])[ok] ** 2, dim=-1)) / refn).item())
    emx = torch.sqrt(torch.sum(w2 * (outm["J"] - out["J"])[ok] ** 2, dim=-1)) / refn
    conv = {k: int(np.count_nonzero(v == 0)) for k, v in st.items()}
    rate = {k: ws * conv[k] / (res[k] * 1e-3) for k in res}
    return {"metric": "converged collision solves/s (nodes*steps/s)", "unit": "solves/s", "dtype": "f64",
            "config": {"workload": f"core/tail mix, {n} nodes (half rho > 1e13, half rho < 1e10), dt log-uniform "
                                   "1e-7..1e-5 s, 4 species, Grid C 16x2, all processes, Anderson depth 3, "
                                   "FP64 tol 1e-10, mixed tol 1e-10 (inner) and 1e-9 (outer)",
                       "nodes_per_gpu": n, "timed_steps_per_arm": K,
                       "inner_iters_min": int(ni.min()), "inner_iters_max": int(ni.max()),
                       "inner_iters_mean": float(ni.mean()),
                       "tuned_variant": {"fp64": {"blocks_per_sm": minb, "grid_pct": pct},
                                         "mixed": {"blocks_per_sm": minbm, "grid_pct": pctm}},
                       "status_counts": counts, "status_agreement_persistent_plain": same_status,
                       "max_rel_J_difference_persistent_plain": dmax,
                       "mixed_max_rel_J_error_vs_fp64_by_species": emx.max(dim=0).values.tolist()},
            "persistent_graph": {"value": rate["persistent"], "ms_per_step": res["persistent"]},
            "mixed_persistent": {"value": rate["mixed"], "ms_per_step": res["mixed"]},
            "plain_per_iteration": {"value": rate["plain"], "ms_per_step": res["plain"]},
            "speedup_persistent_vs_plain": rate["persistent"] / rate["plain"],
            "speedup_mixed_persistent_vs_plain_fp64": rate["mixed"] / rate["plain"]}


def _host_step_bytes(host, out):
    return (sum(v.numel() * v.element_size() for v in host.values()),
            sum(v.numel() * v.element_size() for v in out.values()))


def run_nmc(args):
    import torch
    from paper_2601_00976_gb300 import nmc, flops
    from paper_2601_00976_gb300.dist import Group, workload_seed, weak_scaling_value
    global PEAKS
    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", torch.cuda.current_device())
    group = Group(dev)
    barrier, allmax, allsum = group.barrier, group.allmax, group.allsum
    stream = torch.cuda.current_stream()

    # ---------------- headline: mixed persistent solve of the 64-energy perturbed batch ----------------
    edges, eps, tables, inp = _workload(workload_seed(rank, 0), args.nodes)
    ne = len(eps)
    ctx = nmc.Context(edges, NQ, NS, tables)
    t = {k: torch.tensor(v, device=dev) for k, v in inp.items()}
    p64 = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM)
    pmx = nmc.default_params(tol_inner=MIXED_TOL[0], tol_outer=MIXED_TOL[1], m_inner=MEM, m_outer=MEM,
                             precision=nmc.MIXED)
    ppl = nmc.default_params(tol_inner=TOL, tol_outer=TOL, m_inner=MEM, m_outer=MEM, mode=nmc.MODE_PLAIN)
    # the autotuner picks the fused kernel's variant for each precision on a slice of the batch (untimed)
    sub = {k: v[: min(args.nodes, 1 << 17)].contiguous() for k, v in t.items()}
    tuned = {}
    for name, prm in (("mixed", pmx),) + ((("fp64", p64),) if args.compare_steps > 0 else ()):
        minb, pct, _ = ctx.autotune(prm, sub["rho"], sub["T"], sub["Ye"], sub["D"], sub["I"], sub["dt"], sub["scale"])
        tuned[name] = {"blocks_per_sm": minb, "grid_pct": pct}
    del sub
    # the FMA-pipe peaks, measured with the GPU warm (after the autotuner's launches)
    PEAKS = measure_peaks(stream)
    omx = ctx.collision_solve(pmx, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    per_step, total_ms = _time_path(ctx, pmx, t, omx, args.steps, args.warmup, barrier, stream)
    clk.stop()

    def summary(out, per, tot):
        n_in = out["n_inner"].cpu().numpy().astype(np.int64)
        n_out = out["n_outer"].cpu().numpy().astype(np.int64)
        status = out["status"].cpu().numpy()
        fl = float(np.sum(flops.node_flops(NS, ne, H_ELEM, NQ, MEM, n_in, n_out)))
        fl64 = float(np.sum(flops.mixed_fp64_flops(NS, ne, n_out)))
        return dict(total_ms=allmax(tot), kern_ms=statistics.mean(per), flops=fl, flops_fp64_share=fl64,
                    n_in=n_in, n_out=n_out, converged=allsum(int(np.count_nonzero(status == 0))),
                    status_counts={str(int(u)): int(c) for u, c in zip(*np.unique(status, return_counts=True))})
    rmx = summary(omx, per_step, total_ms)

    # ---------------- FP64 persistent and plain FP64 launches on the same inputs ----------------
    r64 = rpl = None
    err = None
    if args.compare_steps > 0:
        o64 = ctx.collision_solve(p64, t["rho"], t["T"], t["Ye"], t["D"], t["I"], t["dt"], t["scale"])
        per, tot = _time_path(ctx, p64, t, o64, args.compare_steps, 0, barrier, stream)
        r64 = summary(o64, per, tot)
        # the plain kernels' first launches on a slice (untimed), then the batch
        ctx.collision_solve(ppl, t["rho"][:256], t["T"][:256], t["Ye"][:256], t["D"][:256], t["I"][:256],
                            t["dt"][:256], t["scale"][:256])
        opl = {k: torch.empty_like(v) for k, v in o64.items()}
        per, tot = _time_path(ctx, ppl, t, opl, args.compare_steps, 0, barrier, stream)
        rpl = summary(opl, per, tot)
        # accuracy of the mixed path against the FP64 path on the same inputs (every node both converged)
        ok = (o64["status"] == 0) & (omx["status"] == 0)
        wt = torch.tensor(ctx.w2, device=dev)
        ref = torch.sqrt(torch.sum(wt * o64["J"][ok] ** 2, dim=-1))
        eD = torch.sqrt(torch.sum(wt * (omx["J"] - o64["J"])[ok] ** 2, dim=-1)) / ref
        rD = o64["J"][ok]
        fl_ = 1e-4 * rD.abs().amax(dim=-1, keepdim=True)
        eB = ((omx["J"][ok] - rD).abs() / torch.maximum(rD.abs(), fl_)).amax(dim=(0, 2))
        err = {"nodes_compared": int(ok.sum().item()), "fp64_tol": TOL,
               "D_wnorm_by_species": eD.max(dim=0).values.tolist(), "D_per_bin_by_species_floor_1e-4": eB.tolist()}
        for k in ("Ye", "eps", "T"):
            err[k] = float((torch.abs(omx[k] - o64[k]) / torch.abs(o64[k]))[ok].max().item())
        del o64, opl

    # ---------------- end to end: host buffers, copies inside the timed region ----------------
    e2e = None
    if not args.no_e2e:
        host = {k: torch.tensor(v).pin_memory() for k, v in inp.items()}
        hout = ctx.host_outputs(args.nodes)
        h2d, d2h = _host_step_bytes(host, hout)
        ctx.collision_solve_host(pmx, host, hout)   # warm-up: staging buffers and streams
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.collision_solve_host(pmx, host, hout)
        barrier()
        e2e_s = allmax((time.perf_counter() - t0) / args.steps)
        conv = allsum(int((hout["status"] == 0).sum().item()))
        e2e = {"value": conv / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": args.steps,
               "pipeline": "collision_solve_host: chunks of the batch, H2D / solve / D2H on three streams"}
        del host, hout
    gpu_sample = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        gpu_sample = {k: v[:CPU_SAMPLE].cpu().numpy() for k, v in omx.items()}
    ctx.close()
    del t, omx
    inp_head = {k: v[: CPU_SAMPLE + 16 * CPU_PER_CORE * 2] for k, v in inp.items()}
    del inp
    torch.cuda.empty_cache()

    # ---------------- side measurements on Grid C (32 energies) ----------------
    edges_c, eps_c = _grid(N_ELEM, DE1)
    from paper_2601_00976_gb300 import synthetic
    ctxc = nmc.Context(edges_c, NQ, NS, synthetic.make_tables(eps_c, NS, seed=0))
    vel = time_velocity(args, ctxc, eps_c, dev, rank, barrier, allmax, stream) if args.velocity_nodes > 0 else None
    c2p = time_c2p(args, ctxc, eps_c, dev, rank, barrier, allmax, stream) if args.c2p_nodes > 0 else None
    itp = time_interp(args, ctxc, eps_c, dev, rank, barrier, allmax, stream) if args.interp_points > 0 else None
    rlx = time_relaxation(args, dev, rank, barrier, allmax) if args.relaxation_problems > 0 else None
    adj = time_adjoint(args, ctxc, eps_c, dev, rank, barrier, allmax, stream) if args.adjoint_nodes > 0 else None
    torch.cuda.empty_cache()
    bat = (time_batching(args, ctxc, eps_c, dev, rank, barrier, allmax, stream)
           if args.batching_nodes > 0 and ws == 1 else None)
    ctxc.close()

    cpu = oracle_err = None
    if gpu_sample is not None:
        cpu, oracle_err = cpu_baseline(edges, tables, inp_head, gpu_sample)
    if rank == 0:
        def line_value(r, steps):   # converged nodes of every rank per step, over the slowest rank's time
            return weak_scaling_value(r["converged"], steps, r["total_ms"])

        def roof64(r):
            ach = r["flops"] / (r["kern_ms"] * 1e-3) / 1e12
            return {"bound": "alu", "achieved": ach, "peak": PEAKS["fp64"], "unit": "TFLOP/s",
                    "frac": ach / PEAKS["fp64"], "traffic": _traffic("fused_kernel<double>", args.nodes),
                    "kernel": "fused_kernel<double>", "peak_source": "FP64 FMA pipe, " + PEAK_NOTE,
                    "algorithmic_flops_per_launch": r["flops"], "kernel_ms": r["kern_ms"]}

        # mixed path: bound time = FP32 work / FP32 peak + FP64 work / FP64 peak (both measured); the
        # peak reported is the rate that bound implies for this launch's work
        f64w = rmx["flops_fp64_share"]
        f32w = rmx["flops"] - f64w
        t_bound = (f32w / (PEAKS["fp32"] * 1e12) + f64w / (PEAKS["fp64"] * 1e12))
        ach = rmx["flops"] / (rmx["kern_ms"] * 1e-3) / 1e12
        peff = rmx["flops"] / t_bound / 1e12
        roofmx = {"bound": "alu", "achieved": ach, "peak": peff, "unit": "TFLOP/s", "frac": ach / peff,
                  "traffic": _traffic("fused_kernel<float>", args.nodes), "kernel": "fused_kernel<float>",
                  "peak_source": ("FP32 and FP64 FMA pipes, " + PEAK_NOTE + f": {PEAKS['fp32']:.1f} and "
                                  f"{PEAKS['fp64']:.3f} TFLOP/s; bound time = FP32 work / FP32 peak + FP64 work "
                                  "/ FP64 peak over the launch's algorithmic work"),
                  "algorithmic_flops_per_launch": rmx["flops"], "algorithmic_fp64_flops_per_launch": f64w,
                  "bound_ms": t_bound * 1e3, "kernel_ms": rmx["kern_ms"]}
        # the contraction loop's own bound: every inner iteration reads each node's kernel matrices from
        # shared memory, K_Out of each species twice (rows and columns) and K_Ann of each pair by both of
        # its species, 12 ns ne^2 bytes in FP32, against the shared-memory pipe's rate measured by
        # nmc_smem_probe (lane-consecutive 4-byte loads, one 128-byte wavefront per warp load)
        clk_sum = clk.summary()
        smem_bytes = float(rmx["n_in"].sum()) * 12.0 * NS * ne * ne
        smem_ach = smem_bytes / (rmx["kern_ms"] * 1e-3) / 1e9
        roof_smem = {"bound": "smem", "achieved": smem_ach, "peak": PEAKS["smem_gbs"], "unit": "GB/s",
                     "frac": smem_ach / PEAKS["smem_gbs"], "kernel": "fused_kernel<float>",
                     "algorithmic_bytes_per_launch": smem_bytes,
                     "model": "kernel-matrix operands of the inner iterations (12 ns ne^2 bytes per node-iteration)",
                     "peak_source": "measured: nmc_smem_probe, lane-consecutive 4-byte loads (CUDA events)",
                     "probe_cost_per_warp_load_relative_to_one_wavefront": PEAKS["smem_relative_cost"]}
        value = line_value(rmx, args.steps)
        cfg = {"workload": WORKLOAD, "precision": "mixed", "nodes_per_gpu": args.nodes,
               "l2": "inputs_larger_than_l2", "tolerances": {"fp64": [TOL, TOL], "mixed": list(MIXED_TOL)},
               "mixed_solves_per_s": value, "status_counts_mixed": rmx["status_counts"],
               "mean_inner_iters": float(rmx["n_in"].mean()), "mean_outer_iters": float(rmx["n_out"].mean()),
               "max_inner_iters": int(rmx["n_in"].max()), "tuned_variants": tuned,
               "converged_fraction": rmx["converged"] / (ws * args.nodes)}
        if r64 is not None:
            v64, vpl = line_value(r64, args.compare_steps), line_value(rpl, args.compare_steps)
            cfg.update({"fp64_persistent_solves_per_s": v64, "fp64_plain_solves_per_s": vpl,
                        "status_counts_fp64": r64["status_counts"], "status_counts_fp64_plain": rpl["status_counts"],
                        "fp64_timed_steps": args.compare_steps,
                        "speedup_mixed_vs_fp64_persistent": value / v64,
                        "speedup_mixed_persistent_vs_plain_fp64": value / vpl,
                        "speedup_fp64_persistent_vs_plain": v64 / vpl,
                        "mixed_max_rel_error_vs_fp64": err})
        if oracle_err is not None:
            cfg["mixed_max_rel_error_vs_oracle"] = oracle_err
        line = {
            "metric": METRIC,
            "value": value, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": rmx["total_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": cfg,
            "roofline": roofmx,
            "roofline_smem": roof_smem,
            "roofline_fp64": roof64(r64) if r64 is not None else None,
            "peaks_measured": {"fp64_tflops": PEAKS["fp64"], "fp32_tflops": PEAKS["fp32"], "how": PEAK_NOTE,
                               "smem_gbs": PEAKS["smem_gbs"]},
            "gpu_launches": args.steps,
            "clocks": clk_sum,
        }
        if e2e is not None:
            line["e2e"] = e2e
        for key, obj in (("velocity", vel), ("c2p", c2p), ("opacity_interp", itp), ("relaxation", rlx),
                         ("adjoint", adj), ("batching", bat), ("cpu_baseline", cpu)):
            if obj is not None:
                line[key] = obj
        print(json.dumps(line), flush=True)
    group.close()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nmc(args)


if __name__ == "__main__":
    main()
