"""Benchmark of the GB300 Poisson MaZe step (one JSON line on rank 0).

A step is one full MaZe MD step (S1-S9) of one synthetic molten-NaCl box.
Default workload: 1000 ions (500 Na+, 500 Cl-), L = 31.5 Angstrom, 32^3 grid,
1200 K, dt = 1 fs, constraint tolerance 1e-10, cubic B-spline assignment,
warm-started multigrid constraint solve in mixed precision (FP32 V-cycle,
double-float outer iteration, exact integer reductions). Inputs are resident
in HBM when the timed region starts; L2 is flushed (256 MiB write) between
timed steps, outside the per-step CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload nacl64|nacl1000|nacl512000|batch128|serve]
                  [--solver cg|mg] [--precision fp64|mixed]

--workload batch128 advances 128 replica boxes (216-4096 ions, 16^3-48^3
grids) together, one persistent kernel launch per step; --workload serve runs
the continuous-batching serving loop on a Poisson request stream.

Under torchrun every rank runs an independent replica box (weak scaling, no
collective on the data path); value = steps of all ranks / max rank time.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

if "reference" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2505_20418_gb300 import synth  # noqa: E402

METRIC = "MaZe steps/s, solve GB/s vs HBM peak, p50/p99 step latency at stated force error"
KERNELS_PER_STEP_CELLS = 7    # move, spread, 3 cell-list kernels, solve, forces
KERNELS_PER_STEP_NOCELLS = 4
KERNELS_PER_STEP_FUSED = 2     # mixed precision up to 64^3, no cell list: S1-S6 in one cluster launch, the forces
KERNELS_PER_STEP_SPLIT = 4     # mixed up to 64^3 with a cell list: S1-S3, S8 beside the solve, S7/S9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def mg_levels(N):
    sizes = [N]
    while sizes[-1] % 2 == 0 and sizes[-1] >= 8:
        sizes.append(sizes[-1] // 2)
    return sizes


def solve_bytes_per_launch(N, iters, solver="cg", nu=(2, 2), precision="fp64"):
    """Algorithmic DRAM bytes of one solve launch (one pass per vector touch).

    FP64 (8 B per value). Common: S4 pass 56 B/pt (read phi^k, phi^{k-1}, q,
    y; write phi_p, sigma_p, r) and the S6 correction 32 B/pt (read phi_p, y;
    write phi, y). CG: 64 B/pt per iteration (read r, p, write p; read p, y,
    r, write y, r) plus 24 B/pt for the true-residual confirmation. MG, per
    V-cycle and level of n_l points: 32 B/pt per red-black sweep (x read
    twice, b read, x written), residual 24 B/pt, full weighting 9 B/pt,
    prolongation to black points 9 B/pt; coarsest solve 16 B/pt; residual
    check on the finest level 16 B/pt.

    Mixed (double-float pairs of 8 B for phi, y, sigma_p; FP32 V-cycle):
    S4 40 B/pt (read phi^k, phi^{k-1}, q; write phi_p, sigma_p); per
    residual check 20 B/pt (read y, sigma_p; write r in FP32); per V-cycle
    level 16 B/pt per sweep, 12 residual, 4.5 restriction, 4.5
    prolongation; per update 20 B/pt (read y, e; write y); S6 40 B/pt (mean of
    y, then read y, phi_p; write y, phi)."""
    ng = N ** 3
    lv = mg_levels(N)
    if precision == "mixed":
        per_v = sum(n ** 3 * ((nu[0] + nu[1]) * 16 + 12 + 4.5 + 4.5) for n in lv[:-1]) + lv[-1] ** 3 * 8
        return ng * (40 + 40) + (iters + 1) * ng * 20 + iters * (per_v + ng * 20)
    base = ng * (56 + 32)
    if solver == "cg":
        return base + ng * (64 * iters + 24)
    per_v = sum(n ** 3 * ((nu[0] + nu[1]) * 32 + 24 + 9 + 9) for n in lv[:-1]) + lv[-1] ** 3 * 16 + ng * 16
    return base + per_v * iters


def run_cpu_baseline(w, solver="mg", budget_s=15.0):
    """The FP64 oracle as it stands, on a bounded sample of the same workload."""
    import oracle as O
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order, solver=solver)
    st = O.init(pos, vel, types, p, tf)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        st = O.step(st, p, tf)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} MD steps of the same {w.n_ions}-ion {w.N}^3 box from its initial state, "
                      f"numpy FP64, single thread ({dt:.1f} s)"}


def bench_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle as O
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order, solver=args.solver)
    st = O.init(pos, vel, types, p, tf)
    for _ in range(args.warmup):
        st = O.step(st, p, tf)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = O.step(st, p, tf)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, args),
            "p50_us": 1e6 * float(np.percentile(times, 50)), "p99_us": 1e6 * float(np.percentile(times, 99)),
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed MD steps after {args.warmup} warm-up steps of the "
                                       f"{w.n_ions}-ion {w.N}^3 box, numpy FP64, one host thread"},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def replica_workload(name, rank):
    """The box a rank advances: same workload, independent seed per rank
    (replicas shard one per GPU with no collective on the data path)."""
    w = synth.workload(name)
    w.seed = w.seed + rank
    return w


def max_over_ranks(x, dist=None, device="cpu"):
    """Max of a per-rank float over all ranks (identity on one rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, steps_per_rank, rank_seconds):
    """Whole-job throughput of independent replicas: all ranks' steps divided
    by the slowest rank's time."""
    return world * steps_per_rank / rank_seconds


def config_dict(w, args):
    return {"workload": f"molten NaCl {w.n_ions} ions, L={w.L} A, {w.N}^3 grid, {w.T:.0f} K, dt={w.dt} fs, "
                        f"tol={w.tol:g}, P={w.order}, r_cut={w.rc} A",
            "n_ions": w.n_ions, "grid": w.N, "solver": args.solver, "precision": args.precision,
            "l2": "flushed between timed steps and before each timed e2e exchange (256 MiB write outside "
                  "the timing)"}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# roofline kernel, from one ncu capture of the kernels as they stand; the
# command and the other counters are in the named summary under profiles/.
# A kernel changed after its capture must drop its entry (traffic null).
MEASURED_TRAFFIC = {
    ("nacl1000", "k_mixed_cluster", "mixed", "mg"): (1195520, "profiles/k_mixed_cluster_nacl1000.md"),
    ("nacl512000", "k_mixed_grid", "mixed", "mg"): (10840736000, "profiles/k_mixed_grid_nacl512000.md"),
}


def measured_traffic(workload, kernel, precision, solver):
    hit = MEASURED_TRAFFIC.get((workload, kernel, precision, solver))
    return None if hit is None else hit[0]


def has_cells(w):
    """True when the box takes the cell list (at least 3 cells of r_cut a side)."""
    return int(np.floor(w.L / w.rc)) >= 3


def solve_kernel_name(args, w):
    """The solve kernel a step launches for this precision, solver and grid."""
    if args.precision == "mixed":
        if w.N > 64:
            return "k_mixed_grid"
        return "k_mixed_cluster" if has_cells(w) else "k_cluster_step"
    return "k_mg_solve" if args.solver == "mg" else "k_cg_solve"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nacl1000",
                    choices=["nacl64", "nacl1000", "nacl64000", "nacl512000", "batch128", "serve", "study"])
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--boxes", type=int, default=128, help="batch128: number of replica boxes")
    ap.add_argument("--cluster-ctas", type=int, default=0, help="batch128: CTAs per box (0: autotune)")
    ap.add_argument("--solver", default="mg", choices=["cg", "mg"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "batch128":
        if args.impl == "reference":
            return bench_batch_reference(args)
        return bench_batch(args)
    if args.workload == "study":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the iteration study is a GPU measurement; the "
                              "oracle's iteration counts are pinned in tests/test_oracle_pins.py"}), flush=True)
            return None
        return bench_study(args)
    if args.workload == "serve":
        if args.impl == "reference":
            return bench_serve_reference(args)
        return bench_serve(args)
    w = synth.workload(args.workload)
    if args.impl == "reference":
        return bench_reference(args, w)

    import torch
    import torch.distributed as dist
    from paper_2505_20418_gb300 import maze as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M.load()

    # every rank advances its own replica (independent seed)
    w = replica_workload(args.workload, rank)
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    stream = torch.cuda.Stream(device=dev)
    solver = M.MAZE_SOLVER_MG if args.solver == "mg" else M.MAZE_SOLVER_CG
    precision = M.MAZE_MIXED if args.precision == "mixed" else M.MAZE_FP64
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order,
                    solver=solver, precision=precision, stream=stream.cuda_stream)
    sim.set_timing(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s0 = sim.stats()
    for _ in range(args.warmup):
        sim.step_async(1)
    torch.cuda.synchronize()
    s1 = sim.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    solve_ms = []
    phase_ms = []
    timing_error = None
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    it_before = s1["total_iters"]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
            sim.step_async(1)
            ev[k][1].record(stream)
        try:
            ph = sim.timing()                    # synchronises: reads the in-graph phase events
            solve_ms.append(ph[2])
            phase_ms.append(ph)
        except Exception as e:                   # timing events unavailable: roofline left null
            timing_error = str(e)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist if world > 1 else None, dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    s2 = sim.stats()
    if s2["status"] != 0:
        raise RuntimeError(f"step failed: {s2}")
    iters = (s2["total_iters"] - it_before) / args.steps

    # force error at the stated tolerance: GPU forces vs the oracle's exact
    # discrete solution on the GPU's final positions (rank 0, not timed)
    ferr = None
    if rank == 0:
        import oracle as O
        x = sim.get(M.MAZE_POS)
        F = sim.get(M.MAZE_FORCE)
        p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order)
        phi_ex, _ = O.exact_potential(x, types, p)
        Q = np.where(types == 0, 1.0, -1.0)
        if w.n_ions <= 5000:
            idx = np.arange(w.n_ions)
            Fo = O.gather_forces(x, Q, phi_ex, w.L, w.N, w.order) + O.tf_forces(x, types, w.L, tf, w.rc)[0]
        else:   # large boxes: 64 sampled ions, brute-force pairs for those only
            idx = np.random.default_rng(5).choice(w.n_ions, 64, replace=False)
            Fo = (O.gather_forces(x[idx], Q[idx], phi_ex, w.L, w.N, w.order)
                  + O.tf_forces_on(idx, x, types, w.L, tf, w.rc))
        scale = np.sqrt((np.linalg.norm(F, axis=1) ** 2).mean())
        nrm = np.linalg.norm(Fo, axis=1)
        ferr = float((np.linalg.norm(F[idx] - Fo, axis=1) / np.maximum(nrm, scale)).max())

    # end to end through the C ABI with host buffers: per step upload the ion
    # state from pinned host memory, run the step, read back positions + stats
    e2e = None
    if not args.no_e2e:
        io = sim.exchange_buffers()   # pinned host positions and velocities
        n_e2e = min(args.steps, 100)
        sim.set_timing(False)    # a user's step: no phase events in the graph
        for _ in range(5):       # untimed warm-up (the GPU idled during the force check)
            sim.exchange(io)
        if world > 1:
            dist.barrier()
        e2e_s = 0.0
        for _ in range(n_e2e):
            # L2 flushed before each exchange, outside its timing (as for the
            # device-timed steps)
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # maze_step_io: upload, one step, positions, velocities and the
            # record back, one synchronisation
            sim.exchange(io)
            e2e_s += time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dist if world > 1 else None, dev)
        e2e = {"value": weak_scaling_value(world, n_e2e, e2e_s), "unit": "steps/s",
               "h2d_bytes_per_step": 2 * 24 * w.n_ions,
               "d2h_bytes_per_step": 2 * 24 * w.n_ions + 104}

    if rank == 0:
        ng = w.N ** 3
        bytes_launch = solve_bytes_per_launch(w.N, iters, args.solver, precision=args.precision)
        mean_solve_s = statistics.mean(solve_ms) / 1e3 if solve_ms else float("nan")
        achieved = bytes_launch / mean_solve_s / 1e9
        peak, peak_kind = peaks()
        cpu = None if args.no_cpu else run_cpu_baseline(w, args.solver)
        if args.precision == "mixed" and w.N <= 64:
            kps = KERNELS_PER_STEP_SPLIT if has_cells(w) else KERNELS_PER_STEP_FUSED
        else:
            kps = KERNELS_PER_STEP_CELLS if has_cells(w) else KERNELS_PER_STEP_NOCELLS
        line = {
            "metric": METRIC, "value": weak_scaling_value(world, args.steps, total_s), "unit": "steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f32x2",
            "data": "synthetic", "config": config_dict(w, args),
            "p50_us": 1e3 * float(np.percentile(step_ms, 50)), "p99_us": 1e3 * float(np.percentile(step_ms, 99)),
            "iters_per_step": iters, "force_error": ferr,
            "phase_us": dict(zip(["move_spread", "cells", "solve", "forces"],
                                 [round(1e3 * float(v), 2) for v in np.mean(phase_ms, axis=0)])) if phase_ms else None,
            "solve_gbs": achieved, "solve_us": 1e6 * mean_solve_s,
            "roofline": {"kernel": solve_kernel_name(args, w), "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": measured_traffic(args.workload, solve_kernel_name(args, w), args.precision,
                                                     args.solver),
                         "algorithmic_bytes_per_launch": bytes_launch},
            "cpu_baseline": cpu, "e2e": e2e, "timing_error": timing_error,
            "gpu_launches": kps * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Batched replicas and serving

BATCH_BOXES = 128


def oracle_box_step_seconds(w, steps=2):
    """Seconds per MD step of the FP64 oracle on one box (after step 0)."""
    import oracle as O
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order, solver="mg")
    st = O.init(pos, vel, types, p, tf)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = O.step(st, p, tf)
    return (time.perf_counter() - t0) / steps


def mix_rate(ws, per_size_seconds):
    """Box-steps/s of advancing the boxes ``ws`` one after another, given the
    seconds per step of one box of each size."""
    t = sum(per_size_seconds[w.n_ions] for w in ws) / len(ws)
    return 1.0 / t


def batch_cpu_baseline(ws, steps=2):
    sizes = sorted({w.n_ions for w in ws})
    t0 = time.perf_counter()
    per = {n: oracle_box_step_seconds(next(w for w in ws if w.n_ions == n), steps) for n in sizes}
    dt = time.perf_counter() - t0
    return {"value": mix_rate(ws, per), "unit": "box-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} MD steps of one box of each size {sizes} (after its step 0), numpy FP64, one "
                      f"thread ({dt:.1f} s), weighted by the size mix of the {len(ws)} boxes"}


def batch_config(ws, extra=None):
    from collections import Counter
    c = Counter(w.n_ions for w in ws)
    d = {"workload": f"{len(ws)} molten-NaCl replica boxes, ion counts drawn uniformly from "
                     f"{sorted(c)} (grids 16^3-48^3, ~1 A spacing), 1200 K, dt=1 fs, tol=1e-10, P=4, "
                     f"r_cut=min(L/2, 9 A), seeds 3001-{3000 + len(ws)}",
         "boxes": len(ws), "mix": {str(k): v for k, v in sorted(c.items())},
         "ions_total": sum(w.n_ions for w in ws), "grid_points_total": sum(w.N ** 3 for w in ws),
         "solver": "mg", "precision": "mixed"}
    if extra:
        d.update(extra)
    return d


def bench_batch(args):
    import torch
    from paper_2505_20418_gb300 import maze as M
    torch.cuda.set_device(0)
    M.load()
    ws = synth.batch_workloads(args.boxes)
    tf = synth.tosi_fumi_nacl()
    stream = torch.cuda.Stream()
    states = [synth.make_state(w) for w in ws]
    need = sum(M.MazeBatch.box_bytes(*st, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order)
               for w, st in zip(ws, states))
    b = M.MazeBatch(need + (64 << 20), len(ws), cluster_ctas=args.cluster_ctas, stream=stream.cuda_stream)
    ids = [b.add(*st, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order) for w, st in zip(ws, states)]
    if args.cluster_ctas == 0:
        cta, tune_ms = b.tune(3)
    else:
        cta, tune_ms = args.cluster_ctas, None
    b.step(args.warmup)
    it0 = sum(b.stats(i)["total_iters"] for i in ids)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    big = need > (160 << 20)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            if not big:
                flush.zero_()
            ev[k][0].record(stream)
            b.step_async(1)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_s = sum(step_ms) / 1e3
    st = b.step_status(0)
    stats = [b.stats(i) for i in ids]
    if any(s["status"] != 0 for s in stats) or st != 0:
        raise RuntimeError("a box failed during the timed steps")
    iters = (sum(s["total_iters"] for s in stats) - it0) / (args.steps * len(ids))
    # force error of one box of each size against the oracle's exact
    # discrete solution on the GPU's current positions (not timed)
    import oracle as O
    ferr = 0.0
    for n in sorted({w.n_ions for w in ws}):
        j = next(k for k, w in enumerate(ws) if w.n_ions == n)
        w = ws[j]
        x = b.get(ids[j], M.MAZE_POS)
        F = b.get(ids[j], M.MAZE_FORCE)
        types = states[j][2]
        p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order)
        phi_ex, _ = O.exact_potential(x, types, p)
        Q = np.where(types == 0, 1.0, -1.0)
        Fo = O.gather_forces(x, Q, phi_ex, w.L, w.N, w.order) + O.tf_forces(x, types, w.L, tf, w.rc)[0]
        scale = np.sqrt((np.linalg.norm(F, axis=1) ** 2).mean())
        ferr = max(ferr, float((np.linalg.norm(F - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), scale)).max()))
    # the same boxes advanced one after another by single-box contexts:
    # the plain FP64 path and the single-box mixed path (per size class)
    single = {}
    for prec in ("fp64", "mixed"):
        per = {}
        for n in sorted({w.n_ions for w in ws}):
            j = next(k for k, w in enumerate(ws) if w.n_ions == n)
            w = ws[j]
            sim = M.MazeSim(*states[j], w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order,
                            solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED if prec == "mixed" else M.MAZE_FP64,
                            stream=stream.cuda_stream)
            sim.step(3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                sim.step_async(20)
                e1.record(stream)
            torch.cuda.synchronize()
            per[n] = e0.elapsed_time(e1) / 1e3 / 20
            sim.close()
        single[prec] = mix_rate(ws, per)
    # end to end through the C ABI with host buffers: per step every box's
    # positions and velocities go up from pinned host memory, the step runs,
    # positions, velocities and statistics come back
    e2e = None
    if not args.no_e2e:
        host = [(torch.from_numpy(b.get(i, M.MAZE_POS)).pin_memory(), torch.from_numpy(b.get(i, M.MAZE_VEL)).pin_memory())
                for i in ids]
        n_e2e = 5
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            for i, (hp, hv) in zip(ids, host):
                b.set(i, M.MAZE_POS, hp.numpy())
                b.set(i, M.MAZE_VEL, hv.numpy())
            b.step(1)
            for i, (hp, hv) in zip(ids, host):
                hp.numpy()[:] = b.get(i, M.MAZE_POS)
                hv.numpy()[:] = b.get(i, M.MAZE_VEL)
            b.all_stats()
        e2e_s = time.perf_counter() - t0
        nion = sum(w.n_ions for w in ws)
        e2e = {"value": len(ids) * n_e2e / e2e_s, "unit": "box-steps/s", "h2d_bytes_per_step": 2 * 24 * nion,
               "d2h_bytes_per_step": 2 * 24 * nion + 104 * len(ids)}
    bytes_launch = sum(solve_bytes_per_launch(w.N, iters, "mg", precision="mixed") + 200 * w.n_ions for w in ws)
    mean_s = total_s / args.steps
    achieved = bytes_launch / mean_s / 1e9
    peak, peak_kind = peaks()
    cpu = None if args.no_cpu else batch_cpu_baseline(ws)
    b.close()
    line = {
        "metric": METRIC, "value": len(ids) * args.steps / total_s, "unit": "box-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f32x2", "data": "synthetic",
        "config": batch_config(ws, {"cluster_ctas": cta, "tune_ms_per_step": tune_ms,
                                    "l2": "working set larger than L2, not flushed" if big else
                                    "flushed between timed steps (256 MiB write outside the step events)"}),
        "batch_steps_per_s": args.steps / total_s,
        "ion_steps_per_s": sum(w.n_ions for w in ws) * args.steps / total_s,
        "p50_us": 1e3 * float(np.percentile(step_ms, 50)), "p99_us": 1e3 * float(np.percentile(step_ms, 99)),
        "iters_per_step": iters, "force_error": ferr,
        "single_box_paths": {"fp64_box_steps_per_s": single["fp64"], "mixed_box_steps_per_s": single["mixed"],
                             "how": "one box of each size timed alone (20 steps, CUDA events), weighted by the mix"},
        "roofline": {"kernel": "k_batch_step", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": bytes_launch},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def bench_batch_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    ws = synth.batch_workloads(args.boxes)
    cpu = batch_cpu_baseline(ws, steps=max(1, min(args.steps, 2)))
    v = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "box-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(ws) / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": batch_config(ws), "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "box-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVE_RATE = 200.0


def bench_serve(args):
    import torch
    from paper_2505_20418_gb300 import maze as M
    from paper_2505_20418_gb300 import serve
    torch.cuda.set_device(0)
    M.load()
    reqs = serve.poisson_requests(args.requests, SERVE_RATE)
    stream = torch.cuda.Stream()
    srv = serve.Server(16 << 30, 512, stream=stream.cuda_stream, chunk=4)
    # warm-up: a few short requests through the same server (module load, graph)
    srv.run(serve.poisson_requests(4, 1000.0, seed=4999, sizes=(216, 1000), steps=(args.warmup, args.warmup)),
            realtime=False)
    clocks = ClockSampler(0)
    clocks.start()
    out = srv.run(reqs, realtime=True, max_wall=300.0)
    clk = clocks.stop()
    info = srv.batch.info()
    srv.close()
    line = {
        "metric": METRIC, "value": out["steps_per_s"], "unit": "box-steps/s", "n_gpus": 1,
        "steps": out["box_steps"], "warmup": args.warmup, "ms_per_step": out["p50_step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f32x2",
        "data": "synthetic",
        "config": {"workload": f"serving loop: {args.requests} requests, Poisson arrivals at {SERVE_RATE:g}/s, "
                               "boxes of 64-13824 ions (grids 16^3-64^3), 50-2000 steps each, mixed precision, "
                               "admission by device memory (16 GiB arena, 512 slots), continuous batching",
                   "requests": args.requests, "rate_per_s": SERVE_RATE, "cluster_ctas": info["cluster_ctas"]},
        "p50_step_ms": out["p50_step_ms"], "p99_step_ms": out["p99_step_ms"], "served": out["served"],
        "wall_s": out["wall_s"], "ion_steps_per_s": out["ion_steps"] / out["wall_s"],
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": out["steps_per_s"], "unit": "box-steps/s",
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "the serving loop itself is end to end: host state in, final state out per request"},
        "gpu_launches": out["launches"], "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def bench_serve_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    print(json.dumps({"impl": "reference", "unavailable": "the oracle has no serving loop; see --workload batch128 "
                      "--impl reference for the oracle's per-box rate"}), flush=True)


def bench_study(args):
    """Iteration counts of Sec. III.A on synthetic molten NaCl: V-cycles per
    step to tol = 1e-7 for the MaZe solve and the direct multigrid solves
    with static and time-propagated starts (Fig. tol_vs_v_cycles), on the
    1000-ion box, and the solid-vs-molten comparison of Table
    convergence_solid_molten on a 512-ion box (300 K with 0.05 A lattice
    noise vs 2800 K), mixed precision, averaged over steps 50-150."""
    import torch
    from paper_2505_20418_gb300 import maze as M
    torch.cuda.set_device(0)
    M.load()
    tf = synth.tosi_fumi_nacl()
    schemes = {"maze": M.MAZE_SCHEME_MAZE, "mg-timeprop": M.MAZE_SCHEME_MG_TIMEPROP,
               "mg-static": M.MAZE_SCHEME_MG_STATIC}

    def vcycles(w, scheme, skip=50, count=100):
        pos, vel, types = synth.make_state(w)
        sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=1e-7, order=w.order,
                        solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, scheme=schemes[scheme])
        sim.step(skip)
        a = sim.stats()["total_iters"]
        sim.step(count)
        v = (sim.stats()["total_iters"] - a) / count
        sim.close()
        return v

    molten = synth.workload("nacl1000")
    e3 = {k: vcycles(molten, k) for k in schemes}
    solid = synth.replica(512, 6001, T=300.0, sigma=0.05)
    hot = synth.replica(512, 6001, T=2800.0)
    e5 = {}
    for k in schemes:
        s_, m_ = vcycles(solid, k), vcycles(hot, k)
        e5[k] = {"solid_300K": s_, "molten_2800K": m_, "slowdown": m_ / s_ if s_ > 0 else None}
    line = {"metric": "V-cycles per MD step to tol 1e-7 (Sec. III.A)", "value": e3["maze"], "unit": "V-cycles/step",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "f32+f32x2",
            "config": {"workload": "iteration study: molten NaCl 1000 ions / 32^3 (1200 K start), and 512 ions / "
                                   "24^3 solid (300 K, 0.05 A noise) vs hot (2800 K); steps 50-150, mixed precision"},
            "convergence_by_scheme_1000_ions": e3,
            "ratio_vs_maze": {k: e3[k] / e3["maze"] for k in e3},
            "solid_vs_molten_512_ions": e5,
            "paper_for_context": {"h_A": 0.172, "maze": 4, "mg-timeprop": "about 8", "mg-static": "about 28",
                                  "solid_vs_molten": {"maze": "2 -> 5", "mg-timeprop": "3 -> 11", "mg-static": "7 -> 22"}}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
