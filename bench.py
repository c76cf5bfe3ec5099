"""Benchmark of the GB300 Poisson MaZe step (one JSON line on rank 0).

A step is one full MaZe MD step (S1-S9) of one synthetic molten-NaCl box.
Default workload: 512000 ions (256000 Na+, 256000 Cl-), L = 252 Angstrom,
256^3 grid, 1200 K, dt = 1 fs, constraint tolerance 1e-10, cubic B-spline
assignment, warm-started multigrid constraint solve with FP64 state whose
V-cycle corrections are exact 64-bit integers (--precision fp64fix). The same
box with the all-FP64 V-cycle is timed after it and reported under "fp64",
and in mixed precision (FP32 V-cycle, double-float outer iteration, exact
integer reductions) under "mixed". Inputs are resident in HBM when the timed
region starts; L2 is flushed (256 MiB write) between timed steps, outside the
per-step CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload nacl64|nacl1000|nacl8000|nacl64000|nacl512000|batch128|serve|study]
                  [--solver cg|mg] [--precision fp64fix|fp64|mixed]

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
KERNELS_PER_STEP_HALF = 8     # one force block per cell: ... solve, pairs once each + gather, finish
KERNELS_PER_STEP_OVERLAP = 9  # the same with the pairs beside the solve: move, 3 cell-list kernels, pairs, spread,
#                               solve, gather, finish
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
    """Grid sizes of the multigrid hierarchy as the kernels build it: halve
    while the edge is even and above 8 (an 8^3 grid once), so the coarsest
    level has at most 8^3 points."""
    sizes = [N]
    while sizes[-1] % 2 == 0 and (sizes[-1] > 8 or (sizes[-1] == 8 and len(sizes) == 1)):
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

    FP64 state with the integer V-cycle (fp64fix; every level but the
    coarsest stored split by colour, so a half-sweep reads one colour): S4
    64 B/pt (read phi^k, phi^{k-1}, q, y; write phi_p, sigma_p, r_0, q
    cleared), r_0 to fixed point 16 B/pt, S6 48 B/pt (read y, E, phi_p;
    write y, phi); per V-cycle and level 24 B/pt per sweep, residual 16 B/pt,
    full weighting 5.5 B/pt, prolongation 9 B/pt; the stopping test 12 B/pt
    of the finest level; coarsest 16 B/pt.

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
    if precision == "fp64fix":
        per_v = sum(n ** 3 * ((nu[0] + nu[1]) * 24 + 16 + 5.5 + 9) for n in lv[:-1]) + lv[-1] ** 3 * 16 + ng * 12
        return ng * (64 + 16 + 48) + per_v * iters
    base = ng * (56 + 32)
    if solver == "cg":
        return base + ng * (64 * iters + 24)
    per_v = sum(n ** 3 * ((nu[0] + nu[1]) * 32 + 24 + 9 + 9) for n in lv[:-1]) + lv[-1] ** 3 * 16 + ng * 16
    return base + per_v * iters


def survey_bytes_per_launch(N, iters, solver="mg", precision="fp64"):
    """The same launch on the coarser per-point unit of the hot-path scope
    table: 167 B/pt per FP64 V-cycle over all levels, 64 B/pt per FP64 CG
    iteration, 72 B/pt of S4/S6/charge clearing per solve; mixed precision
    halves every figure."""
    ng = N ** 3
    per = 167.0 if solver == "mg" else 64.0
    b = ng * (72.0 + per * iters)
    return b / 2 if precision == "mixed" else b


def fp64_mg_ops_per_launch(N, iters, nu=(2, 2)):
    """Algorithmic FP64 operations of one FP64 multigrid solve launch, one per
    add, multiply or fused multiply-add (the FP64 pipe issues each of them at
    the same rate), for the operations the method states and nothing else:

      S4, per point: phi_p = 2 phi^k - phi^{k-1} (1), the two six-neighbour
        sums of phi^k and phi^{k-1} (10), M phi_p = 2 s_k - s_{k-1} - 6 phi_p
        (2), sigma_p = (h/4pi) M phi_p + q (1): 14;
      first residual of the warm start, every point: six-neighbour sum (5),
        -6 y (1), subtraction (1): 7;
      per V-cycle, each level of n_l points above the coarsest: a red-black
        Gauss-Seidel update (six-neighbour sum, then (s - b)/6 as one FMA on
        a pre-scaled b: 6) per point and sweep, less 5 of the 6 at the red
        half of the first sweep from a zero guess on coarse levels; the
        residual at red points (7 per red point; black residuals are zero
        after the black half-sweep); full weighting from the 13 red points
        of the 27 (13 per coarse point); trilinear prolongation to black
        points (2 for the 3/4 of them with one odd coordinate, 8 for the
        rest; the red ones are overwritten by the next half-sweep); the
        coarsest level: a dense product with the pseudo-inverse (n_c^2);
      per V-cycle, the convergence test: residual at red points (7 each);
      the mean of y (1 per point) and S6 phi = phi_p - (4pi/h)(y - mean) (2).
    """
    ng = N ** 3
    lv = mg_levels(N)
    sweeps = nu[0] + nu[1]
    per_v = 0.0
    for l, n in enumerate(lv[:-1]):
        p = n ** 3
        sm = sweeps * 6.0 - (2.5 if l > 0 else 0.0)
        per_v += p * (sm + 3.5 + 1.75) + (p / 8.0) * 13.0
    per_v += float(lv[-1] ** 3) ** 2 + ng * 3.5
    return ng * (14.0 + 7.0 + 1.0 + 2.0) + iters * per_v


def fp64_peak_tops(sms):
    """FP64 pipe peak of a GB300: 2 FP64 operations per clock per SM (the
    rate ncu lists for the FP64 pipe: 64 lanes of 1/32 rate per SM) times
    the SMs times the maximum SM clock, in 10^12 operations per second."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return 2.0 * sms * mhz * 1e6 / 1e12


def oracle_sample(w):
    """The bounded sample the oracle is timed on: the box itself when one of
    its steps takes a few seconds; for the 256^3 and 128^3 boxes, the
    8000-ion 64^3 box of the same molten NaCl (same density, grid spacing,
    temperature, tolerance and seed recipe), whose per-step work (ions, grid
    points, pairs) is 1/64 (1/8) of theirs. Returns (workload, work ratio)."""
    if w.n_ions > 8000:
        s = synth.workload("nacl8000")
        return s, float(w.n_ions) / s.n_ions
    return w, 1.0


def _oracle_steps(name_or_w, solver, budget_s, max_steps, warmup=0):
    """Oracle MD steps of one box for up to ``budget_s`` seconds (at least
    one): (steps, seconds, per-step seconds)."""
    import oracle as O
    w = synth.workload(name_or_w) if isinstance(name_or_w, str) else name_or_w
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order, solver=solver)
    st = O.init(pos, vel, types, p, tf)
    for _ in range(warmup):
        st = O.step(st, p, tf)
    times = []
    t0 = time.perf_counter()
    while not times or (time.perf_counter() - t0 < budget_s and len(times) < max_steps):
        t1 = time.perf_counter()
        st = O.step(st, p, tf)
        times.append(time.perf_counter() - t1)
    return len(times), sum(times), times


def _oracle_worker(args):
    name, solver, budget_s = args
    n, dt, _ = _oracle_steps(name, solver, budget_s, 10 ** 6)
    return n, dt


def run_cpu_baseline(w, solver="mg", budget_s=15.0):
    """The FP64 oracle as it stands, on a bounded sample of the same workload,
    on one host thread."""
    ws, ratio = oracle_sample(w)
    n, dt, _ = _oracle_steps(ws, solver, budget_s, 10 ** 6)
    what = (f"{n} MD steps of the same {w.n_ions}-ion {w.N}^3 box from its initial state" if ratio == 1.0 else
            f"{n} MD steps of the {ws.n_ions}-ion {ws.N}^3 box of the same molten NaCl (1/{ratio:g} of the "
            f"{w.n_ions}-ion {w.N}^3 box's ions and grid points), value scaled by 1/{ratio:g}")
    return {"value": n / dt / ratio, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}; numpy FP64, single thread ({dt:.1f} s)"}


def run_cpu_all_cores(w, solver="mg", budget_s=10.0):
    """The same oracle sample on every host core at once: one independent
    single-thread oracle process per core, each advancing its own copy of the
    sample box (spawned processes, so the parent's CUDA context is not
    inherited). Aggregate throughput, scaled like the single-thread figure,
    and the seconds per grid point per V-cycle of one oracle V-cycle."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle as O
    ws, ratio = oracle_sample(w)
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, [(_sample_name(ws), solver, budget_s)] * cores))
    rate = sum(n / dt for n, dt in res)
    # one V-cycle of the oracle on the sample grid (context for the paper's
    # CPU seconds per grid point per V-cycle)
    rng = np.random.default_rng(7)
    b = rng.normal(size=(ws.N,) * 3)
    b -= b.mean()
    x = np.zeros_like(b)
    t0 = time.perf_counter()
    nv = 3
    for _ in range(nv):
        x = O.vcycle(x, b, 1e-10)
    tv = (time.perf_counter() - t0) / nv
    return {"value": rate / ratio, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent single-thread oracle processes, each advancing its own "
                      f"{ws.n_ions}-ion {ws.N}^3 box for {budget_s:g} s; aggregate steps/s scaled by 1/{ratio:g}",
            "s_per_point_per_vcycle": tv / ws.N ** 3}


def _sample_name(ws):
    for name in ("nacl64", "nacl1000", "nacl8000", "nacl64000", "nacl512000"):
        if synth.workload(name).name == ws.name:
            return name
    raise KeyError(ws.name)


def bench_reference(args, w):
    """--impl reference: the oracle on the host cores. Each timed step is one
    oracle MD step of the bounded sample box (oracle_sample); the value is
    scaled by the work ratio to steps/s of the named workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ws, ratio = oracle_sample(w)
    n, tot, times = _oracle_steps(ws, args.solver, float("inf"), args.steps, warmup=args.warmup)
    val = args.steps / tot / ratio
    what = (f"{args.steps} timed MD steps after {args.warmup} warm-up steps of the {w.n_ions}-ion {w.N}^3 box"
            if ratio == 1.0 else
            f"{args.steps} timed MD steps after {args.warmup} warm-up steps of the {ws.n_ions}-ion {ws.N}^3 box "
            f"of the same molten NaCl (1/{ratio:g} of the {w.n_ions}-ion {w.N}^3 box's ions and grid points), "
            f"steps/s scaled by 1/{ratio:g}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps * ratio,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, args, reference=True),
            "p50_us": 1e6 * ratio * float(np.percentile(times, 50)),
            "p99_us": 1e6 * ratio * float(np.percentile(times, 99)),
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{what}; numpy FP64, one host thread"},
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


def config_dict(w, args, reference=False):
    """The workload of the line. The CUDA arm's headline precision is the
    one --precision names; the reference arm is always the FP64 oracle."""
    prec = "fp64" if reference else args.precision
    return {"workload": f"molten NaCl {w.n_ions} ions, L={w.L} A, {w.N}^3 grid, {w.T:.0f} K, dt={w.dt} fs, "
                        f"tol={w.tol:g}, P={w.order}, r_cut={w.rc} A",
            "n_ions": w.n_ions, "grid": w.N, "solver": args.solver, "precision": prec,
            "l2": "flushed between timed steps and before each timed e2e exchange (256 MiB write outside "
                  "the timing)"}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# roofline kernel, from one ncu capture of the kernels as they stand; the
# command and the other counters are in the named summary under profiles/.
# A kernel changed after its capture must drop its entry (traffic null).
MEASURED_TRAFFIC = {
    ("nacl512000", "k_mgfix_solve", "fp64fix", "mg"): (10833341000, "profiles/k_mgfix_solve_nacl512000.md"),
    ("nacl512000", "k_mg_solve", "fp64", "mg"): (19889471000, "profiles/k_mg_solve_nacl512000_fp64.md"),
    ("nacl512000", "k_mixed_grid", "mixed", "mg"): (6902114000, "profiles/k_mixed_grid_nacl512000.md"),
}


def measured_traffic(workload, kernel, precision, solver):
    hit = MEASURED_TRAFFIC.get((workload, kernel, precision, solver))
    return None if hit is None else hit[0]


# The arithmetic each --precision computes in: FP64; FP64 state with the
# multigrid corrections in exact 64-bit integers; FP32 grid arithmetic with
# double-float (FP32 pair) outer vectors. FP64 boxes with at least two cells
# per SM evaluate the Tosi-Fumi pairs in double-float on the FP32 pipe (~1e-13
# relative): "+f32x2" (dtype()).
DTYPES = {"fp64": "f64", "fp64fix": "f64+i64", "mixed": "f32+f32x2"}


def dtype(precision, w, sms=152):
    """DTYPES, with the double-float pair arithmetic of large FP64 boxes."""
    if precision != "mixed" and has_cells(w) and int(np.floor(w.L / w.rc)) ** 3 >= 2 * sms:
        return DTYPES[precision] + "+f32x2"
    return DTYPES[precision]


def precision_code(M, precision):
    """The C ABI's precision constant for a --precision name."""
    return {"fp64": M.MAZE_FP64, "mixed": M.MAZE_MIXED, "fp64fix": M.MAZE_FP64_FIXMG}[precision]


def has_cells(w):
    """True when the box takes the cell list (at least 3 cells of r_cut a side)."""
    return int(np.floor(w.L / w.rc)) >= 3


def solve_kernel_name(precision, solver, w):
    """The solve kernel a step launches for this precision, solver and grid."""
    if precision == "mixed":
        if w.N > 64:
            return "k_mixed_grid"
        return "k_mixed_cluster" if has_cells(w) else "k_cluster_step"
    if precision == "fp64fix":
        return "k_mgfix_solve"
    return "k_mg_solve" if solver == "mg" else "k_cg_solve"


def overlapped(precision, w, sms=152):
    """True when the step runs the pairs beside the solve (the integer
    V-cycle on grids of 128^3 and more with at least 2 cells per SM, unless
    MAZE_OVERLAP=0)."""
    return (precision == "fp64fix" and w.N >= 128 and has_cells(w) and int(np.floor(w.L / w.rc)) ** 3 >= 2 * sms
            and os.environ.get("MAZE_OVERLAP") != "0")


def kernels_per_step(precision, w, sms=152):
    if precision == "mixed" and w.N <= 64:
        return KERNELS_PER_STEP_SPLIT if has_cells(w) else KERNELS_PER_STEP_FUSED
    if overlapped(precision, w, sms):
        return KERNELS_PER_STEP_OVERLAP
    if has_cells(w) and int(np.floor(w.L / w.rc)) ** 3 >= 2 * sms:   # FP64, or mixed above 64^3
        return KERNELS_PER_STEP_HALF
    return KERNELS_PER_STEP_CELLS if has_cells(w) else KERNELS_PER_STEP_NOCELLS


def force_error_vs_oracle(M, sim, w, types, tf):
    """Per-ion force error of the GPU's current forces against the oracle's
    exact discrete solution on the GPU's current positions (all ions up to
    5000, else 64 sampled ions with brute-force pairs for those)."""
    import oracle as O
    x = sim.get(M.MAZE_POS)
    F = sim.get(M.MAZE_FORCE)
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order)
    phi_ex, _ = O.exact_potential(x, types, p)
    Q = np.where(types == 0, 1.0, -1.0)
    if w.n_ions <= 5000:
        idx = np.arange(w.n_ions)
        Fo = O.gather_forces(x, Q, phi_ex, w.L, w.N, w.order) + O.tf_forces(x, types, w.L, tf, w.rc)[0]
    else:
        idx = np.random.default_rng(5).choice(w.n_ions, 64, replace=False)
        Fo = (O.gather_forces(x[idx], Q[idx], phi_ex, w.L, w.N, w.order)
              + O.tf_forces_on(idx, x, types, w.L, tf, w.rc))
    scale = np.sqrt((np.linalg.norm(F, axis=1) ** 2).mean())
    nrm = np.linalg.norm(Fo, axis=1)
    return float((np.linalg.norm(F[idx] - Fo, axis=1) / np.maximum(nrm, scale)).max())


def time_box(args, M, w, precision, solver, stream, flush, dist=None, dev="cpu", world=1, rank=0, e2e=True):
    """Time ``args.steps`` steps of one box (after ``args.warmup`` untimed
    ones): per-step CUDA events on the context stream with an L2 flush
    between steps outside the events, the solve kernel's time from events
    inside the step graph; then the force error against the oracle (rank 0)
    and, when asked, the end-to-end exchange through the C ABI."""
    import torch
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order,
                    solver=M.MAZE_SOLVER_MG if solver == "mg" else M.MAZE_SOLVER_CG,
                    precision=precision_code(M, precision), stream=stream.cuda_stream)
    sim.set_timing(True)
    for _ in range(args.warmup):
        sim.step_async(1)
    torch.cuda.synchronize()
    s1 = sim.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    solve_ms, phase_ms, timing_error = [], [], None
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else
                          int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
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
    out = {"steps_per_s": weak_scaling_value(world, args.steps, total_s), "total_s": total_s,
           "ms_per_step": 1e3 * total_s / args.steps, "step_ms": step_ms,
           "iters_per_step": (s2["total_iters"] - s1["total_iters"]) / args.steps,
           "solve_s": statistics.mean(solve_ms) / 1e3 if solve_ms else float("nan"),
           "phase_us": dict(zip(["move_spread", "cells", "solve", "forces"],
                                [round(1e3 * float(v), 2) for v in np.mean(phase_ms, axis=0)])) if phase_ms else None,
           "timing_error": timing_error, "clocks": clk, "force_error": None, "e2e": None}
    if rank == 0:
        out["force_error"] = force_error_vs_oracle(M, sim, w, types, tf)
    if e2e:
        # end to end through the C ABI with host buffers: per step upload the
        # ion state from pinned host memory, run the step, read back
        # positions, velocities and the record (maze_step_io, one sync)
        io = sim.exchange_buffers()
        n_e2e = min(args.steps, 100)
        sim.set_timing(False)    # a user's step: no phase events in the graph
        for _ in range(5):       # untimed warm-up (the GPU idled during the force check)
            sim.exchange(io)
        if world > 1:
            dist.barrier()
        e2e_s = 0.0
        for _ in range(n_e2e):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.exchange(io)
            e2e_s += time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dist if world > 1 else None, dev)
        out["e2e"] = {"value": weak_scaling_value(world, n_e2e, e2e_s), "unit": "steps/s",
                      "h2d_bytes_per_step": 2 * 24 * w.n_ions, "d2h_bytes_per_step": 2 * 24 * w.n_ions + 104}
    sim.close()
    return out


def full_run(M, w, precision, solver, stream, flush):
    """The configuration's whole run: a fresh box advanced its w.steps steps
    from its initial state, every step timed with CUDA events (L2 flushed
    between steps, outside the events), as a user runs it (no phase events in
    the graphs). The V-cycle count per step grows as the lattice start melts
    (steps 3 to ~35 need 4 at 512000 ions, later ones 5), so the K timed steps
    after W warm-up steps of the line are an early window of this run; this
    key gives the whole run beside them."""
    import torch
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order,
                    solver=M.MAZE_SOLVER_MG if solver == "mg" else M.MAZE_SOLVER_CG,
                    precision=precision_code(M, precision), stream=stream.cuda_stream)
    sim.set_timing(False)
    ms, its = [], []
    prev = sim.stats()["total_iters"]
    for _ in range(w.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            sim.step_async(1)
            e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        t = sim.stats()["total_iters"]
        its.append(t - prev)
        prev = t
    st = sim.stats()
    sim.close()
    if st["status"] != 0:
        raise RuntimeError(f"full run failed: {st}")
    q = max(1, len(ms) // 4)
    return {"what": f"the configuration's {w.steps} steps from its initial state on a fresh box, each timed "
                    "(untimed graphs, L2 flushed between steps)",
            "steps": w.steps, "steps_per_s": 1e3 * len(ms) / sum(ms), "ms_per_step": sum(ms) / len(ms),
            "iters_per_step": sum(its) / len(its),
            "last_quarter": {"ms_per_step": sum(ms[-q:]) / q, "iters_per_step": sum(its[-q:]) / q}}


def rooflines(w, precision, solver, iters, solve_s, workload, sms):
    """The solve kernel against its roofs: HBM (measured copy peak) always;
    for FP64 multigrid also the FP64 pipe. ``roofline`` is the binding one
    (the roof whose time for the algorithmic work is longer). Algorithmic
    bytes are the hot-path scope table's per-point unit (survey_bytes_per_launch);
    the finer one-pass-per-vector-touch model (solve_bytes_per_launch) is
    reported beside it."""
    kernel = solve_kernel_name(precision, solver, w)
    peak, peak_kind = peaks()
    b = survey_bytes_per_launch(w.N, iters, solver, precision)
    bm = solve_bytes_per_launch(w.N, iters, solver, precision=precision)
    hbm = {"kernel": kernel, "bound": "hbm", "achieved": b / solve_s / 1e9, "peak": peak,
           "peak_kind": peak_kind, "unit": "GB/s", "frac": b / solve_s / 1e9 / peak,
           "traffic": measured_traffic(workload, kernel, precision, solver), "algorithmic_bytes_per_launch": b,
           "model_bytes_per_launch": bm, "model_frac": bm / solve_s / 1e9 / peak}
    if precision != "fp64" or solver != "mg":
        return hbm, None
    ops = fp64_mg_ops_per_launch(w.N, iters)
    pk = fp64_peak_tops(sms)
    alu = {"kernel": kernel, "bound": "alu", "achieved": ops / solve_s / 1e12, "peak": pk,
           "peak_kind": "derived: 2 FP64 operations per clock per SM x SMs x maximum SM clock",
           "unit": "TOP/s (FP64 add, multiply or FMA = 1 operation)", "frac": ops / solve_s / 1e12 / pk,
           "traffic": hbm["traffic"], "algorithmic_ops_per_launch": ops, "algorithmic_bytes_per_launch": b}
    if ops / (pk * 1e12) >= b / (peak * 1e9):
        return alu, hbm
    return hbm, alu


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nacl512000",
                    choices=["nacl64", "nacl1000", "nacl8000", "nacl64000", "nacl512000", "batch128", "serve",
                             "study"])
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--boxes", type=int, default=128, help="batch128: number of replica boxes")
    ap.add_argument("--cluster-ctas", type=int, default=0, help="batch128: CTAs per box (0: autotune)")
    ap.add_argument("--solver", default="mg", choices=["cg", "mg"])
    ap.add_argument("--precision", default="fp64fix", choices=["fp64fix", "fp64", "mixed"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-full", action="store_true", help="skip the configuration's whole run beside the line")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the runs beside an FP64 line (the other FP64 form and mixed precision)")
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
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # every rank advances its own replica (independent seed)
    w = replica_workload(args.workload, rank)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    head = time_box(args, M, w, args.precision, args.solver, stream, flush, dist, dev, world, rank,
                    e2e=not args.no_e2e)
    # the same box beside an FP64 multigrid headline (extra keys): the other
    # FP64 form of the solve, and mixed precision
    mixed = other64 = serial = None
    if args.precision in ("fp64", "fp64fix") and args.solver == "mg" and not args.no_mixed:
        alt = "fp64" if args.precision == "fp64fix" else "fp64fix"
        other64 = (alt, time_box(args, M, w, alt, "mg", stream, flush, dist, dev, world, rank, e2e=False))
        if args.precision == "fp64fix" and os.environ.get("MAZE_OVERLAP") != "0":
            # the headline runs the pairs beside the solve: the solve kernel
            # alone, from the same box with the overlap off
            os.environ["MAZE_OVERLAP"] = "0"
            try:
                serial = time_box(args, M, w, "fp64fix", "mg", stream, flush, dist, dev, world, rank, e2e=False)
            finally:
                del os.environ["MAZE_OVERLAP"]
        mixed = time_box(args, M, w, "mixed", "mg", stream, flush, dist, dev, world, rank, e2e=False)

    whole = None
    if rank == 0 and not args.no_full:
        whole = full_run(M, w, args.precision, args.solver, stream, flush)

    if rank == 0:
        roof, other = rooflines(w, args.precision, args.solver, head["iters_per_step"], head["solve_s"],
                                args.workload, sms)
        cpu = None if args.no_cpu else run_cpu_baseline(w, args.solver)
        cpu_all = None
        if not args.no_cpu:
            try:
                cpu_all = run_cpu_all_cores(w, args.solver)
            except Exception as e:          # a worker that could not start: reported, not fatal
                cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
        line = {
            "metric": METRIC, "value": head["steps_per_s"], "unit": "steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype(args.precision, w, sms),
            "data": "synthetic", "config": config_dict(w, args),
            "p50_us": 1e3 * float(np.percentile(head["step_ms"], 50)),
            "p99_us": 1e3 * float(np.percentile(head["step_ms"], 99)),
            "iters_per_step": head["iters_per_step"], "force_error": head["force_error"],
            "phase_us": head["phase_us"], "solve_us": 1e6 * head["solve_s"],
            "roofline": roof, "roofline_other": other,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": head["e2e"],
            "timing_error": head["timing_error"],
            "gpu_launches": kernels_per_step(args.precision, w, sms) * args.steps, "clocks": head["clocks"],
            "full_run": whole,
        }
        if other64 is not None:
            alt, o = other64
            oroof, oother = rooflines(w, alt, "mg", o["iters_per_step"], o["solve_s"], args.workload, sms)
            line[alt] = {
                "what": ("the same box and steps with the FP64 V-cycle (every multigrid operation in FP64 "
                         "arithmetic)" if alt == "fp64" else
                         "the same box and steps with the integer V-cycle (FP64 state, corrections in exact "
                         "64-bit integers)") + ", timed the same way after the headline run",
                "dtype": dtype(alt, w, sms), "steps_per_s": o["steps_per_s"], "ms_per_step": o["ms_per_step"],
                "iters_per_step": o["iters_per_step"], "force_error": o["force_error"],
                "phase_us": o["phase_us"], "solve_us": 1e6 * o["solve_s"], "roofline": oroof,
                "roofline_other": oother, "gpu_launches": kernels_per_step(alt, w, sms) * args.steps,
                "clocks": o["clocks"]}
        if serial is not None:
            sroof, _ = rooflines(w, "fp64fix", "mg", serial["iters_per_step"], serial["solve_s"], args.workload, sms)
            line["serial"] = {
                "what": "the same box with the pairs after the solve on one stream (MAZE_OVERLAP=0): the solve "
                        "kernel alone on the GPU; in the headline it shares every SM with the pair kernel",
                "steps_per_s": serial["steps_per_s"], "ms_per_step": serial["ms_per_step"],
                "iters_per_step": serial["iters_per_step"], "force_error": serial["force_error"],
                "phase_us": serial["phase_us"], "solve_us": 1e6 * serial["solve_s"], "roofline": sroof,
                "gpu_launches": KERNELS_PER_STEP_HALF * args.steps, "clocks": serial["clocks"]}
        if mixed is not None:
            mroof, _ = rooflines(w, "mixed", "mg", mixed["iters_per_step"], mixed["solve_s"], args.workload, sms)
            line["mixed"] = {
                "what": "the same box and steps in mixed precision (FP32 V-cycle, double-float outer SHAKE "
                        "iteration, FP64 reductions), timed the same way after the headline run",
                "steps_per_s": mixed["steps_per_s"], "ms_per_step": mixed["ms_per_step"],
                "speedup_vs_headline": mixed["steps_per_s"] / head["steps_per_s"],
                "iters_per_step": mixed["iters_per_step"], "force_error": mixed["force_error"],
                "phase_us": mixed["phase_us"], "solve_us": 1e6 * mixed["solve_s"], "roofline": mroof,
                "gpu_launches": kernels_per_step("mixed", w, sms) * args.steps, "clocks": mixed["clocks"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Batched replicas and serving

BATCH_BOXES = 128
# FP64 tolerance at which the FP64 path's per-ion force error (~1e-6 on the
# 1000- and 4096-ion boxes) is still at or below the mixed path's (~4e-6 at
# any tolerance: its floor is FP32 spreading, gather and pairs); at 3e-7 it
# is already ~1.5e-5. Equal accuracy for the FP64-vs-mixed comparison.
FP64_EQUAL_ACCURACY_TOL = 1e-7


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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    big = need > (160 << 20)

    def timed_steps(n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        torch.cuda.synchronize()
        for k in range(n):
            with torch.cuda.stream(stream):
                if not big:
                    flush.zero_()
                ev[k][0].record(stream)
                b.step_async(1)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in ev]

    # one cluster size for every box (the one-size tuner), then the
    # per-size-class autotuner; the line's value is the autotuned batch
    if args.cluster_ctas == 0:
        cta, tune_ms = b.tune(3)
    else:
        cta, tune_ms = args.cluster_ctas, None
    b.step(args.warmup)
    one_ms = timed_steps(args.steps)
    table = b.autotune(3)
    b.step(args.warmup)
    it0 = sum(b.stats(i)["total_iters"] for i in ids)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    step_ms = timed_steps(args.steps)
    clk = clocks.stop()
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
    # the same boxes advanced one after another by single-box contexts: the
    # plain FP64 path at the batch's tolerance, the FP64 path at the loosest
    # tolerance whose force error stays at or below the mixed path's (equal
    # accuracy), and the single-box mixed path (one box per size class)
    single, single_err = {}, {}
    for name, prec, tol in (("fp64", "fp64", None), ("fp64_equal_accuracy", "fp64", FP64_EQUAL_ACCURACY_TOL),
                            ("mixed", "mixed", None)):
        per, err = {}, 0.0
        for n in sorted({w.n_ions for w in ws}):
            j = next(k for k, w in enumerate(ws) if w.n_ions == n)
            w = ws[j]
            sim = M.MazeSim(*states[j], w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=tol or w.tol, order=w.order,
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
            err = max(err, force_error_vs_oracle(M, sim, w, states[j][2], tf))
            sim.close()
        single[name] = mix_rate(ws, per)
        single_err[name] = err
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
    bytes_launch = sum(survey_bytes_per_launch(w.N, iters, "mg", "mixed") + 200 * w.n_ions for w in ws)
    mean_s = total_s / args.steps
    achieved = bytes_launch / mean_s / 1e9
    peak, peak_kind = peaks()
    cpu = None if args.no_cpu else batch_cpu_baseline(ws)
    b.close()
    line = {
        "metric": METRIC, "value": len(ids) * args.steps / total_s, "unit": "box-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f32x2", "data": "synthetic",
        "config": batch_config(ws, {"cluster_ctas": "per size class (autotuned)", "tune_ms_per_step": tune_ms,
                                    "l2": "working set larger than L2, not flushed" if big else
                                    "flushed between timed steps (256 MiB write outside the step events)"}),
        "batch_steps_per_s": args.steps / total_s,
        "autotune_table": table,
        "one_size_fits_all": {"cluster_ctas": cta, "box_steps_per_s": len(ids) * len(one_ms) / (sum(one_ms) / 1e3),
                              "ms_per_step": sum(one_ms) / len(one_ms),
                              "how": "maze_batch_tune: one cluster size for every box, the configured V-cycle"},
        "ion_steps_per_s": sum(w.n_ions for w in ws) * args.steps / total_s,
        "p50_us": 1e3 * float(np.percentile(step_ms, 50)), "p99_us": 1e3 * float(np.percentile(step_ms, 99)),
        "iters_per_step": iters, "force_error": ferr,
        "single_box_paths": {"fp64_box_steps_per_s": single["fp64"], "fp64_force_error": single_err["fp64"],
                             "fp64_equal_accuracy_box_steps_per_s": single["fp64_equal_accuracy"],
                             "fp64_equal_accuracy_tol": FP64_EQUAL_ACCURACY_TOL,
                             "fp64_equal_accuracy_force_error": single_err["fp64_equal_accuracy"],
                             "mixed_box_steps_per_s": single["mixed"], "mixed_force_error": single_err["mixed"],
                             "batched_mixed_vs_fp64_equal_accuracy": len(ids) * args.steps / total_s
                             / single["fp64_equal_accuracy"],
                             "how": "one box of each size timed alone (20 steps, CUDA events), weighted by the mix; "
                                    "force errors: the largest over one box of each size against the oracle's "
                                    "exact discrete solution after the 23 steps"},
        "roofline": {"kernel": "k_batch_step", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": bytes_launch},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * (1 + len({t["cluster_ctas"] for t in table})), "clocks": clk,
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
        "p50_step_ms": out["p50_step_ms"], "p99_step_ms": out["p99_step_ms"],
        "with_arrivals": out["with_arrivals"], "without_arrivals": out["without_arrivals"],
        "served": out["served"],
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
