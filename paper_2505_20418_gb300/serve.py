"""Serving loop: continuous batching of independent MaZe simulations.

Requests (one seeded molten-NaCl box each, asking for a number of MaZe
steps) arrive over time. The loop admits a request as soon as the batch has a
free slot and arena room for its buffers (admission by device memory), keeps
every admitted simulation's positions, velocities and warm-start potential
resident on the GPU, and advances all admitted simulations together, one
persistent kernel launch per step (``maze_batch_*``). A request leaves when
its steps are done; its final state is read back then. Requests that arrive
while others are running join at the next step boundary, so their work shares
the same launches.

All arithmetic runs in libmaze's kernels; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import maze as M
from . import synth


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    work: synth.Workload
    steps: int
    # filled in by the server
    sid: int | None = None      # simulation id in the batch
    admitted: float | None = None
    finished: float | None = None
    done: int = 0
    status: int = 0
    final_pos: np.ndarray | None = None
    final_vel: np.ndarray | None = None


def poisson_requests(n: int, rate: float, seed: int = 5000, sizes=(64, 216, 512, 1000, 1728, 4096, 13824),
                     steps=(50, 2000)) -> list:
    """n requests with exponential inter-arrival times (mean 1/rate), box
    sizes drawn uniformly from ``sizes`` and step counts uniformly from the
    inclusive range ``steps``; request r's box is seeded seed + 1 + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    counts = rng.choice(np.asarray(sizes), size=n)
    nsteps = rng.integers(steps[0], steps[1] + 1, size=n)
    out = []
    for r in range(n):
        if int(counts[r]) == 64:
            w = synth.workload("nacl64")
            w.seed = seed + 1 + r
        else:
            w = synth.replica(int(counts[r]), seed + 1 + r)
        out.append(Request(r, float(t[r]), w, int(nsteps[r])))
    return out


class Server:
    """Continuous-batching MaZe server over one MazeBatch."""

    def __init__(self, arena_bytes: int, max_sims: int, cluster_ctas: int = 0, stream=None, chunk: int = 8,
                 batch=None):
        # ``batch``: an object with the MazeBatch methods used below (tests
        # pass a host-side stand-in to check the scheduling alone)
        self.batch = batch if batch is not None else M.MazeBatch(arena_bytes, max_sims, cluster_ctas=cluster_ctas,
                                                                 stream=stream)
        self.tf = synth.tosi_fumi_nacl()
        self.chunk = int(chunk)

    def close(self):
        self.batch.close()

    def _try_admit(self, q: Request) -> bool:
        w = q.work
        pos, vel, types = synth.make_state(w)
        sid = self.batch.try_add(pos, vel, types, w.L, w.N, self.tf, r_cut=w.rc, dt=w.dt, tol=w.tol,
                                 order=w.order)
        if sid is None:
            return False
        q.sid = sid
        return True

    def run(self, requests, realtime: bool = True, max_wall: float = 600.0) -> dict:
        """Serve ``requests`` (sorted by arrival). With ``realtime`` the loop
        admits a request only once the wall clock has passed its arrival time;
        otherwise arrivals are replayed as fast as the engine goes (every
        request is eligible at once).

        Each loop iteration lets the requests whose admission (step 0) has
        finished on the GPU join, queues the next k steps of every joined
        simulation, admits arrived requests while those steps run (a
        newcomer's set-up and step 0 go to the batch's admission stream and
        never hold up the running simulations), then waits for the steps and
        retires finished simulations. Returns per-step latencies (one sample
        per simulation per step: the loop iteration's time over its k steps),
        split into iterations that admitted a request and iterations that did
        not, and aggregate throughput."""
        pending = sorted(requests, key=lambda q: q.arrival)
        active: list[Request] = []
        waiting: dict[int, Request] = {}        # admitted, step 0 still running
        lat: list[float] = []
        lat_adm: list[float] = []
        lat_quiet: list[float] = []
        chunk_lat: list[float] = []
        box_steps = 0
        ion_steps = 0
        t0 = time.perf_counter()
        i = 0
        while (i < len(pending) or active or waiting) and time.perf_counter() - t0 < max_wall:
            t_iter = time.perf_counter()
            if waiting:
                for sid in self.batch.refresh():
                    active.append(waiting.pop(sid))
            # queue k steps of every joined simulation (no request overshoots)
            k = min(self.chunk, min(q.steps - q.done for q in active)) if active else 0
            if k:
                self.batch.step_ready_async(k)
            # admission while those steps run: arrived requests, in arrival
            # order, while there is room
            now = time.perf_counter() - t0
            joined = 0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                q = pending[i]
                if not self._try_admit(q):
                    break
                q.admitted = time.perf_counter() - t0
                waiting[q.sid] = q
                joined += 1
                i += 1
            if not k:
                if i < len(pending) and realtime and not waiting:
                    time.sleep(max(0.0, min(pending[i].arrival - now, 0.01)))
                elif waiting:
                    time.sleep(0.0002)
                continue
            # wait for the queued steps; statuses of everything stepped
            st = self.batch.sync_status()
            for q in active:
                q.done += k
            box_steps += k * len(active)
            ion_steps += k * sum(q.work.n_ions for q in active)
            # retire finished (or failed) simulations
            stats = self.batch.all_stats() if st != M.MAZE_OK else None
            keep = []
            for q in active:
                if stats is not None and stats[q.sid]["status"] != M.MAZE_OK:
                    q.status = stats[q.sid]["status"]
                if q.done >= q.steps or q.status != M.MAZE_OK:
                    q.final_pos = self.batch.get(q.sid, M.MAZE_POS)
                    q.final_vel = self.batch.get(q.sid, M.MAZE_VEL)
                    q.finished = time.perf_counter() - t0
                    self.batch.remove(q.sid)
                else:
                    keep.append(q)
            # latency of each step as its simulations saw it: the whole loop
            # iteration (the launches, admission, retirement) over its k steps
            per = (time.perf_counter() - t_iter) / k
            chunk_lat.append(per)
            samples = [per] * (k * len(active))
            lat.extend(samples)
            (lat_adm if joined else lat_quiet).extend(samples)
            active = keep
        wall = time.perf_counter() - t0

        def pct(v, p):
            return 1e3 * float(np.percentile(np.asarray(v), p)) if v else None

        return {
            "requests": len(requests), "served": sum(q.finished is not None for q in requests),
            "wall_s": wall, "box_steps": box_steps, "ion_steps": ion_steps,
            "steps_per_s": box_steps / wall if wall > 0 else 0.0,
            "p50_step_ms": pct(lat, 50) or 0.0, "p99_step_ms": pct(lat, 99) or 0.0,
            "with_arrivals": {"p50_step_ms": pct(lat_adm, 50), "p99_step_ms": pct(lat_adm, 99),
                              "steps": len(lat_adm)},
            "without_arrivals": {"p50_step_ms": pct(lat_quiet, 50), "p99_step_ms": pct(lat_quiet, 99),
                                 "steps": len(lat_quiet)},
            "launches": len(chunk_lat),
        }
