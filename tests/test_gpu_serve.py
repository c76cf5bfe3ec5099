"""Serving loop on the GPU: requests of different box sizes join and leave a
running batch (continuous batching); each request's final state equals, bit
for bit, the same simulation run alone for the same number of steps."""
import numpy as np
import pytest

from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import serve, synth

pytestmark = pytest.mark.gpu


def test_each_request_alone_equals_in_the_mix():
    reqs = serve.poisson_requests(10, rate=2000.0, sizes=(64, 216, 512, 1000), steps=(5, 30), seed=91)
    srv = serve.Server(1 << 30, 4, chunk=4)     # 4 slots: later requests wait for earlier ones
    out = srv.run(reqs, realtime=False)
    srv.close()
    assert out["served"] == len(reqs)
    assert out["box_steps"] == sum(q.steps for q in reqs)
    tf = synth.tosi_fumi_nacl()
    for q in reqs:
        assert q.status == 0
        w = q.work
        pos, vel, types = synth.make_state(w)
        sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order,
                        solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED)
        sim.step(q.steps)
        assert np.array_equal(sim.get(M.MAZE_POS), q.final_pos), q.rid
        assert np.array_equal(sim.get(M.MAZE_VEL), q.final_vel), q.rid
        sim.close()


def test_realtime_arrivals_report_latency():
    reqs = serve.poisson_requests(6, rate=200.0, sizes=(64, 216), steps=(10, 20), seed=92)
    srv = serve.Server(1 << 30, 8, chunk=2)
    out = srv.run(reqs, realtime=True, max_wall=60.0)
    srv.close()
    assert out["served"] == 6
    assert 0 < out["p50_step_ms"] <= out["p99_step_ms"]
    assert out["steps_per_s"] > 0
