"""The allocation-free solve entry point against the context-based solve.

maze_solve_shake_noalloc serves callers that cannot call cudaMalloc (a
framework that owns all device memory through its own pool, a loop that must
not take cudaMalloc's implicit synchronisation, a fixed memory budget): the
caller owns sigma_p and y, and the solver's work vectors live in a fixed
file-scope device array. Here it must reproduce maze_solve's y on the same
sigma_p and warm start, on two calls in a row (the second call must not see
leftovers of the first), and reject grids above its fixed limit.
"""
import numpy as np
import pytest

from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _context():
    w = synth.workload("nacl1000")
    pos, vel, types = synth.make_state(w)
    return M.MazeSim(pos, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc, dt=w.dt, tol=TOL), w


def _reference_solve(sim):
    """One context-based solve on the current positions: (sigma_p, y0, y)."""
    y0 = sim.get(M.MAZE_Y)
    sim.spread()
    it, res = sim.solve()
    return sim.get(M.MAZE_SIGMA), y0, sim.get(M.MAZE_Y), it


def test_noalloc_solve_matches_maze_solve_twice():
    import torch
    sim, w = _context()
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(2 + call)
        sigma, y0, y_ref, it_ref = _reference_solve(sim)
        d_sigma = torch.from_numpy(sigma.ravel().copy()).cuda()
        d_y = torch.from_numpy(y0.ravel().copy()).cuda()
        torch.cuda.synchronize()
        st, it, res = M.maze_solve_shake_noalloc(w.N, d_sigma.data_ptr(), d_y.data_ptr(), TOL, 10000,
                                                 stream.cuda_stream)
        assert st == M.MAZE_OK, M.maze_last_error()
        assert res < TOL
        y = d_y.cpu().numpy().reshape(y_ref.shape)
        assert abs(it - it_ref) <= 2
        assert np.abs(y - y_ref).max() < 1e-9 * max(1.0, np.abs(y_ref).max())
        assert abs(y.mean()) < 1e-12
    sim.close()


def test_noalloc_rejects_grids_above_its_limit():
    import torch
    d = torch.zeros(80 ** 3, dtype=torch.float64, device="cuda")
    e = torch.zeros(80 ** 3, dtype=torch.float64, device="cuda")
    st, _, _ = M.maze_solve_shake_noalloc(80, d.data_ptr(), e.data_ptr(), 1e-10, 10)
    assert st == M.MAZE_ERR_INVALID
    assert "grid_N <= 64" in M.maze_last_error()


def test_noalloc_at_its_size_limit_matches_maze_solve():
    """grid_N = 64 fills the fixed scratch exactly (the 13824-ion box)."""
    import torch
    w = synth.replica(13824, 5001)
    pos, vel, types = synth.make_state(w)
    sim = M.MazeSim(pos, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc, dt=w.dt, tol=TOL)
    sim.step(1)
    sigma, y0, y_ref, it_ref = _reference_solve(sim)
    d_sigma = torch.from_numpy(sigma.ravel().copy()).cuda()
    d_y = torch.from_numpy(y0.ravel().copy()).cuda()
    torch.cuda.synchronize()
    st, it, res = M.maze_solve_shake_noalloc(64, d_sigma.data_ptr(), d_y.data_ptr(), TOL, 10000,
                                             torch.cuda.current_stream().cuda_stream)
    assert st == M.MAZE_OK, M.maze_last_error()
    assert res < TOL and abs(it - it_ref) <= 2
    y = d_y.cpu().numpy().reshape(y_ref.shape)
    assert np.abs(y - y_ref).max() < 1e-9 * max(1.0, np.abs(y_ref).max())
    sim.close()


def test_noalloc_reports_not_converged_and_nonfinite():
    import torch
    sim, w = _context()
    sim.step(2)
    sigma, y0, _, _ = _reference_solve(sim)
    sim.close()
    stream = torch.cuda.current_stream().cuda_stream
    d_sigma = torch.from_numpy(sigma.ravel().copy()).cuda()
    # one CG iteration cannot reach 1e-12 from the previous step's y
    d_y = torch.from_numpy(y0.ravel().copy()).cuda()
    st, it, res = M.maze_solve_shake_noalloc(w.N, d_sigma.data_ptr(), d_y.data_ptr(), TOL, 1, stream)
    assert st == M.MAZE_ERR_NOT_CONVERGED
    assert it == 1 and np.isfinite(res) and res >= TOL
    assert torch.isfinite(d_y).all()
    # a NaN in sigma_p, then an infinity in the warm start
    bad = sigma.ravel().copy()
    bad[777] = np.nan
    d_bad = torch.from_numpy(bad).cuda()
    d_y = torch.from_numpy(y0.ravel().copy()).cuda()
    st, _, res = M.maze_solve_shake_noalloc(w.N, d_bad.data_ptr(), d_y.data_ptr(), TOL, 100, stream)
    assert st == M.MAZE_ERR_NONFINITE and not np.isfinite(res)
    y_inf = y0.ravel().copy()
    y_inf[5] = np.inf
    d_y = torch.from_numpy(y_inf).cuda()
    st, _, _ = M.maze_solve_shake_noalloc(w.N, d_sigma.data_ptr(), d_y.data_ptr(), TOL, 100, stream)
    assert st == M.MAZE_ERR_NONFINITE
    # and a good call afterwards still converges (no state left behind)
    d_y = torch.from_numpy(y0.ravel().copy()).cuda()
    st, _, res = M.maze_solve_shake_noalloc(w.N, d_sigma.data_ptr(), d_y.data_ptr(), TOL, 10000, stream)
    assert st == M.MAZE_OK and res < TOL


def test_noalloc_rejects_aliased_buffers():
    import torch
    d = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    st, _, _ = M.maze_solve_shake_noalloc(32, d.data_ptr(), d.data_ptr(), 1e-10, 10)
    assert st == M.MAZE_ERR_INVALID
    assert "distinct" in M.maze_last_error()
