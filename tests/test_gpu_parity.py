"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Force metric (per ion alpha): |F_gpu - F_ref| / max(|F_ref|, rms_beta |F_ref|);
the bar is 1e-10 in FP64 mode with both sides solving the constraint to
tol = 1e-13 (the tolerance sets how close two correct solutions are: their
potentials differ by up to (4pi/h) |M^+| tol).
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-13
FORCE_BAR = 1e-10


def force_err(F, Fref):
    nrm = np.linalg.norm(Fref, axis=1)
    rms = np.sqrt((nrm ** 2).mean())
    return float((np.linalg.norm(F - Fref, axis=1) / np.maximum(nrm, rms)).max())


def case(name):
    """(pos, vel, types, L, N, rc, P) for the parity boxes."""
    if name == "nacl64":
        w = synth.workload("nacl64")
        pos, vel, types = synth.make_state(w)
        return pos, vel, types, w.L, w.N, w.rc, 4
    if name == "nacl64_P2":
        w = synth.workload("nacl64")
        pos, vel, types = synth.make_state(w)
        return pos, vel, types, w.L, w.N, w.rc, 2
    if name == "nacl1000":
        w = synth.workload("nacl1000")
        pos, vel, types = synth.make_state(w)
        return pos, vel, types, w.L, w.N, w.rc, 4
    if name == "nacl216_N24":      # non-power-of-two grid, all-pairs (2 cells per edge)
        w = synth.Workload("n216", 6, 18.9, 24, seed=31)
        pos, vel, types = synth.make_state(w)
        return pos, vel, types, w.L, w.N, w.rc, 4
    if name == "nacl1728_N40":     # 4 cells per edge, N = 40
        w = synth.Workload("n1728", 12, 37.8, 40, seed=32)
        pos, vel, types = synth.make_state(w)
        return pos, vel, types, w.L, w.N, w.rc, 4
    if name == "tiny8_N14":        # an edge of 2 (mod 4): the one-point-per-thread sweeps, coarsest 7^3
        pos, types = synth.random_neutral(8, 8.0, 5, min_dist=2.3)
        vel = synth.maxwell(types, 1200.0, np.random.default_rng(5))
        return pos, vel, types, 8.0, 14, 4.0, 4
    if name == "tiny8_N8":         # minimum grid, 8 ions
        pos, types = synth.random_neutral(8, 8.0, 5, min_dist=2.3)
        vel = synth.maxwell(types, 1200.0, np.random.default_rng(5))
        return pos, vel, types, 8.0, 8, 4.0, 4
    raise KeyError(name)


SOLVERS = {"cg": M.MAZE_SOLVER_CG, "mg": M.MAZE_SOLVER_MG}


def make(name, tol=TOL, solver="cg", **kw):
    pos, vel, types, L, N, rc, P = case(name)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=tol, order=P, solver=SOLVERS[solver], **kw)
    p = O.Params(L=L, N=N, dt=1.0, tol=tol, rc=rc, P=P, solver=solver)
    return sim, p, tf, (pos, vel, types)


CASES = ["nacl64", "nacl64_P2", "nacl1000", "nacl216_N24", "nacl1728_N40", "tiny8_N8", "tiny8_N14"]


@pytest.mark.parametrize("name", CASES)
def test_spread_parity(name):
    sim, p, tf, (pos, vel, types) = make(name)
    rng = np.random.default_rng(1)
    newpos = rng.uniform(0, p.L, size=pos.shape)
    newpos[0] = [0.0, p.L - 1e-12, 0.5 * p.h]        # seam and node edge cases
    sim.set(M.MAZE_POS, newpos)
    sim.spread()
    q = sim.get(M.MAZE_CHARGE)
    Q = np.where(types == 0, 1.0, -1.0)
    qo = O.spread(O.wrap(newpos, p.L), Q, p.L, p.N, p.P)
    assert np.abs(q - qo).max() < 1e-13
    assert abs(q.sum()) < 1e-12
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
@pytest.mark.parametrize("name", CASES)
def test_step0_parity(name, solver):
    sim, p, tf, (pos, vel, types) = make(name, solver=solver)
    st = O.init(pos, vel, types, p, tf)
    F = sim.get(M.MAZE_FORCE)
    assert force_err(F, st.F) < FORCE_BAR
    assert force_err(sim.get(M.MAZE_FORCE_EL), st.F_el) < FORCE_BAR
    phi = sim.get(M.MAZE_PHI)
    assert abs(phi.mean()) < 1e-12
    assert np.abs(phi - st.phi).max() < 1e-9 * max(1.0, np.abs(st.phi).max())
    assert np.array_equal(phi, sim.get(M.MAZE_PHI_PREV))
    s = sim.stats()
    assert s["status"] == 0 and s["step"] == 0 and s["resid"] < TOL
    assert abs(s["v_tf"] - st.V_tf) < 1e-10 * max(1.0, abs(st.V_tf))
    assert abs(s["v_disc"] - st.V_disc) < 1e-9 * max(1.0, abs(st.V_disc))
    assert abs(s["ke"] - O.kinetic(st, p)) < 1e-12 * O.kinetic(st, p)
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
@pytest.mark.parametrize("name", ["nacl64", "nacl64_P2", "nacl1000", "nacl1728_N40", "nacl216_N24"])
def test_one_step_parity(name, solver):
    sim, p, tf, (pos, vel, types) = make(name, solver=solver)
    st = O.step(O.init(pos, vel, types, p, tf), p, tf)
    sim.step(1)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < FORCE_BAR
    d = sim.get(M.MAZE_POS) - st.pos
    d -= p.L * np.round(d / p.L)
    assert np.abs(d).max() < 1e-13 * p.L
    assert np.abs(sim.get(M.MAZE_VEL) - st.vel).max() < 1e-12 * np.abs(st.vel).max()
    s = sim.stats()
    assert s["step"] == 1 and s["status"] == 0 and s["resid"] < TOL
    assert abs(s["v_work"] - st.V_work) < 1e-9 * max(1.0, abs(st.V_work))
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_solve_and_gather_from_oracle_state(solver):
    """maze_spread / maze_solve / maze_gather on an oracle mid-trajectory state."""
    sim, p, tf, (pos, vel, types) = make("nacl1000", solver=solver)
    st = O.init(pos, vel, types, p, tf)
    for _ in range(3):
        st = O.step(st, p, tf)
    nxt = O.step(st, p, tf)
    sim.set(M.MAZE_POS, nxt.pos)
    sim.set(M.MAZE_PHI, st.phi)
    sim.set(M.MAZE_PHI_PREV, st.phi_prev)
    sim.set(M.MAZE_Y, st.y)
    sim.spread()
    it, res = sim.solve()
    assert res < TOL
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(nxt.pos, Q, p.L, p.N, p.P)
    _, sp = O.sigma_p(st.phi, st.phi_prev, q, p.h)
    assert np.abs(sim.get(M.MAZE_SIGMA) - sp).max() < 1e-13 * max(1.0, np.abs(sp).max())
    assert abs(it - nxt.iters) <= max(1 if solver == "mg" else 3, 0.1 * nxt.iters)
    phi = sim.get(M.MAZE_PHI)
    assert np.abs(phi - nxt.phi).max() < 1e-9
    assert np.array_equal(sim.get(M.MAZE_PHI_PREV), st.phi)
    sim.gather()
    assert force_err(sim.get(M.MAZE_FORCE), nxt.F) < FORCE_BAR
    assert force_err(sim.get(M.MAZE_FORCE_EL), nxt.F_el) < FORCE_BAR
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_trajectory_nacl64_100_steps(solver):
    sim, p, tf, (pos, vel, types) = make("nacl64", solver=solver)
    st = O.init(pos, vel, types, p, tf)
    for k in range(4):
        for _ in range(25):
            st = O.step(st, p, tf)
        sim.step(25)
        assert force_err(sim.get(M.MAZE_FORCE), st.F) < 1e-9, k
    s = sim.stats()
    assert s["step"] == 100
    assert abs(s["e_tot"] - O.energies(st, p)["e_tot"]) < 1e-9 * abs(O.energies(st, p)["e_tot"])
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_energy_and_momentum_conservation_nacl1000(solver):
    """NVE with V_work (Eq. E_nostra): total energy fluctuates far less than
    V_work; total momentum stays at the solver-tolerance level."""
    sim, p, tf, _ = make("nacl1000", tol=1e-10, solver=solver)
    E, Vw = [], []
    for _ in range(100):
        sim.step(2)
        s = sim.stats()
        E.append(s["e_tot"])
        Vw.append(s["v_work"])
        assert s["status"] == 0
    E, Vw = np.array(E), np.array(Vw)
    assert E.std() / Vw.std() < 2e-4
    assert np.abs(s["momentum"]).max() < 1e-6
    sim.close()


@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_deterministic_and_checkpoint_resume_bitwise(solver):
    a, p, tf, _ = make("nacl1000", tol=1e-10, solver=solver)
    b, _, _, _ = make("nacl1000", tol=1e-10, solver=solver)
    a.step(10)
    blob = a.get_state()
    a.step(10)
    b.step(20)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI):
        assert np.array_equal(a.get(what), b.get(what))
    c, _, _, _ = make("nacl1000", tol=1e-10, solver=solver)
    c.set_state(blob)
    c.step(10)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI, M.MAZE_PHI_PREV, M.MAZE_Y):
        assert np.array_equal(a.get(what), c.get(what))
    sa, sc = a.stats(), c.stats()
    assert sa["step"] == sc["step"] == 20 and sa["v_work"] == sc["v_work"]
    for s in (a, b, c):
        s.close()


def test_not_converged_is_reported_and_stops():
    # step 0 has its own iteration cap, so a tiny max_iter only hits the steps
    sim, p, tf, _ = make("nacl1000", tol=1e-10, max_iter=2)
    with pytest.raises(M.MazeError) as e:
        sim.step(3)
    assert e.value.status == M.MAZE_ERR_NOT_CONVERGED
    s = sim.stats()
    assert s["step"] == 1 and s["iters"] == 2 and s["status"] == M.MAZE_ERR_NOT_CONVERGED
    # the failed step completed consistently (forces of its last iterate)
    assert np.isfinite(sim.get(M.MAZE_FORCE)).all()
    sim.close()


@pytest.mark.parametrize("solver,precision", [("cg", M.MAZE_FP64), ("mg", M.MAZE_FP64), ("mg", M.MAZE_MIXED)])
def test_nonfinite_warm_start_is_reported(solver, precision):
    """A NaN in the warm start y makes the residual non-finite: the solve must
    report MAZE_ERR_NONFINITE, not a converged result (an fmax-based norm
    would drop the NaN and report a small residual)."""
    sim, p, tf, _ = make("nacl1000", tol=1e-10, solver=solver, precision=precision)
    y = sim.get(M.MAZE_Y)
    y.ravel()[12345] = np.nan
    sim.set(M.MAZE_Y, y)
    sim.spread()
    st, it, res = M.maze_solve(sim.h)
    assert st == M.MAZE_ERR_NONFINITE, (st, it, res)
    assert not np.isfinite(res)
    sim.close()


def test_zero_steps_is_noop():
    sim, p, tf, _ = make("nacl64")
    x = sim.get(M.MAZE_POS)
    sim.step(0)
    assert np.array_equal(x, sim.get(M.MAZE_POS)) and sim.stats()["step"] == 0
    sim.close()


@pytest.mark.slow
@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_large_box_sampled_parity(solver):
    """512000 ions, 256^3 grid, one step at tol 1e-10: the constraint holds on
    the whole grid and sampled forces match the oracle evaluated on the GPU's
    own positions and potential."""
    w = synth.workload("nacl512000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, solver=SOLVERS[solver])
    sim.step(1)
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < w.tol
    x = sim.get(M.MAZE_POS)
    phi = sim.get(M.MAZE_PHI)
    F = sim.get(M.MAZE_FORCE)
    h = w.L / w.N
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(x, Q, w.L, w.N, 4)
    sig = (h / (4 * np.pi)) * O.apply_M(phi) + q
    assert O.inf_norm(sig) < 2 * w.tol
    idx = np.random.default_rng(9).choice(len(x), 48, replace=False)
    Fo = O.gather_forces(x[idx], Q[idx], phi, w.L, w.N, 4) + O.tf_forces_on(idx, x, types, w.L, tf, w.rc)
    scale = np.sqrt((F ** 2).sum(1).mean())
    err = np.linalg.norm(F[idx] - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), scale)
    assert err.max() < FORCE_BAR
    sim.close()


def test_mg_iterations_match_the_oracle_on_a_trajectory():
    """Same hierarchy, smoother and transfer operators as the oracle: the
    V-cycle counts per step agree (within one) over 20 steps at tol 1e-10."""
    sim, p, tf, (pos, vel, types) = make("nacl1000", tol=1e-10, solver="mg")
    st = O.init(pos, vel, types, p, tf)
    for _ in range(20):
        st = O.step(st, p, tf)
        sim.step(1)
        assert abs(sim.stats()["iters"] - st.iters) <= 1


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_gives_up_with_timeout(which):
    """Failure detection without a GPU fault: a grid barrier or grid reduction
    waiting for a round no block completes gives up after its poll limit
    (about a second), records MAZE_ERR_TIMEOUT and returns; the GPU stays
    usable (a context built and stepped afterwards converges)."""
    import time
    t0 = time.perf_counter()
    st, rec = M.maze_wait_probe(which)
    dt = time.perf_counter() - t0
    assert st == M.MAZE_OK, M.maze_last_error()
    assert rec == M.MAZE_ERR_TIMEOUT
    assert dt < 30.0
    sim, p, tf, _ = make("nacl64", tol=1e-10)
    sim.step(2)
    assert sim.stats()["status"] == M.MAZE_OK
    sim.close()


def test_once_per_pair_forces_parity_and_determinism():
    """FP64 boxes with at least 2 cells per SM evaluate each Tosi-Fumi pair
    once (Newton's third law) with fixed-point per-ion sums; the 8000-ion /
    64^3 box (7^3 cells) takes that path: step 0 and one step against the
    oracle at the FP64 bar, and two runs bit for bit equal."""
    w = synth.workload("nacl8000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sims = [M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=TOL, solver=M.MAZE_SOLVER_MG)
            for _ in range(2)]
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=TOL, rc=w.rc, P=4, solver="mg")
    st = O.init(pos, vel, types, p, tf)
    assert force_err(sims[0].get(M.MAZE_FORCE), st.F) < FORCE_BAR
    st = O.step(st, p, tf)
    for s in sims:
        s.step(1)
    assert force_err(sims[0].get(M.MAZE_FORCE), st.F) < FORCE_BAR
    assert abs(sims[0].stats()["v_tf"] - st.V_tf) < 1e-9 * abs(st.V_tf)
    for s in sims:
        s.step(3)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE):
        assert np.array_equal(sims[0].get(what), sims[1].get(what))
    for s in sims:
        s.close()


def test_double_float_pairs_match_the_fp64_pairs(monkeypatch):
    """The once-per-pair kernel of FP64 boxes runs its pair arithmetic in
    double-float on the FP32 pipe; MAZE_PAIRS_FP64=1 selects the same kernel
    with FP64 arithmetic. On the 8000-ion / 64^3 box (7^3 cells) the two
    agree within the FP64 force bar, at step 0 and after a step, in the
    forces and the Tosi-Fumi energy. Both forms round every pair's share to
    2^-40 eV/A (the FP64 form within half a unit, the double-float form
    within one), so an ion's ~100 shares differ by about 1e-11 eV/A in
    total: ~3e-11 of the rms force, which the pair arithmetic itself
    (~1e-13 relative) stays far below."""
    w = synth.workload("nacl8000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sims = []
    for fp64 in (False, True):
        if fp64:
            monkeypatch.setenv("MAZE_PAIRS_FP64", "1")
        else:
            monkeypatch.delenv("MAZE_PAIRS_FP64", raising=False)
        sims.append(M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=TOL, solver=M.MAZE_SOLVER_MG))
    for k in range(2):
        if k:
            for s in sims:
                s.step(1)
        Fd, Ff = sims[0].get(M.MAZE_FORCE), sims[1].get(M.MAZE_FORCE)
        assert force_err(Fd, Ff) < FORCE_BAR
        vd, vf = sims[0].stats()["v_tf"], sims[1].stats()["v_tf"]
        assert abs(vd - vf) < 1e-10 * abs(vf)
    for s in sims:
        s.close()
