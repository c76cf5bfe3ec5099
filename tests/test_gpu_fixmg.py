"""GPU parity of precision MAZE_FP64_FIXMG (FP64 state, multigrid V-cycles as
FP64 defect correction with exact 64-bit integer corrections) against the
FP64 CPU oracle, at the FP64 bars of test_gpu_parity; and against the FP64
multigrid kernel, whose iterates it equals in exact arithmetic."""
import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth

from tests.test_gpu_parity import FORCE_BAR, TOL, case, force_err

pytestmark = pytest.mark.gpu


def make(name, tol=TOL, precision=M.MAZE_FP64_FIXMG, **kw):
    pos, vel, types, L, N, rc, P = case(name)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=tol, order=P, solver=M.MAZE_SOLVER_MG,
                    precision=precision, **kw)
    p = O.Params(L=L, N=N, dt=1.0, tol=tol, rc=rc, P=P, solver="mg")
    return sim, p, tf, (pos, vel, types)


@pytest.mark.parametrize("name", ["nacl64", "nacl64_P2", "nacl1000", "nacl216_N24", "nacl1728_N40", "tiny8_N8",
                                  "tiny8_N14"])
def test_step0_and_one_step_parity(name):
    sim, p, tf, (pos, vel, types) = make(name)
    st = O.init(pos, vel, types, p, tf)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < FORCE_BAR
    phi = sim.get(M.MAZE_PHI)
    assert abs(phi.mean()) < 1e-12
    assert np.abs(phi - st.phi).max() < 1e-9 * max(1.0, np.abs(st.phi).max())
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < TOL
    assert abs(s["v_disc"] - st.V_disc) < 1e-9 * max(1.0, abs(st.V_disc))
    st = O.step(st, p, tf)
    sim.step(1)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < FORCE_BAR
    d = sim.get(M.MAZE_POS) - st.pos
    d -= p.L * np.round(d / p.L)
    assert np.abs(d).max() < 1e-13 * p.L
    s = sim.stats()
    assert s["step"] == 1 and s["status"] == 0 and s["resid"] < TOL
    assert abs(s["v_work"] - st.V_work) < 1e-9 * max(1.0, abs(st.V_work))
    sim.close()


def test_solve_and_gather_from_oracle_state():
    sim, p, tf, (pos, vel, types) = make("nacl1000")
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
    # S4's Laplacian is summed exactly in integers: sigma_p at the oracle's precision
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(nxt.pos, Q, p.L, p.N, p.P)
    _, sp = O.sigma_p(st.phi, st.phi_prev, q, p.h)
    assert np.abs(sim.get(M.MAZE_SIGMA) - sp).max() < 1e-13 * max(1.0, np.abs(sp).max())
    assert abs(it - nxt.iters) <= 1
    assert np.abs(sim.get(M.MAZE_PHI) - nxt.phi).max() < 1e-9
    sim.gather()
    assert force_err(sim.get(M.MAZE_FORCE), nxt.F) < FORCE_BAR
    sim.close()


def test_iterations_match_the_oracle_and_the_fp64_kernel():
    """Over 20 steps at tol 1e-10 the V-cycle counts agree with the oracle's
    (within one) and the potential with the FP64 multigrid kernel's to far
    below the tolerance's reach."""
    sim, p, tf, (pos, vel, types) = make("nacl1000", tol=1e-10)
    ref, _, _, _ = make("nacl1000", tol=1e-10, precision=M.MAZE_FP64)
    st = O.init(pos, vel, types, p, tf)
    same = 0
    for _ in range(20):
        st = O.step(st, p, tf)
        sim.step(1)
        ref.step(1)
        a, b = sim.stats()["iters"], ref.stats()["iters"]
        assert abs(a - st.iters) <= 1
        same += a == b
    assert same >= 18
    phi, phr = sim.get(M.MAZE_PHI), ref.get(M.MAZE_PHI)
    assert np.abs(phi - phr).max() < 1e-8 * np.abs(phr).max()
    sim.close()
    ref.close()


def test_trajectory_nacl64_100_steps():
    sim, p, tf, (pos, vel, types) = make("nacl64")
    st = O.init(pos, vel, types, p, tf)
    for k in range(4):
        for _ in range(25):
            st = O.step(st, p, tf)
        sim.step(25)
        assert force_err(sim.get(M.MAZE_FORCE), st.F) < 1e-9, k
    s = sim.stats()
    assert abs(s["e_tot"] - O.energies(st, p)["e_tot"]) < 1e-9 * abs(O.energies(st, p)["e_tot"])
    sim.close()


def test_deterministic_and_checkpoint_resume_bitwise():
    a, p, tf, _ = make("nacl1000", tol=1e-10)
    b, _, _, _ = make("nacl1000", tol=1e-10)
    a.step(10)
    blob = a.get_state()
    a.step(10)
    b.step(20)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI, M.MAZE_Y):
        assert np.array_equal(a.get(what), b.get(what))
    c, _, _, _ = make("nacl1000", tol=1e-10)
    c.set_state(blob)
    c.step(10)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI, M.MAZE_PHI_PREV, M.MAZE_Y):
        assert np.array_equal(a.get(what), c.get(what))
    for s in (a, b, c):
        s.close()


def test_nonfinite_warm_start_is_reported():
    sim, p, tf, _ = make("nacl1000", tol=1e-10)
    y = sim.get(M.MAZE_Y)
    y.ravel()[12345] = np.nan
    sim.set(M.MAZE_Y, y)
    sim.spread()
    st, it, res = M.maze_solve(sim.h)
    assert st == M.MAZE_ERR_NONFINITE, (st, it, res)
    sim.close()


def test_not_converged_is_reported():
    sim, p, tf, _ = make("nacl1000", tol=1e-10, max_iter=1)
    with pytest.raises(M.MazeError) as e:
        sim.step(3)
    assert e.value.status == M.MAZE_ERR_NOT_CONVERGED
    assert sim.stats()["iters"] == 1
    sim.close()


def test_cg_solver_is_rejected():
    pos, vel, types, L, N, rc, P = case("nacl64")
    with pytest.raises(M.MazeError) as e:
        M.MazeSim(pos, vel, types, L, N, synth.tosi_fumi_nacl(), r_cut=rc, dt=1.0, tol=TOL,
                  solver=M.MAZE_SOLVER_CG, precision=M.MAZE_FP64_FIXMG)
    assert e.value.status == M.MAZE_ERR_INVALID


@pytest.mark.slow
def test_large_box_parity_and_agreement_with_fp64():
    """512000 ions, 256^3: the constraint holds on the whole grid, sampled
    forces match the oracle on the GPU's own positions and potential, and
    the potential equals the FP64 kernel's within the tolerance's reach."""
    w = synth.workload("nacl512000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sims = [M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, solver=M.MAZE_SOLVER_MG,
                      precision=pr) for pr in (M.MAZE_FP64_FIXMG, M.MAZE_FP64)]
    for s in sims:
        s.step(2)
    sim = sims[0]
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < w.tol
    assert abs(s["iters"] - sims[1].stats()["iters"]) <= 1
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
    phr = sims[1].get(M.MAZE_PHI)
    assert np.abs(phi - phr).max() < 1e-7 * np.abs(phr).max()
    for s in sims:
        s.close()


def test_overlapped_step_matches_the_serial_step(monkeypatch):
    """On large boxes the pairs run on a second stream beside a narrower
    solve (k_pairs_only), and S7 after it (k_gather_cells). The pair and
    V-cycle sums are exact integers; the FP64 mean of y is summed per thread,
    so the two launch forms agree to rounding (MAZE_OVERLAP=0 turns the
    overlap off), and each form is bitwise reproducible."""
    w = synth.workload("nacl64000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sims = []
    for ov in ("0", None, None):
        if ov is None:
            monkeypatch.delenv("MAZE_OVERLAP", raising=False)
        else:
            monkeypatch.setenv("MAZE_OVERLAP", ov)
        sims.append(M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol,
                              solver=M.MAZE_SOLVER_MG, precision=M.MAZE_FP64_FIXMG))
    for s in sims:
        s.step(1)
    F0, F1 = sims[0].get(M.MAZE_FORCE), sims[1].get(M.MAZE_FORCE)
    assert force_err(F1, F0) < 1e-12
    p0, p1 = sims[0].get(M.MAZE_PHI), sims[1].get(M.MAZE_PHI)
    assert np.abs(p1 - p0).max() < 1e-12 * np.abs(p0).max()
    assert sims[0].stats()["iters"] == sims[1].stats()["iters"]
    for s in sims[1:]:
        s.step(4)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI, M.MAZE_Y):
        assert np.array_equal(sims[1].get(what), sims[2].get(what))
    for s in sims:
        s.close()
