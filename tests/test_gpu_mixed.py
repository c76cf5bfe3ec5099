"""Mixed precision (FP32 V-cycle and grid arithmetic, double-float outer
SHAKE iteration, exact integer reductions) against the FP64 oracle.

Bar: per-ion force error |F - F_ref| / max(|F_ref|, rms|F_ref|) <= 1e-5 at the
configured tolerance; the constraint residual itself meets tol.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth
from tests.test_gpu_parity import case, force_err

pytestmark = pytest.mark.gpu

MIXED_BAR = 1e-5


def make(name, tol=1e-10, **kw):
    pos, vel, types, L, N, rc, P = case(name)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=tol, order=P,
                    solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, **kw)
    p = O.Params(L=L, N=N, dt=1.0, tol=tol, rc=rc, P=P, solver="mg")
    return sim, p, tf, (pos, vel, types)


@pytest.mark.parametrize("name", ["nacl64", "nacl64_P2", "nacl1000", "nacl216_N24", "nacl1728_N40", "tiny8_N8"])
def test_mixed_step0_and_one_step(name):
    sim, p, tf, (pos, vel, types) = make(name)
    st = O.init(pos, vel, types, p, tf)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < MIXED_BAR
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < p.tol
    st = O.step(st, p, tf)
    sim.step(1)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < MIXED_BAR
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < p.tol and abs(s["iters"] - st.iters) <= 1
    # the constraint holds on the whole grid for the GPU's own phi and q
    x = sim.get(M.MAZE_POS)
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(x, Q, p.L, p.N, p.P)
    sig = (p.h / (4 * np.pi)) * O.apply_M(sim.get(M.MAZE_PHI)) + q
    assert O.inf_norm(sig) < p.tol + 1e-6    # FP32 spreading of q
    sim.close()


def test_mixed_vcycles_match_fp64_over_trajectory():
    sim, p, tf, (pos, vel, types) = make("nacl1000")
    st = O.init(pos, vel, types, p, tf)
    for _ in range(20):
        st = O.step(st, p, tf)
        sim.step(1)
        assert abs(sim.stats()["iters"] - st.iters) <= 1
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < MIXED_BAR


def test_mixed_energy_conservation_and_determinism():
    a, p, tf, _ = make("nacl1000")
    b, _, _, _ = make("nacl1000")
    E, Vw = [], []
    for _ in range(50):
        a.step(2)
        s = a.stats()
        E.append(s["e_tot"])
        Vw.append(s["v_work"])
    assert np.std(E) / np.std(Vw) < 2e-4
    b.step(100)
    assert np.array_equal(a.get(M.MAZE_POS), b.get(M.MAZE_POS))
    blob = a.get_state()
    a.step(5)
    c, _, _, _ = make("nacl1000")
    c.set_state(blob)
    c.step(5)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_PHI, M.MAZE_Y):
        assert np.array_equal(a.get(what), c.get(what))
    for s in (a, b, c):
        s.close()


@pytest.mark.slow
def test_mixed_large_box_grid_form():
    """512000 ions / 256^3: the cooperative-grid form of the mixed solver."""
    w = synth.workload("nacl512000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol,
                    solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED)
    sim.step(1)
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < w.tol
    x = sim.get(M.MAZE_POS)
    phi = sim.get(M.MAZE_PHI)
    F = sim.get(M.MAZE_FORCE)
    Q = np.where(types == 0, 1.0, -1.0)
    idx = np.random.default_rng(9).choice(len(x), 48, replace=False)
    Fo = O.gather_forces(x[idx], Q[idx], phi, w.L, w.N, 4) + O.tf_forces_on(idx, x, types, w.L, tf, w.rc)
    scale = np.sqrt((F ** 2).sum(1).mean())
    err = np.linalg.norm(F[idx] - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), scale)
    assert err.max() < MIXED_BAR
    sim.close()


@pytest.mark.parametrize("n_ions", [4096, 13824])
def test_mixed_parity_on_the_largest_replica_grids(n_ions):
    """The largest grids of the batched boxes (4096 ions, 48^3: the
    multiply-high index decode on a non-power-of-two grid) and of the served
    boxes (13824 ions, 64^3: the V-cycle in global scratch instead of the
    cluster's shared memory), step 0 and one step against the oracle."""
    w = synth.replica(n_ions, 7000 + n_ions)
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    tol = 1e-10
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=tol, order=w.order,
                    solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED)
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=tol, rc=w.rc, P=w.order, solver="mg")
    st = O.init(pos, vel, types, p, tf)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < MIXED_BAR
    st = O.step(st, p, tf)
    sim.step(1)
    s = sim.stats()
    assert s["status"] == 0 and s["resid"] < tol and abs(s["iters"] - st.iters) <= 1
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < MIXED_BAR
    x = sim.get(M.MAZE_POS)
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(x, Q, p.L, p.N, p.P)
    sig = (p.h / (4 * np.pi)) * O.apply_M(sim.get(M.MAZE_PHI)) + q
    assert O.inf_norm(sig) < tol + 1e-6    # FP32 spreading of q
    sim.close()


def test_mixed_energies_against_the_oracle():
    """Mixed-precision energies against the FP64 oracle on the same 20-step
    trajectory (1000 ions): kinetic, Tosi-Fumi, discrete electrostatic
    (Eq. energy_discr), V_work (Eq. E_nostra) and their total within the
    mixed bar of 1e-5 relative (V_work, which starts at zero, relative to the
    kinetic plus pair energy); the constraint residual below tol on both."""
    sim, p, tf, (pos, vel, types) = make("nacl1000")
    st = O.init(pos, vel, types, p, tf)
    for _ in range(20):
        st = O.step(st, p, tf)
        sim.step(1)
    s = sim.stats()
    e = O.energies(st, p)
    for key in ("ke", "v_tf", "v_disc", "e_tot"):
        assert abs(s[key] - e[key]) <= MIXED_BAR * abs(e[key]), (key, s[key], e[key])
    assert abs(s["v_work"] - e["v_work"]) <= MIXED_BAR * (e["ke"] + abs(e["v_tf"]))
    assert s["resid"] < p.tol and st.resid < p.tol
    sim.close()


def test_mixed_once_per_pair_forces_large_box():
    """Mixed-precision boxes above 64^3 evaluate each Tosi-Fumi pair once
    (FP32 arithmetic, fixed-point per-ion sums): the 64000-ion / 128^3 box,
    sampled ions against the oracle's gather on the GPU's potential plus
    brute-force pairs, within the mixed bar; two runs bit for bit equal."""
    w = synth.workload("nacl64000")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    sims = [M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=w.tol, solver=M.MAZE_SOLVER_MG,
                      precision=M.MAZE_MIXED) for _ in range(2)]
    for s in sims:
        s.step(2)
    st = sims[0].stats()
    assert st["status"] == 0 and st["resid"] < w.tol
    x = sims[0].get(M.MAZE_POS)
    phi = sims[0].get(M.MAZE_PHI)
    F = sims[0].get(M.MAZE_FORCE)
    Q = np.where(types == 0, 1.0, -1.0)
    idx = np.random.default_rng(11).choice(len(x), 48, replace=False)
    Fo = O.gather_forces(x[idx], Q[idx], phi, w.L, w.N, 4) + O.tf_forces_on(idx, x, types, w.L, tf, w.rc)
    scale = np.sqrt((F ** 2).sum(1).mean())
    err = np.linalg.norm(F[idx] - Fo, axis=1) / np.maximum(np.linalg.norm(Fo, axis=1), scale)
    assert err.max() < MIXED_BAR
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE):
        assert np.array_equal(sims[0].get(what), sims[1].get(what))
    for s in sims:
        s.close()
