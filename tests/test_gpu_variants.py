"""GPU parity of the paper's variants (Sec. III.A, Eq. F_Benoit) against the
FP64 oracle, through the C ABI:

* the direct Poisson baselines: multigrid (or CG) on Eq. linearproblem
  started from phi^k ("static") or from 2 phi^k - phi^{k-1}
  ("time-propagated"), stopping on Eq. res_poisson;
* the force estimator of Eq. F_Benoit (minus the gradient of the weights).
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth
from tests.test_gpu_parity import SOLVERS, case, force_err

pytestmark = pytest.mark.gpu

SCHEMES = {"mg-static": M.MAZE_SCHEME_MG_STATIC, "mg-timeprop": M.MAZE_SCHEME_MG_TIMEPROP,
           "maze": M.MAZE_SCHEME_MAZE}
PRECISIONS = {"fp64-mg": ("mg", M.MAZE_FP64, 1e-9, 1e-12), "fp64-cg": ("cg", M.MAZE_FP64, 1e-9, 1e-12),
              "mixed-mg": ("mg", M.MAZE_MIXED, 1e-5, 1e-9)}


def make(name, scheme, prec, force="cd"):
    solver, precision, bar, tol = PRECISIONS[prec]
    pos, vel, types, L, N, rc, P = case(name)
    tf = synth.tosi_fumi_nacl()
    fe = M.MAZE_FORCE_GRADW if force == "gradw" else M.MAZE_FORCE_CD
    sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=tol, order=P, solver=SOLVERS[solver],
                    precision=precision, scheme=SCHEMES[scheme], force_estimator=fe)
    # step 0 of the oracle to the same tolerance in the units of its scheme's
    # first solve (step 0 always solves the constraint, in units of e)
    p = O.Params(L=L, N=N, dt=1.0, tol=tol, rc=rc, P=P, solver=solver, scheme=scheme, force=force)
    return sim, p, tf, (pos, vel, types), bar


@pytest.mark.parametrize("prec", list(PRECISIONS))
@pytest.mark.parametrize("scheme", ["mg-static", "mg-timeprop"])
def test_direct_schemes(scheme, prec):
    sim, p, tf, (pos, vel, types), bar = make("nacl64", scheme, prec)
    st = O.init(pos, vel, types, p, tf)
    for k in range(6):
        st = O.step(st, p, tf)
        sim.step(1)
        s = sim.stats()
        assert s["status"] == 0
        # the reported residual is Eq. res_poisson's, below tol
        assert s["resid"] < p.tol
        assert abs(s["iters"] - st.iters) <= 1, (k, s["iters"], st.iters)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < bar
    # the constraint of the direct scheme on the GPU's own state
    x = sim.get(M.MAZE_POS)
    phi = sim.get(M.MAZE_PHI)
    Q = np.where(types == 0, 1.0, -1.0)
    q = O.spread(x, Q, p.L, p.N, p.P)
    slack = 2e-5 if prec == "mixed-mg" else 1e-9     # FP32 spreading of q (x 4pi/h) in mixed precision
    assert O.inf_norm(O.apply_M(phi) + (4 * np.pi / p.h) * q) < p.tol + slack
    sim.close()


def test_schemes_order_of_vcycles():
    """Sec. III.A: on a molten box the MaZe solve needs the fewest V-cycles,
    the time-propagated direct solve more, the static one the most (same
    tolerance on each scheme's own residual)."""
    its = {}
    for scheme in ("maze", "mg-timeprop", "mg-static"):
        pos, vel, types, L, N, rc, P = case("nacl1000")
        tf = synth.tosi_fumi_nacl()
        sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=1e-7, order=P,
                        solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, scheme=SCHEMES[scheme])
        sim.step(20)
        a = sim.stats()["total_iters"]
        sim.step(40)
        its[scheme] = (sim.stats()["total_iters"] - a) / 40
        sim.close()
    assert its["maze"] < its["mg-timeprop"] < its["mg-static"], its


@pytest.mark.parametrize("prec", ["fp64-mg", "mixed-mg"])
@pytest.mark.parametrize("name", ["nacl64", "nacl64_P2", "nacl1000"])
def test_gradw_estimator(name, prec):
    sim, p, tf, (pos, vel, types), bar = make(name, "maze", prec, force="gradw")
    st = O.init(pos, vel, types, p, tf)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < bar
    for _ in range(3):
        st = O.step(st, p, tf)
    sim.step(3)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < bar
    # it is a different estimator: the central-difference forces differ
    Fcd = O.gather_forces(st.pos, np.where(types == 0, 1.0, -1.0), st.phi, p.L, p.N, p.P) + st.F_tf
    assert force_err(Fcd, st.F) > 10 * bar
    sim.close()


def test_batch_runs_the_variants():
    """A batch holding boxes of every scheme and estimator matches each box
    run alone, bit for bit."""
    specs = [("maze", "cd"), ("mg-static", "cd"), ("mg-timeprop", "gradw"), ("maze", "gradw")]
    w = synth.replica(512, 5)
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    b = M.MazeBatch(1 << 30, 4)
    ids = []
    for scheme, force in specs:
        fe = M.MAZE_FORCE_GRADW if force == "gradw" else M.MAZE_FORCE_CD
        ids.append(b.add(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=1e-9, order=w.order,
                         scheme=SCHEMES[scheme], force_estimator=fe))
    b.step(5)
    for i, (scheme, force) in zip(ids, specs):
        fe = M.MAZE_FORCE_GRADW if force == "gradw" else M.MAZE_FORCE_CD
        sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, r_cut=w.rc, dt=w.dt, tol=1e-9, order=w.order,
                        solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, scheme=SCHEMES[scheme],
                        force_estimator=fe)
        sim.step(5)
        for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI):
            assert np.array_equal(b.get(i, what), sim.get(what)), (scheme, force, what)
        sim.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64-mg", "mixed-mg"])
def test_ovrvo_langevin_matches_oracle(prec):
    """OVRVO with the same Philox key: the GPU draws the same Gaussian numbers
    (integer-exact generator), so the trajectories agree to the force bar."""
    solver, precision, bar, tol = PRECISIONS[prec]
    pos, vel, types, L, N, rc, P = case("nacl64")
    tf = synth.tosi_fumi_nacl()
    kw = dict(langevin_gamma=0.02, langevin_T=1500.0, seed=0x1234567890AB)
    sim = M.MazeSim(pos, vel, types, L, N, tf, r_cut=rc, dt=1.0, tol=tol, order=P, solver=SOLVERS[solver],
                    precision=precision, **kw)
    p = O.Params(L=L, N=N, dt=1.0, tol=tol, rc=rc, P=P, solver=solver, gamma=kw["langevin_gamma"],
                 T_bath=kw["langevin_T"], seed=kw["seed"])
    st = O.init(pos, vel, types, p, tf)
    # first step: velocities carry the O-step noise of both O steps
    st = O.step(st, p, tf)
    sim.step(1)
    v = sim.get(M.MAZE_VEL)
    assert np.abs(v - st.vel).max() < 1e-6 * np.abs(st.vel).max()
    for _ in range(7):
        st = O.step(st, p, tf)
    sim.step(7)
    assert force_err(sim.get(M.MAZE_FORCE), st.F) < bar * 100
    assert np.abs(sim.get(M.MAZE_POS) - st.pos).max() < 1e-6
    sim.close()


def test_o_step_noise_is_bit_exact():
    """Uncharged, non-interacting ions: the step is pure O-V-R-V-O with zero
    forces, so the velocities are a v + sd xi composed twice; the GPU's Philox
    numbers must equal the oracle's to the last bit (any differing bit changes
    xi at O(1))."""
    n = 64
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    zero = synth.TosiFumi(A=(0.0,) * 3, B=1.0, s=(0.0,) * 3, C=(0.0,) * 3, D=(0.0,) * 3)
    kw = dict(langevin_gamma=0.5, langevin_T=1000.0, seed=77)
    sim = M.MazeSim(pos, vel, types, w.L, w.N, zero, r_cut=w.rc, dt=1.0, tol=1e-10, solver=M.MAZE_SOLVER_MG,
                    charge=(0.0, 0.0), **kw)
    p = O.Params(L=w.L, N=w.N, dt=1.0, tol=1e-10, rc=w.rc, solver="mg", charge=(0.0, 0.0),
                 gamma=0.5, T_bath=1000.0, seed=77)
    st = O.init(pos, vel, types, p, zero)
    for _ in range(3):
        st = O.step(st, p, zero)
    sim.step(3)
    assert np.abs(sim.get(M.MAZE_VEL) - st.vel).max() < 1e-12 * np.abs(st.vel).max()
    assert n == len(types)
    sim.close()


def test_batch_langevin_box_equals_alone():
    w = synth.replica(216, 8)
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    kw = dict(r_cut=w.rc, dt=w.dt, tol=1e-9, order=w.order, langevin_gamma=0.01, langevin_T=1200.0, seed=3)
    b = M.MazeBatch(1 << 30, 2)
    i = b.add(pos, vel, types, w.L, w.N, tf, **kw)
    b.step(6)
    sim = M.MazeSim(pos, vel, types, w.L, w.N, tf, solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, **kw)
    sim.step(6)
    for what in (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE):
        assert np.array_equal(b.get(i, what), sim.get(what))
    sim.close()
    b.close()
