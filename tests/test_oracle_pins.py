"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties one part of the oracle to mathematics or to a value fixed
outside it: a dense matrix written from the footnote's definition of M, the
closed-form eigenvalues of a circulant operator, a dense pseudo-inverse,
textbook B-spline values, the rock-salt Madelung constant through an
independent Ewald sum, Ewald forces, momentum conservation (Sec. II.A),
energy conservation of V_work (Eq. E_nostra, Sec. III.C), time
reversibility (Sec. III.C) and the SHAKE identity (Eqs. SHAKEy, SHAKEPhiFinal).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import synth
from tests.ewald import ewald

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def madelung():
    with open(os.path.join(GOLDEN, "madelung_nacl.txt")) as f:
        return float([l for l in f if not l.startswith("#")][0])


def dense_M(N):
    """M from the footnote: -6 on the diagonal, +1 for each of the six
    periodic neighbours in (i, j, k), flat index n = i + jN + kN^2."""
    n = N ** 3
    A = np.zeros((n, n))
    for k in range(N):
        for j in range(N):
            for i in range(N):
                a = i + j * N + k * N * N
                A[a, a] += -6.0
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    b = (i + di) % N + ((j + dj) % N) * N + ((k + dk) % N) * N * N
                    A[a, b] += 1.0
    return A


def flat(v):
    return v.ravel()  # [k, j, i] C-order -> n = i + jN + kN^2


@pytest.mark.parametrize("N", [3, 4, 5])
def test_apply_M_matches_dense_footnote(N):
    A = dense_M(N)
    rng = np.random.default_rng(N)
    x = rng.normal(size=(N, N, N))
    np.testing.assert_allclose(flat(O.apply_M(x)), A @ flat(x), rtol=0, atol=1e-13)
    assert np.allclose(A, A.T)  # symmetric, as the footnote recalls


def test_plane_waves_are_eigenvectors():
    N = 6
    lam = O.M_eigenvalues(N)
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    for kz, ky, kx in ((0, 0, 1), (1, 2, 3), (5, 0, 2)):
        wave = np.cos(2 * np.pi * (kx * i + ky * j + kz * k) / N)
        np.testing.assert_allclose(O.apply_M(wave), lam[kz, ky, kx] * wave, atol=1e-12)
    assert lam[0, 0, 0] == 0.0 and lam.max() <= 0 and math.isclose(lam.min(), -12.0)


@pytest.mark.parametrize("N", [4, 6])
def test_exact_solve_is_pseudo_inverse(N):
    A = dense_M(N)
    rng = np.random.default_rng(1)
    b = rng.normal(size=(N, N, N))
    b -= b.mean()
    ref = np.linalg.lstsq(A, flat(b), rcond=None)[0]
    np.testing.assert_allclose(flat(O.solve_exact(b)), ref, atol=1e-11)


@pytest.mark.parametrize("solver", ["cg", "mg"])
def test_iterative_solvers_vs_dense_lstsq(solver):
    """P8: N = 8, dense 512 x 512 M solved by lstsq vs the oracle's PLCG and MG."""
    N = 8
    A = dense_M(N)
    rng = np.random.default_rng(2)
    b = rng.normal(size=(N, N, N))
    b -= b.mean()
    ref = np.linalg.lstsq(A, flat(b), rcond=None)[0]
    y, info = O.solve(b, np.zeros_like(b), 1e-12, solver)
    assert info.converged and info.resid < 1e-12
    np.testing.assert_allclose(flat(y - y.mean()), ref - ref.mean(), atol=1e-11)
    assert np.max(np.abs(A @ flat(y) - flat(b))) < 1e-12


def test_plcg_warm_start_no_work():
    N = 8
    rng = np.random.default_rng(3)
    b = rng.normal(size=(N, N, N))
    b -= b.mean()
    y = O.solve_exact(b)
    _, info = O.plcg(b, y, 1e-10)
    assert info.iters == 0


def test_mg_transfer_operators():
    """Full weighting is 1/8 of the transpose of trilinear prolongation, both
    preserve constants, and one V-cycle contracts the error strongly."""
    rng = np.random.default_rng(4)
    u = rng.normal(size=(8, 8, 8))
    v = rng.normal(size=(4, 4, 4))
    lhs = np.sum(O.restrict_fw(u) * v)
    rhs = np.sum(u * O.prolong_trilinear(v)) / 8.0
    assert abs(lhs - rhs) < 1e-12
    np.testing.assert_allclose(O.restrict_fw(np.full((8, 8, 8), 3.0)), 3.0)
    np.testing.assert_allclose(O.prolong_trilinear(np.full((4, 4, 4), 2.0)), 2.0)
    # prolongation of a linear-in-x coarse field is linear where no wrap occurs
    ramp = np.broadcast_to(np.arange(4.0)[None, None, :], (4, 4, 4))
    fine = O.prolong_trilinear(ramp)
    np.testing.assert_allclose(fine[0, 0, :7], np.arange(7) / 2.0)
    # V-cycle convergence factor on a random zero-mean rhs
    N = 32
    b = rng.normal(size=(N, N, N))
    b -= b.mean()
    x = np.zeros_like(b)
    r0 = O.inf_norm(b)
    x = O.vcycle(x, b, 1e-12)
    r1 = O.inf_norm(b - O.apply_M(x))
    x = O.vcycle(x, b, 1e-12)
    r2 = O.inf_norm(b - O.apply_M(x))
    assert r1 / r0 < 0.2 and r2 / r1 < 0.2


def test_rbgs_is_gauss_seidel():
    """A red half-sweep sets each red point so that its residual vanishes."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(6, 6, 6))
    b = rng.normal(size=(6, 6, 6))
    red = O.red_mask(6)
    nb = O.apply_M(x) + 6 * x
    xr = np.where(red, (nb - b) / 6.0, x)
    r = b - O.apply_M(xr)
    assert np.max(np.abs(r[red])) < 1e-12
    xs = O.rbgs_sweep(x, b)
    r = b - O.apply_M(xs)
    assert np.max(np.abs(r[~red])) < 1e-12      # black points are exact after the sweep


def test_bspline_textbook_values():
    # cubic B-spline at integer and half-integer offsets
    np.testing.assert_allclose(O.bspline(np.array([-1.0, 0.0, 1.0, 2.0]), 4), [1 / 6, 2 / 3, 1 / 6, 0.0])
    np.testing.assert_allclose(O.bspline(np.array([-1.5, -0.5, 0.5, 1.5]), 4), [1 / 48, 23 / 48, 23 / 48, 1 / 48])
    np.testing.assert_allclose(O.bspline(np.array([0.25, -0.75]), 2), [0.75, 0.25])
    # partition of unity and reproduction of linear functions, random offsets
    rng = np.random.default_rng(6)
    pos = rng.uniform(0, 10, size=(50, 3))
    for P in (2, 4):
        nodes, dist = O.support(pos, 10.0, 10, P)
        w = O.bspline(dist, P)
        np.testing.assert_allclose(w.sum(-1), 1.0, atol=1e-14)
        np.testing.assert_allclose((w * dist).sum(-1), 0.0, atol=1e-14)
    # derivative is the derivative
    d = np.linspace(-2.2, 2.2, 41)
    for P in (2, 4):
        fd = (O.bspline(d + 1e-6, P) - O.bspline(d - 1e-6, P)) / 2e-6
        ok = np.abs(np.abs(d) - np.round(np.abs(d))) > 1e-3
        np.testing.assert_allclose(O.bspline_deriv(d, P)[ok], fd[ok], atol=1e-6)


@pytest.mark.parametrize("P", [2, 4])
def test_spread_conserves_charge_and_dipole(P):
    rng = np.random.default_rng(7)
    L, N = 10.0, 20
    pos = rng.uniform(3.0, 7.0, size=(12, 3))      # away from the periodic seam
    Q = rng.normal(size=12)
    q = O.spread(pos, Q, L, N, P)
    assert abs(q.sum() - Q.sum()) < 1e-12
    h = L / N
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    for c, idx in enumerate((i, j, k)):
        assert abs((q * idx * h).sum() - (Q * pos[:, c]).sum()) < 1e-11
    # an ion on a node with P = 2 puts all of its charge on that node
    q1 = O.spread(np.array([[2.0, 3.0, 4.5]]), np.array([1.0]), L, N, 2)
    assert q1[9, 6, 4] == 1.0 and abs(q1).sum() == 1.0


def test_madelung_from_ewald_and_grid():
    """P3: an independent Ewald sum gives the rock-salt Madelung energy; the
    grid energy (self-energy removed, App. A) converges to it as h^2."""
    Mad = madelung()
    L, n = 12.6, 4
    d = L / n
    pos, types = synth.rocksalt(n, L, 0.0, np.random.default_rng(0))
    Q = np.where(types == 0, 1.0, -1.0)
    E, F = ewald(pos, Q, L)
    ref = -Mad * (len(Q) / 2) * O.K_E / d
    assert abs(E * O.K_E - ref) < 1e-9 * abs(ref)
    assert np.abs(F).max() < 1e-12
    E1, _ = ewald(pos[:1], np.array([1.0]), L)     # one charge + background
    errs = []
    for N in (16, 32, 64):
        p = O.Params(L=L, N=N, dt=1.0, tol=1e-12)
        phi, q = O.exact_potential(pos, types, p)
        Vd = O.discrete_energy(q, phi)
        q1 = O.spread(pos[:1], np.array([1.0]), L, N, 4)
        q1 -= q1.mean()
        Es = O.discrete_energy(q1, -(4 * np.pi / p.h) * O.solve_exact(q1))
        est = Vd - len(Q) * (Es - E1 * O.K_E)
        errs.append(abs(est - ref))
        # on the perfect lattice aligned with the grid the field force vanishes
        assert np.abs(O.gather_forces(pos, Q, phi, L, N, 4)).max() < 1e-12
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0   # O(h^2)
    assert errs[2] < 0.005 * abs(ref)


@pytest.mark.parametrize("P", [2, 4])
def test_forces_converge_to_ewald(P):
    """P4: random 8-ion box; grid forces approach Ewald forces as h shrinks."""
    L = 10.0
    pos, types = synth.random_neutral(8, L, 7, min_dist=2.0)
    Q = np.where(types == 0, 1.0, -1.0)
    _, Fe = ewald(pos, Q, L)
    Fe *= O.K_E
    errs = []
    for N in (16, 32, 64):
        p = O.Params(L=L, N=N, dt=1.0, tol=1e-12, P=P)
        phi, _ = O.exact_potential(pos, types, p)
        F = O.gather_forces(pos, Q, phi, L, N, P)
        errs.append(np.abs(F - Fe).max() / np.abs(Fe).max())
        # P5: momentum conservation of Eq. F_nostra
        assert np.abs(F.sum(0)).max() < 1e-12 * np.abs(F).sum()
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.005


def test_tilde_force_breaks_momentum():
    """Eq. F_Benoit does not conserve momentum, Eq. F_nostra does (Sec. II.A)."""
    L, N = 10.0, 16
    pos, types = synth.random_neutral(8, L, 11, min_dist=2.0)
    Q = np.where(types == 0, 1.0, -1.0)
    p = O.Params(L=L, N=N, dt=1.0, tol=1e-12)
    phi, _ = O.exact_potential(pos, types, p)
    F = O.gather_forces(pos, Q, phi, L, N, 4)
    Ft = O.gather_forces_tilde(pos, Q, phi, L, N, 4)
    assert np.abs(F.sum(0)).max() < 1e-12
    assert np.abs(Ft.sum(0)).max() > 1e-6
    # F~ is exactly minus the gradient of the discrete energy 1/2 phi^T q,
    # self-energy included (that is where its noise comes from)
    eps = 1e-5
    for a, c in ((0, 0), (3, 2), (5, 1)):
        e = []
        for sgn in (1, -1):
            pp = pos.copy(); pp[a, c] += sgn * eps
            ph, q = O.exact_potential(pp, types, p)
            e.append(O.discrete_energy(q, ph))
        fd = -(e[0] - e[1]) / (2 * eps)
        assert abs(fd - Ft[a, c]) < 1e-5 * max(1.0, abs(Ft[a, c]))


def test_tf_force_is_minus_gradient():
    tf = synth.tosi_fumi_nacl()
    L = 12.0
    pos, types = synth.random_neutral(6, L, 3, min_dist=2.2)
    F, V = O.tf_forces(pos, types, L, tf, 6.0)
    assert np.abs(F.sum(0)).max() < 1e-10
    eps = 1e-6
    for a in range(3):
        for c in range(3):
            pp = pos.copy(); pp[a, c] += eps
            pm = pos.copy(); pm[a, c] -= eps
            fd = -(O.tf_forces(pp, types, L, tf, 6.0)[1] - O.tf_forces(pm, types, L, tf, 6.0)[1]) / (2 * eps)
            assert abs(fd - F[a, c]) < 1e-6 * max(1.0, abs(F[a, c]))
    np.testing.assert_allclose(O.tf_forces_on([0, 4], pos, types, L, tf, 6.0), F[[0, 4]], atol=1e-12)


def test_tf_pair_energy_at_contact():
    """With the dispersion terms removed, the pair energy at r = s is A."""
    tf = synth.tosi_fumi_nacl()
    t0 = synth.TosiFumi(A=tf.A, B=tf.B, s=tf.s, C=(0.0,) * 3, D=(0.0,) * 3)
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + tf.s[1], 1.0, 1.0]])
    _, V = O.tf_forces(pos, np.array([0, 1], dtype=np.int32), 20.0, t0, 1e9)
    assert abs(V - tf.A[1]) < 1e-14


def _short_run(n_steps, tol=1e-10, solver="cg", reverse=False):
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=tol, rc=w.rc, solver=solver)
    rec = []
    st = O.run(pos, vel, types, p, tf, n_steps, rec)
    return w, p, tf, rec


def test_nve_work_energy_conserved():
    """P6: with V_work the total energy is conserved far better than its parts
    fluctuate (the paper reports Delta E / Delta V_work = 2.2e-5 at h = 0.172)."""
    w, p, tf, rec = _short_run(60)
    E = np.array([O.energies(s, p)["e_tot"] for s in rec])
    Vw = np.array([s.V_work for s in rec])
    KE = np.array([O.kinetic(s, p) for s in rec])
    assert E.std() / Vw.std() < 2e-4
    assert E.std() / KE.std() < 2e-3
    assert all(s.resid < p.tol for s in rec)


def test_shake_identity_and_constraint():
    """P2/P9: after each step the constraint (h/4pi) M phi + q = 0 holds to the
    solver tolerance, and phi equals the exact discrete potential."""
    w, p, tf, rec = _short_run(5, tol=1e-12)
    for s in rec[1:]:
        Q = np.where(s.types == 0, 1.0, -1.0)
        q = O.spread(s.pos, Q, p.L, p.N, p.P)
        sig = (p.h / (4 * np.pi)) * O.apply_M(s.phi) + q
        assert O.inf_norm(sig) < 2e-12
        ex, _ = O.exact_potential(s.pos, s.types, p)
        assert O.inf_norm(s.phi - s.phi.mean() - ex) < 1e-9


def test_static_system_needs_no_solver_work():
    """With ions at rest on the lattice the Verlet proposal phi_p = 2 phi^k -
    phi^{k-1} already satisfies the constraint, so SHAKE needs 0 iterations."""
    L, n = 12.6, 4
    pos, types = synth.rocksalt(n, L, 0.0, np.random.default_rng(0))
    tf = synth.TosiFumi(A=(0.0,) * 3, B=1.0, s=(0.0,) * 3, C=(0.0,) * 3, D=(0.0,) * 3)
    p = O.Params(L=L, N=16, dt=1.0, tol=1e-10, rc=6.3)
    st = O.init(pos, np.zeros_like(pos), types, p, tf)
    for _ in range(3):
        st = O.step(st, p, tf)
        assert st.iters == 0


def test_maze_start_beats_static_start():
    """Sec. III.A.1 / App. B: warm-started SHAKE needs fewer iterations than a
    direct Poisson solve started from the previous potential."""
    w, p, tf, rec = _short_run(12, solver="cg")
    maze_it, static_it = [], []
    for prev, cur in zip(rec[5:-1], rec[6:]):
        maze_it.append(cur.iters)
        Q = np.where(cur.types == 0, 1.0, -1.0)
        q = O.spread(cur.pos, Q, p.L, p.N, p.P)
        # direct Poisson M phi = -4 pi q / h from phi^k, same residual units (e)
        b = q
        y0 = -(p.h / (4 * np.pi)) * prev.phi
        _, info = O.plcg(b, y0, p.tol)
        static_it.append(info.iters)
    assert np.mean(maze_it) < np.mean(static_it)


def test_time_reversibility():
    """Sec. III.C: run forward, flip the velocities and the phi history, run
    back; the positions return (tight tolerance)."""
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-12, rc=w.rc)
    st = O.init(pos, vel, types, p, tf)
    start = st.pos.copy()
    for _ in range(20):
        st = O.step(st, p, tf)
    st.vel = -st.vel
    st.phi, st.phi_prev = st.phi_prev, st.phi
    st.y = np.zeros_like(st.y)
    for _ in range(20):
        st = O.step(st, p, tf)
    d = st.pos - start
    d -= p.L * np.round(d / p.L)
    rmsd = np.sqrt((d * d).sum(1)).sum() / (len(d) * p.L)
    assert rmsd < 1e-8


def test_cg_and_mg_agree_on_trajectory():
    """The two constraint solvers (App. B and Sec. III.A) give the same
    trajectory to the force tolerance when the constraint is tight."""
    _, p1, _, r1 = _short_run(10, tol=1e-13, solver="cg")
    _, p2, _, r2 = _short_run(10, tol=1e-13, solver="mg")
    for a, b in zip(r1, r2):
        assert np.abs(a.F - b.F).max() < 1e-10 * np.abs(a.F).max()


# ---------------------------------------------------------------------------
# The direct Poisson baselines of Sec. III.A (static / time-propagated start)

@pytest.mark.parametrize("scheme", ["mg-static", "mg-timeprop"])
def test_direct_schemes_reach_the_exact_potential(scheme):
    """A direct solve of Eq. linearproblem to max|M phi + 4 pi q/h| < tol lands
    on the DFT solution: |phi - phi_exact| <= ||M^+||_inf tol."""
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    p = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-9, rc=w.rc, solver="mg", scheme=scheme)
    st = O.init(pos, vel, types, p, tf)
    for _ in range(4):
        st = O.step(st, p, tf)
        assert st.resid < p.tol and st.iters >= 1
        phi_ex, q = O.exact_potential(st.pos, st.types, p)
        # residual of Eq. res_poisson recomputed from scratch
        assert O.inf_norm(O.apply_M(st.phi) + (4 * np.pi / p.h) * q) < p.tol
        # ||M^+||_inf <= N^3 / min|lambda| bounds the error of a tol-residual
        lam = np.abs(O.M_eigenvalues(p.N)).ravel()
        bound = p.N ** 3 / lam[lam > 1e-12].min() * p.tol
        assert O.inf_norm(st.phi - phi_ex) < bound


def test_timeprop_from_zero_y_is_the_maze_step():
    """With y^0 = 0 (the first step after step 0) the SHAKE solve is, by
    linearity, the direct solve started from phi_p = 2 phi^k - phi^{k-1}:
    phi^nu = phi_p - (4 pi/h) y^nu iterate by iterate, so the two take the
    same number of V-cycles when the tolerances match (tol_direct =
    (4 pi/h) tol_maze) and end on the same potential."""
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    pm = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-10, rc=w.rc, solver="mg")
    pd = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-10 * 4 * np.pi / pm.h, rc=w.rc, solver="mg",
                  scheme="mg-timeprop")
    st = O.init(pos, vel, types, pm, tf)
    a = O.step(st, pm, tf)
    b = O.step(st, pd, tf)
    assert a.iters == b.iters >= 2
    assert np.abs(a.phi - b.phi).max() < 1e-9 * np.abs(a.phi).max()


@pytest.mark.parametrize("scheme", ["mg-static", "mg-timeprop"])
def test_direct_schemes_still_system_needs_no_work(scheme):
    """Ions at rest: the start value (phi^k, or 2 phi^k - phi^{k-1} = phi^k)
    already solves Eq. linearproblem, so no V-cycle runs."""
    L, n = 12.6, 4
    pos, types = synth.rocksalt(n, L, 0.0, np.random.default_rng(0))
    tf = synth.TosiFumi(A=(0.0,) * 3, B=1.0, s=(0.0,) * 3, C=(0.0,) * 3, D=(0.0,) * 3)
    p = O.Params(L=L, N=16, dt=1.0, tol=1e-8, rc=6.3, solver="mg", scheme=scheme)
    # step 0 to a tolerance well inside the direct one ((4 pi/h) 1e-12 << 1e-8)
    p0 = O.Params(L=L, N=16, dt=1.0, tol=1e-12, rc=6.3, solver="mg")
    st = O.init(pos, np.zeros_like(pos), types, p0, tf)
    for _ in range(3):
        st = O.step(st, p, tf)
        assert st.iters == 0


# ---------------------------------------------------------------------------
# OVRVO Langevin (Sec. III) and its counter-based Gaussian numbers

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr = tuple(np.array([c], dtype=np.uint64) for c in v[:4])
        out = O.philox4x32(ctr, (v[4], v[5]))
        assert [int(o[0]) for o in out] == v[6:]


def test_gaussians_have_unit_normal_moments():
    z = np.concatenate([O.gaussians(20000, s, st, 12345) for s in range(5) for st in (0, 1)]).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs((z ** 4).mean() - 3) < 5 * math.sqrt(96 / n)
    # distinct counters are uncorrelated; the same counter repeats
    a, b = O.gaussians(20000, 7, 0, 1), O.gaussians(20000, 7, 1, 1)
    assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 5 / math.sqrt(a.size)
    assert np.array_equal(a, O.gaussians(20000, 7, 0, 1))
    assert not np.array_equal(a, O.gaussians(20000, 7, 0, 2))


def test_o_step_preserves_and_reaches_maxwell():
    """The O step is an exact Ornstein-Uhlenbeck update: v ~ N(0, kT/m) stays
    N(0, kT/m); from v = 0 the variance after one step is (1 - a^2) kT/m."""
    n = 50000
    types = (np.arange(n) % 2).astype(np.int32)
    p = O.Params(L=10.0, N=8, dt=1.0, tol=1e-8, gamma=0.05, T_bath=1200.0, seed=99)
    m = np.asarray(p.mass)[types][:, None]
    kt_m = O.K_B * p.T_bath * O.ACC / m
    v0 = np.sqrt(kt_m) * np.random.default_rng(3).normal(size=(n, 3))
    v1 = O.o_step(v0, types, p, 0, 0)
    ratio = (v1 ** 2 / kt_m).mean()
    assert abs(ratio - 1) < 5 * math.sqrt(2 / (3 * n))
    a = math.exp(-p.gamma * p.dt / 2)
    v2 = O.o_step(np.zeros((n, 3)), types, p, 0, 1)
    assert abs((v2 ** 2 / kt_m).mean() - (1 - a * a)) < 5 * (1 - a * a) * math.sqrt(2 / (3 * n))


def test_ovrvo_tends_to_verlet_and_thermalises():
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    tf = synth.tosi_fumi_nacl()
    # gamma -> 0: the O steps vanish, the trajectory is velocity Verlet's (the
    # noise left at gamma = 1e-13 moves ions by ~1e-8 Angstrom in 5 steps)
    pv = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-10, rc=w.rc, solver="mg")
    pl = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-10, rc=w.rc, solver="mg", gamma=1e-13, T_bath=1200.0, seed=5)
    a = O.run(pos, vel, types, pv, tf, 5)
    b = O.run(pos, vel, types, pl, tf, 5)
    assert np.abs(a.pos - b.pos).max() < 1e-6
    # strong friction towards a hot bath from a cold start heats the ions
    cold = np.zeros_like(vel)
    ph = O.Params(L=w.L, N=w.N, dt=w.dt, tol=1e-8, rc=w.rc, solver="mg", gamma=0.2, T_bath=3000.0, seed=6)
    st = O.run(pos, cold, types, ph, tf, 30)
    T = 2 * O.kinetic(st, ph) / (3 * len(types) * O.K_B)
    assert 1500 < T < 6000


# ---------------------------------------------------------------------------
# Unit constants (Sec. II Gaussian units; Sec. III Angstrom / fs / amu) against
# published CODATA 2018 values reached by other routes than the oracle's.

def codata():
    out = {}
    with open(os.path.join(GOLDEN, "codata2018.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def header_constants():
    """The unit constants the CUDA path compiles in (include/maze.h)."""
    out = {}
    with open(os.path.join(os.path.dirname(GOLDEN), "..", "include", "maze.h")) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == "#define" and parts[1] in (
                    "MAZE_KE_EV_ANGSTROM", "MAZE_ACC_UNIT", "MAZE_KB_EV_PER_K"):
                out[parts[1]] = float(parts[2])
    return out


def test_unit_constants_match_codata_2018():
    c = codata()
    ke = c["hartree_energy_eV"] * c["bohr_radius_angstrom"]       # e^2/(4 pi eps0) = E_h a_0
    acc = c["faraday_C_per_mol"] / c["molar_mass_constant_kg_per_mol"] * 1e-10   # e/u, (m/s^2 -> A/fs^2)
    kb = c["boltzmann_eV_per_K"]
    assert abs(O.K_E / ke - 1.0) < 1e-9
    assert abs(O.ACC / acc - 1.0) < 1e-9
    assert abs(O.K_B / kb - 1.0) < 1e-9
    h = header_constants()
    assert set(h) == {"MAZE_KE_EV_ANGSTROM", "MAZE_ACC_UNIT", "MAZE_KB_EV_PER_K"}
    assert abs(h["MAZE_KE_EV_ANGSTROM"] / ke - 1.0) < 1e-9
    assert abs(h["MAZE_ACC_UNIT"] / acc - 1.0) < 1e-9
    assert abs(h["MAZE_KB_EV_PER_K"] / kb - 1.0) < 1e-9
    # a slip by a power of ten (or a missing 4 pi) fails these by orders of magnitude
    assert 14.39 < O.K_E < 14.40 and 9.64e-3 < O.ACC < 9.65e-3


def test_tf_energy_is_continuous_at_the_cutoff():
    """Reading G9: the pair energy is shifted by V(r_c), so a pair entering or
    leaving the cutoff sphere changes V_TF by (almost) nothing, while the
    unshifted energy would jump by V(r_c)."""
    tf = synth.tosi_fumi_nacl()
    L, rc = 40.0, 9.0
    types = np.array([0, 1], dtype=np.int32)
    for eps in (1e-6, 1e-9):
        inside = np.array([[5.0, 5.0, 5.0], [5.0 + rc - eps, 5.0, 5.0]])
        outside = np.array([[5.0, 5.0, 5.0], [5.0 + rc + eps, 5.0, 5.0]])
        _, Vin = O.tf_forces(inside, types, L, tf, rc)
        _, Vout = O.tf_forces(outside, types, L, tf, rc)
        F, _ = O.tf_forces(inside, types, L, tf, rc)
        assert Vout == 0.0
        # the shifted energy just inside the cutoff is |dV/dr| * eps to first order
        assert abs(Vin) <= 2.0 * np.abs(F[0, 0]) * eps + 1e-15
    # and the shift is the unshifted pair energy at r_c
    V_rc = tf.A[1] * math.exp(tf.B * (tf.s[1] - rc)) - tf.C[1] / rc ** 6 - tf.D[1] / rc ** 8
    assert abs(V_rc) > 1e-6            # the jump the shift removes (~1.3e-5 eV for Na-Cl at 9 A)
    near = np.array([[5.0, 5.0, 5.0], [5.0 + 3.0, 5.0, 5.0]])
    _, Vn = O.tf_forces(near, types, L, tf, rc)
    Vn_raw = tf.A[1] * math.exp(tf.B * (tf.s[1] - 3.0)) - tf.C[1] / 3.0 ** 6 - tf.D[1] / 3.0 ** 8
    assert abs(Vn - (Vn_raw - V_rc)) < 1e-12


@pytest.mark.parametrize("n_ions,rc", [(64, 4.0), (216, 6.0), (216, 9.0), (1000, 9.0), (1000, 5.0)])
def test_cell_list_pairs_equal_all_pairs(n_ions, rc):
    """The cell-list pair sum (large boxes) against the all-pairs loop: same
    pairs, same forces and energy up to summation order."""
    tf = synth.tosi_fumi_nacl()
    if n_ions == 64:
        w = synth.workload("nacl64")
    else:
        w = synth.replica(n_ions, 11 + n_ions)
    pos, _, types = synth.make_state(w)
    F1, V1 = O.tf_forces(pos, types, w.L, tf, rc)
    F2, V2 = O.tf_forces_cells(pos, types, w.L, tf, rc)
    scale = np.sqrt((F1 ** 2).sum(1).mean())
    assert np.abs(F2 - F1).max() <= 1e-12 * scale
    assert abs(V2 - V1) <= 1e-12 * abs(V1)
    assert np.abs(F2.sum(0)).max() < 1e-9 * scale * n_ions
