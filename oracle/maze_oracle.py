"""FP64 CPU oracle of the Poisson MaZe hot path (arxiv 2505.20418).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
baseline of bench.py; never by the product path. No code is shared with the
CUDA implementation.

Everything here is a direct restatement of the paper, in its notation:

  * grid of N^3 points, spacing h = L/N, flat index n = i + jN + kN^2
    (Sec. II, footnote to Eq. linearproblem); arrays are held as [k, j, i];
  * M = h^2-scaled 7-point periodic Laplacian, M phi = -4 pi q / h
    (Eq. linearproblem);
  * MaZe constraint sigma = (h/4pi) M phi + q (Eq. Constraints);
  * SHAKE step: phi_p = 2 phi^k - phi^{k-1}, sigma_p = (h/4pi) M phi_p + q^{k+1},
    solve M y = sigma_p (Eq. SHAKEy), phi^{k+1} = phi_p - (4pi/h) y
    (Eq. SHAKEPhiFinal); y starts from the previous step's solution (Sec. II);
  * residual max_n |(M y - sigma_p)_n| (Eq. res_poisson_maze);
  * Jacobi-preconditioned linear CG with J = diag(M) (App. B);
  * multigrid V-cycle: red-black Gauss-Seidel, 27-point full weighting,
    trilinear prolongation, CG on the coarsest grid (Sec. III.A);
  * charge assignment q_n = Q W(r - r_n) with a tensor-product B-spline W,
    central-difference field, force F = -sum_n q_n D phi_n (Eq. F_nostra);
  * V_work = -sum_alpha int F . dr (Eq. E_nostra), discrete energy
    1/2 phi^T q (Eq. energy_discr);
  * Tosi-Fumi pair energy A exp(B(s - r)) - C/r^6 - D/r^8 (Sec. III);
  * velocity Verlet for the ions (Sec. II, Sec. III), or its Langevin
    extension OVRVO (Sec. III) with Philox-4x32-10 Gaussian numbers;
  * the direct Poisson baselines of Sec. III.A (static and time-propagated
    starts) and the force estimator of Eq. F_Benoit.

Readings where the paper is silent (each listed in the design notes):
  * assignment order P in {2, 4}: P=2 is the linear B-spline over the 8
    nearest points, P=4 the cubic B-spline over 4^3 points;
  * Gaussian-unit potential in e/Angstrom; energies and forces are multiplied
    by k_e = e^2/(4 pi eps0) in eV Angstrom;
  * the SHAKE solution y has its mean removed after each solve, and the
    initial potential is the zero-mean solution (the constant mode of the
    periodic M carries no force);
  * step 0: phi^0 solves the constraint from zero, phi^{-1} = phi^0, y = 0;
  * the CG stopping test uses the recursive residual and is confirmed by
    one true residual; a failed confirmation restarts CG from the true one;
  * V_work is integrated with the trapezoid rule on the raw displacement.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# Physical constants (CODATA 2018), derived here independently of the CUDA
# path. Units: Angstrom, fs, amu, e, eV.
_E = 1.602176634e-19            # C
_EPS0 = 8.8541878128e-12        # F/m
_AMU = 1.66053906660e-27        # kg
K_E = _E / (4.0 * math.pi * _EPS0 * 1e-10)     # e^2/(4 pi eps0) in eV*Angstrom
ACC = _E / (_AMU * 1e-10) * 1e10 / 1e30        # 1 eV/(amu*Angstrom) in Angstrom/fs^2
K_B = 1.380649e-23 / _E                        # eV/K


# ---------------------------------------------------------------------------
# Grid operator (Eq. linearproblem and its footnote)

def apply_M(phi: np.ndarray) -> np.ndarray:
    """M phi for the h^2-scaled periodic 7-point Laplacian.

    M_nm = -6 delta_nm + delta_{n,m+-1} + delta_{n,m+-N} + delta_{n,m+-N^2},
    with periodic wrap (footnote to Eq. linearproblem). ``phi`` is [k, j, i].
    """
    out = -6.0 * phi
    for ax in range(3):
        out = out + np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
    return out


def M_eigenvalues(N: int) -> np.ndarray:
    """Eigenvalues of M on the N^3 periodic grid, indexed like the DFT of [k,j,i].

    M is circulant, so the plane wave exp(2 pi i k.n / N) is an eigenvector
    with eigenvalue -6 + 2 cos(2 pi kx/N) + 2 cos(2 pi ky/N) + 2 cos(2 pi kz/N).
    """
    c = 2.0 * np.cos(2.0 * np.pi * np.arange(N) / N)
    return -6.0 + c[:, None, None] + c[None, :, None] + c[None, None, :]


def solve_exact(b: np.ndarray) -> np.ndarray:
    """Zero-mean solution of M y = b by diagonalising M with the 3-D DFT.

    The k = 0 mode (null space of the periodic M) is set to zero, i.e. this
    is the pseudo-inverse M^+ b. Used as the exact discrete reference.
    """
    N = b.shape[0]
    lam = M_eigenvalues(N)
    bh = np.fft.fftn(b)
    lam[0, 0, 0] = 1.0
    yh = bh / lam
    yh[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(yh))


def inf_norm(v: np.ndarray) -> float:
    return float(np.max(np.abs(v))) if v.size else 0.0


# ---------------------------------------------------------------------------
# Charge assignment (Sec. II.A: q_n = Q_alpha W(r_alpha - r_n))

def bspline(d, P: int):
    """Centered cardinal B-spline of P points per axis, at signed distance d
    (in grid units). P=2: linear hat; P=4: cubic B-spline."""
    a = np.abs(np.asarray(d, dtype=np.float64))
    if P == 2:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if P == 4:
        inner = 2.0 / 3.0 - a * a + 0.5 * a ** 3
        outer = (2.0 - a) ** 3 / 6.0
        return np.where(a < 1.0, inner, np.where(a < 2.0, outer, 0.0))
    raise ValueError("assignment order P must be 2 or 4")


def bspline_deriv(d, P: int):
    """dW/dd of :func:`bspline` (used only by the F-tilde estimator, Eq. F_Benoit)."""
    d = np.asarray(d, dtype=np.float64)
    a = np.abs(d)
    s = np.sign(d)
    if P == 2:
        return np.where(a < 1.0, -s, 0.0)
    if P == 4:
        inner = -2.0 * a + 1.5 * a * a
        outer = -0.5 * (2.0 - a) ** 2
        return s * np.where(a < 1.0, inner, np.where(a < 2.0, outer, 0.0))
    raise ValueError("assignment order P must be 2 or 4")


def support(pos: np.ndarray, L: float, N: int, P: int):
    """For each ion and axis: the P grid nodes whose weight can be non-zero and
    the signed distances (in grid units) from the ion to them.

    Returns nodes (N_p, 3, P) int (wrapped into [0, N)) and dist (N_p, 3, P).
    """
    h = L / N
    u = pos / h                                   # position in grid units
    first = np.floor(u).astype(np.int64) - (P // 2 - 1)
    m = first[:, :, None] + np.arange(P)[None, None, :]
    dist = u[:, :, None] - m
    return np.mod(m, N), dist


def assignment(pos, L, N, P):
    """Flat node indices (N_p, P^3) and weights W(r_alpha - r_n) (N_p, P^3)."""
    nodes, dist = support(pos, L, N, P)
    w = bspline(dist, P)                          # (N_p, 3, P)
    # tensor product over (z, y, x) so that the flat order is n = i + jN + kN^2
    ix, iy, iz = nodes[:, 0], nodes[:, 1], nodes[:, 2]
    flat = (iz[:, :, None, None] * N * N + iy[:, None, :, None] * N + ix[:, None, None, :])
    W = w[:, 2][:, :, None, None] * w[:, 1][:, None, :, None] * w[:, 0][:, None, None, :]
    n_p = pos.shape[0]
    return flat.reshape(n_p, -1), W.reshape(n_p, -1)


def spread(pos, Q, L, N, P):
    """q_n = sum_alpha Q_alpha W(r_alpha - r_n) on the [k, j, i] grid (Sec. II.A)."""
    flat, W = assignment(pos, L, N, P)
    q = np.zeros(N ** 3)
    np.add.at(q, flat.ravel(), (Q[:, None] * W).ravel())
    return q.reshape(N, N, N)


def central_difference(phi: np.ndarray, h: float):
    """(D_x phi, D_y phi, D_z phi), D_x phi_n = (phi_{n+1} - phi_{n-1}) / 2h."""
    axes = (2, 1, 0)  # x is the fastest index
    return [(np.roll(phi, -1, axis=a) - np.roll(phi, 1, axis=a)) / (2.0 * h) for a in axes]


def gather_forces(pos, Q, phi, L, N, P):
    """Electrostatic force F_alpha = -k_e sum_n q_n D phi_n with q_n = Q_alpha W
    over the support of ion alpha (Eq. F_nostra). eV/Angstrom, (N_p, 3)."""
    h = L / N
    flat, W = assignment(pos, L, N, P)
    F = np.empty((pos.shape[0], 3))
    for c, D in enumerate(central_difference(phi, h)):
        F[:, c] = -K_E * Q * (W * D.ravel()[flat]).sum(axis=1)
    return F


def gather_forces_tilde(pos, Q, phi, L, N, P):
    """The alternative estimator F~ = -sum_n Q grad_r W(r - r_n) phi_n
    (Eq. F_Benoit), eV/Angstrom. Not momentum-conserving."""
    h = L / N
    nodes, dist = support(pos, L, N, P)
    w = bspline(dist, P)
    dw = bspline_deriv(dist, P) / h
    phif = phi.ravel()
    ix, iy, iz = nodes[:, 0], nodes[:, 1], nodes[:, 2]
    flat = (iz[:, :, None, None] * N * N + iy[:, None, :, None] * N + ix[:, None, None, :])
    vals = phif[flat.reshape(pos.shape[0], -1)].reshape(flat.shape)
    gx = w[:, 2][:, :, None, None] * w[:, 1][:, None, :, None] * dw[:, 0][:, None, None, :]
    gy = w[:, 2][:, :, None, None] * dw[:, 1][:, None, :, None] * w[:, 0][:, None, None, :]
    gz = dw[:, 2][:, :, None, None] * w[:, 1][:, None, :, None] * w[:, 0][:, None, None, :]
    F = np.empty((pos.shape[0], 3))
    for c, g in enumerate((gx, gy, gz)):
        F[:, c] = -K_E * Q * (g * vals).reshape(pos.shape[0], -1).sum(axis=1)
    return F


def discrete_energy(q, phi):
    """V~_c = 1/2 phi^T q (Eq. energy_discr), in eV."""
    return 0.5 * K_E * float(np.sum(q * phi))


# ---------------------------------------------------------------------------
# Linear solvers for M y = b (Eq. SHAKEy)

@dataclasses.dataclass
class SolveInfo:
    iters: int
    resid: float
    converged: bool


def plcg(b, y0, tol, max_iter=10000):
    """Jacobi-preconditioned linear conjugate gradient on M y = b (App. B).

    Preconditioner J_mn = M_mn delta_mn = -6 delta_mn. Stops when the
    recursive residual's infinity norm is below ``tol``; the stop is then
    confirmed with the true residual b - M y, and CG restarts from the true
    residual if the confirmation fails.
    """
    y = y0.copy()
    r = b - apply_M(y)
    it = 0
    res = inf_norm(r)
    if res < tol:
        return y, SolveInfo(0, res, True)
    z = r / -6.0
    p = z.copy()
    rho = float(np.sum(r * z))
    while it < max_iter:
        Mp = apply_M(p)
        alpha = rho / float(np.sum(p * Mp))
        y += alpha * p
        r -= alpha * Mp
        it += 1
        res = inf_norm(r)
        if res < tol:
            r = b - apply_M(y)
            res = inf_norm(r)
            if res < tol:
                return y, SolveInfo(it, res, True)
            z = r / -6.0
            p = z.copy()
            rho = float(np.sum(r * z))
            continue
        z = r / -6.0
        rho_new = float(np.sum(r * z))
        p = z + (rho_new / rho) * p
        rho = rho_new
    return y, SolveInfo(it, inf_norm(b - apply_M(y)), False)


# --- multigrid (Sec. III.A) --------------------------------------------------

def mg_levels(N: int):
    """Grid sizes of the hierarchy: halve while the size is even and above 8
    (an 8^3 grid once, so that there are at least two levels); the coarsest
    level, of at most 8^3 points, is solved exactly. Sec. III.A leaves the
    depth of the hierarchy open."""
    sizes = [N]
    while sizes[-1] % 2 == 0 and (sizes[-1] > 8 or (sizes[-1] == 8 and len(sizes) == 1)):
        sizes.append(sizes[-1] // 2)
    return sizes


def red_mask(N: int) -> np.ndarray:
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return (i + j + k) % 2 == 0


def rbgs_sweep(x, b):
    """One red-black Gauss-Seidel sweep on M x = b: every red point (i+j+k even),
    then every black point, is set to x_n = (sum of its 6 neighbours - b_n) / 6."""
    red = red_mask(x.shape[0])
    for colour in (red, ~red):
        nb = apply_M(x) + 6.0 * x          # sum of the six neighbours
        x = np.where(colour, (nb - b) / 6.0, x)
    return x


def restrict_fw(r):
    """27-point full weighting: coarse point I (fine point 2I) gets the
    tensor-product weights (1/4, 1/2, 1/4) per axis over the 3^3 fine
    neighbourhood."""
    out = r
    for ax in range(3):
        out = 0.25 * np.roll(out, 1, axis=ax) + 0.5 * out + 0.25 * np.roll(out, -1, axis=ax)
    return out[::2, ::2, ::2].copy()


def prolong_trilinear(e):
    """Trilinear interpolation of a coarse-grid correction onto the fine grid:
    even fine indices copy the coarse value, odd ones average the two coarse
    neighbours, per axis (periodic)."""
    out = e
    for ax in range(3):
        n = out.shape[ax]
        shape = list(out.shape)
        shape[ax] = 2 * n
        fine = np.empty(shape)
        sl_even = [slice(None)] * 3
        sl_odd = [slice(None)] * 3
        sl_even[ax] = slice(0, None, 2)
        sl_odd[ax] = slice(1, None, 2)
        fine[tuple(sl_even)] = out
        fine[tuple(sl_odd)] = 0.5 * (out + np.roll(out, -1, axis=ax))
        out = fine
    return out


def coarse_cg(b, tol):
    """'Exact' coarsest-grid solve: plain CG on the mean-projected system from
    zero, to max(1e-3 tol, 1e-14 |b|_inf) in the infinity norm (the paper uses
    CG as the exact coarsest solver; its tolerance is not stated)."""
    b = b - b.mean()
    target = max(1e-3 * tol, 1e-14 * inf_norm(b))
    y, _ = plcg(b, np.zeros_like(b), target, max_iter=500)
    return y - y.mean()


def vcycle(x, b, tol, nu1=2, nu2=2, levels=None):
    """One V-cycle for M x = b on the hierarchy ``levels`` (default
    ``mg_levels`` of the grid), finest first."""
    if levels is None:
        levels = mg_levels(x.shape[0])
    if len(levels) == 1:
        return coarse_cg(b, tol)
    for _ in range(nu1):
        x = rbgs_sweep(x, b)
    r = b - apply_M(x)
    bc = 4.0 * restrict_fw(r)        # M is h^2-scaled: coarse rhs picks up (2h/h)^2
    ec = vcycle(np.zeros_like(bc), bc, tol, nu1, nu2, levels[1:])
    x = x + prolong_trilinear(ec)
    for _ in range(nu2):
        x = rbgs_sweep(x, b)
    return x


def mg_solve(b, y0, tol, max_iter=200, nu1=2, nu2=2):
    """V-cycles from y0 until max|M y - b| < tol, residual checked after each."""
    y = y0.copy()
    res = inf_norm(b - apply_M(y))
    it = 0
    while res >= tol and it < max_iter:
        y = vcycle(y, b, tol, nu1, nu2)
        it += 1
        res = inf_norm(b - apply_M(y))
    return y, SolveInfo(it, res, res < tol)


def solve(b, y0, tol, solver="cg", max_iter=10000):
    if solver == "cg":
        return plcg(b, y0, tol, max_iter)
    if solver == "mg":
        return mg_solve(b, y0, tol, min(max_iter, 200))
    raise ValueError(solver)


# ---------------------------------------------------------------------------
# Tosi-Fumi short-range pairs (Sec. III)

def _tf_pair(r, k, tf):
    """Energy and -dV/dr for pair kind(s) k at distance(s) r."""
    A = np.asarray(tf.A)[k]
    s = np.asarray(tf.s)[k]
    C = np.asarray(tf.C)[k]
    D = np.asarray(tf.D)[k]
    ex = A * np.exp(tf.B * (s - r))
    V = ex - C / r ** 6 - D / r ** 8
    f = tf.B * ex - 6.0 * C / r ** 7 - 8.0 * D / r ** 9     # -dV/dr
    return V, f


def tf_forces(pos, types, L, tf, rc):
    """All-pairs minimum-image Tosi-Fumi forces and energy within r_c.

    Energy is shifted by V(r_c) per pair so that it is continuous at the
    cutoff; forces are plainly truncated. Returns (F (N_p,3), V_TF).
    """
    n = pos.shape[0]
    F = np.zeros((n, 3))
    V = 0.0
    for a in range(n - 1):
        d = pos[a + 1:] - pos[a]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        k = types[a] + types[a + 1:]
        m = r < rc
        if not m.any():
            continue
        Vp, f = _tf_pair(r[m], k[m], tf)
        Vc, _ = _tf_pair(np.full(m.sum(), rc), k[m], tf)
        V += float((Vp - Vc).sum())
        fvec = (f / r[m])[:, None] * d[m]      # force on the partner b
        F[a + 1:][m] += fvec
        F[a] -= fvec.sum(axis=0)
    return F, V


def tf_forces_cells(pos, types, L, tf, rc, chunk=2048):
    """The same sum as :func:`tf_forces`, with the candidate pairs taken from
    a cell list instead of all pairs (needed for boxes of ~10^5 ions and more).

    The box is cut into n_c = floor(L / r_c) >= 3 cells per edge, so a cell
    is at least r_c wide and every pair closer than r_c (minimum image, r_c <=
    L/2) lies in the same or in adjacent cells. Each unordered pair of ions is
    visited once: ion pairs a < b within a cell, and all ion pairs between a
    cell and the 13 neighbours of its "upper" half shell (offsets (dz, dy, dx)
    after (0, 0, 0) in lexicographic order). With n_c >= 3 the 27 neighbour
    cells of a cell are distinct, so no cell pair is visited twice. Returns
    (F (N_p, 3), V_TF)."""
    n = pos.shape[0]
    nc = int(math.floor(L / rc))
    if nc < 3:
        return tf_forces(pos, types, L, tf, rc)
    side = L / nc
    c3 = np.minimum((np.floor(pos / side)).astype(np.int64), nc - 1)     # (n, 3) cell coordinates
    cid = (c3[:, 2] * nc + c3[:, 1]) * nc + c3[:, 0]
    order = np.argsort(cid, kind="stable")
    counts = np.bincount(cid, minlength=nc ** 3)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    mo = int(counts.max())
    table = np.full((nc ** 3, mo), -1, dtype=np.int64)    # ions of each cell, padded with -1
    slot = np.arange(n) - starts[cid[order]]
    table[cid[order], slot] = order
    cz, cy, cx = np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij")
    cz, cy, cx = cz.ravel(), cy.ravel(), cx.ravel()        # cell id = (cz nc + cy) nc + cx
    offsets = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
               if (dz, dy, dx) > (0, 0, 0)]
    F = np.zeros((n, 3))
    V = 0.0
    for off in [(0, 0, 0)] + offsets:
        dz, dy, dx = off
        nb = ((((cz + dz) % nc) * nc + (cy + dy) % nc) * nc + (cx + dx) % nc)
        for c0 in range(0, nc ** 3, chunk):
            A = table[c0:c0 + chunk]                    # (c, mo) ions of the cells
            B = table[nb[c0:c0 + chunk]]                # (c, mo) ions of their neighbour cells
            a = np.broadcast_to(A[:, :, None], (A.shape[0], mo, mo)).ravel()
            b = np.broadcast_to(B[:, None, :], (A.shape[0], mo, mo)).ravel()
            keep = (a >= 0) & (b >= 0)
            if off == (0, 0, 0):
                keep &= a < b
            a, b = a[keep], b[keep]
            d = pos[b] - pos[a]
            d -= L * np.round(d / L)
            r = np.sqrt((d * d).sum(axis=1))
            m = r < rc
            a, b, d, r = a[m], b[m], d[m], r[m]
            k = types[a] + types[b]
            Vp, f = _tf_pair(r, k, tf)
            Vc, _ = _tf_pair(np.full(r.shape, rc), k, tf)
            V += float((Vp - Vc).sum())
            fvec = (f / r)[:, None] * d                 # force on b
            for ax in range(3):
                F[:, ax] += np.bincount(b, weights=fvec[:, ax], minlength=n)
                F[:, ax] -= np.bincount(a, weights=fvec[:, ax], minlength=n)
    return F, V


def pair_forces(pos, types, L, tf, rc):
    """Tosi-Fumi forces and energy: all pairs for small boxes, the cell-list
    sum above 4096 ions (identical up to summation order)."""
    if pos.shape[0] > 4096 and math.floor(L / rc) >= 3:
        return tf_forces_cells(pos, types, L, tf, rc)
    return tf_forces(pos, types, L, tf, rc)


def tf_forces_on(idx, pos, types, L, tf, rc):
    """Tosi-Fumi force on the selected ions only, by brute force over all others."""
    out = np.zeros((len(idx), 3))
    for o, a in enumerate(idx):
        d = pos - pos[a]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        m = (r < rc) & (np.arange(pos.shape[0]) != a)
        _, f = _tf_pair(r[m], types[a] + types[m], tf)
        out[o] = -((f / r[m])[:, None] * d[m]).sum(axis=0)
    return out


# ---------------------------------------------------------------------------
# The MaZe MD step (Sec. II, Fig. algorithm; Sec. III velocity Verlet)

@dataclasses.dataclass
class Params:
    L: float
    N: int
    dt: float
    tol: float
    charge: tuple = (1.0, -1.0)
    mass: tuple = (22.98977, 35.453)
    P: int = 4
    rc: float = 9.0
    solver: str = "cg"
    max_iter: int = 10000
    # "maze" (SHAKE, Eqs. SHAKE-SHAKEPhiFinal), or a direct solve of
    # Eq. linearproblem from the previous potential ("mg-static") or from
    # 2 phi^k - phi^{k-1} ("mg-timeprop"), Sec. III.A
    scheme: str = "maze"
    # electrostatic force: "cd" (Eq. F_nostra) or "gradw" (Eq. F_Benoit)
    force: str = "cd"
    # OVRVO Langevin integrator (Sec. III): friction (1/fs), bath temperature
    # (K), generator key; gamma = 0 is velocity Verlet
    gamma: float = 0.0
    T_bath: float = 0.0
    seed: int = 0

    @property
    def h(self):
        return self.L / self.N


@dataclasses.dataclass
class State:
    pos: np.ndarray
    vel: np.ndarray
    types: np.ndarray
    phi: np.ndarray          # phi^k
    phi_prev: np.ndarray     # phi^{k-1}
    y: np.ndarray            # last SHAKE solution (warm start)
    F_el: np.ndarray
    F_tf: np.ndarray
    V_tf: float
    V_work: float = 0.0
    V_disc: float = 0.0
    step: int = 0
    iters: int = 0
    resid: float = 0.0

    @property
    def F(self):
        return self.F_el + self.F_tf


def _charges(types, p: Params):
    return np.asarray(p.charge)[types]


def _masses(types, p: Params):
    return np.asarray(p.mass)[types]


def wrap(pos, L):
    out = pos - L * np.floor(pos / L)
    out[out >= L] -= L
    return out


def init(pos, vel, types, p: Params, tf) -> State:
    """Step 0: phi^0 solves the constraint from zero (zero-mean solution),
    phi^{-1} = phi^0, y = 0, then the forces F^0."""
    N = p.N
    Q = _charges(types, p)
    pos = wrap(np.asarray(pos, dtype=np.float64), p.L)
    q = spread(pos, Q, p.L, N, p.P)
    y0, info = solve(q, np.zeros_like(q), p.tol, p.solver, p.max_iter)   # sigma_p = q at phi_p = 0
    phi = -(4.0 * np.pi / p.h) * (y0 - y0.mean())
    F_el = electrostatic_forces(pos, Q, phi, p)
    F_tf, V_tf = pair_forces(pos, types, p.L, tf, p.rc)
    st = State(pos=pos, vel=np.array(vel, dtype=np.float64), types=np.asarray(types),
               phi=phi, phi_prev=phi.copy(), y=np.zeros_like(phi),
               F_el=F_el, F_tf=F_tf, V_tf=V_tf, iters=info.iters, resid=info.resid)
    st.V_disc = discrete_energy(q, phi)
    return st


def sigma_p(phi, phi_prev, q, h):
    """phi_p = 2 phi^k - phi^{k-1} and sigma_p = (h/4pi) M phi_p + q (Eq. SHAKE)."""
    phi_p = 2.0 * phi - phi_prev
    return phi_p, (h / (4.0 * np.pi)) * apply_M(phi_p) + q


def step(st: State, p: Params, tf) -> State:
    """One MaZe MD step k -> k+1 (velocity Verlet for ions, SHAKE for phi)."""
    Q = _charges(st.types, p)
    m = _masses(st.types, p)[:, None]
    F_el_old = st.F_el
    vel0 = o_step(st.vel, st.types, p, st.step, 0) if p.gamma > 0 else st.vel
    v_half = vel0 + (0.5 * p.dt * ACC) * st.F / m
    dr = p.dt * v_half
    pos = wrap(st.pos + dr, p.L)
    q = spread(pos, Q, p.L, p.N, p.P)
    if p.scheme == "maze":
        phi_p, sp = sigma_p(st.phi, st.phi_prev, q, p.h)
        y, info = solve(sp, st.y, p.tol, p.solver, p.max_iter)
        y = y - y.mean()
        phi_new = phi_p - (4.0 * np.pi / p.h) * y
    else:
        phi_new, y, info = direct_solve(st, q, p)
    F_el = electrostatic_forces(pos, Q, phi_new, p)
    F_tf, V_tf = pair_forces(pos, st.types, p.L, tf, p.rc)
    vel = v_half + (0.5 * p.dt * ACC) * (F_el + F_tf) / m
    if p.gamma > 0:
        vel = o_step(vel, st.types, p, st.step, 1)
    V_work = st.V_work - 0.5 * float(np.sum((F_el_old + F_el) * dr))
    return State(pos=pos, vel=vel, types=st.types, phi=phi_new, phi_prev=st.phi, y=y,
                 F_el=F_el, F_tf=F_tf, V_tf=V_tf, V_work=V_work,
                 V_disc=discrete_energy(q, phi_new), step=st.step + 1,
                 iters=info.iters, resid=info.resid)


# ---------------------------------------------------------------------------
# Counter-based random numbers for the O steps: Philox-4x32-10 (Salmon,
# Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011),
# written from its published definition, and the Box-Muller transform.

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_U32 = 0xFFFFFFFF


def philox4x32(ctr, key, rounds=10):
    """Philox-4x32 on arrays of counters: ``ctr`` is a tuple of four uint64
    arrays (values < 2^32), ``key`` a pair of ints. Each round multiplies
    words 0 and 2 by the Philox constants, splits the 64-bit products into
    high and low halves and mixes them with words 1 and 3 and the round key;
    the key advances by the Weyl constants between rounds."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _U32 for c in ctr)
    k0, k1 = np.uint64(key[0] & _U32), np.uint64(key[1] & _U32)
    for r in range(rounds):
        if r:
            k0 = np.uint64((int(k0) + _PHILOX_W0) & _U32)
            k1 = np.uint64((int(k1) + _PHILOX_W1) & _U32)
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_U32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_U32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def gaussians(n_ions: int, step: int, stage: int, seed: int):
    """Three standard normals per ion for one O step: Philox-4x32-10 with
    counter (ion, step, stage, 0) and key (seed low, seed high); uniforms
    u = (x + 1/2) 2^-32 and the Box-Muller transform
    (sqrt(-2 ln u0) cos 2 pi u1, sqrt(-2 ln u0) sin 2 pi u1, sqrt(-2 ln u2) cos 2 pi u3)."""
    i = np.arange(n_ions, dtype=np.uint64)
    z = np.zeros(n_ions, dtype=np.uint64)
    x = philox4x32((i, z + np.uint64(step & _U32), z + np.uint64(stage), z), (seed & _U32, (seed >> 32) & _U32))
    u = [(xk.astype(np.float64) + 0.5) * 2.0 ** -32 for xk in x]
    r01 = np.sqrt(-2.0 * np.log(u[0]))
    r23 = np.sqrt(-2.0 * np.log(u[2]))
    return np.stack([r01 * np.cos(2 * np.pi * u[1]), r01 * np.sin(2 * np.pi * u[1]),
                     r23 * np.cos(2 * np.pi * u[3])], axis=1)


def o_step(vel, types, p: Params, step: int, stage: int):
    """O part of OVRVO (Sivak, Chodera, Crooks 2013) over a half step:
    v <- a v + sqrt((1 - a^2) k_B T / m) xi, a = exp(-gamma dt / 2)."""
    a = math.exp(-p.gamma * p.dt / 2.0)
    m = _masses(types, p)[:, None]
    sd = np.sqrt((1.0 - a * a) * K_B * p.T_bath * ACC / m)
    return a * vel + sd * gaussians(vel.shape[0], step, stage, p.seed)


def direct_solve(st: State, q, p: Params):
    """The direct Poisson baselines of Sec. III.A: solve M phi = -(4 pi/h) q
    (Eq. linearproblem) with the same solver, stopping on
    max_n |(M phi + (4 pi/h) q)_n| < tol (Eq. res_poisson), from the converged
    potential of the previous step ("mg-static") or from the putative
    2 phi^k - phi^{k-1} ("mg-timeprop"). The zero-mean solution is kept; y is
    not used by these schemes (returned as zeros)."""
    if p.scheme == "mg-static":
        phi0 = st.phi
    elif p.scheme == "mg-timeprop":
        phi0 = 2.0 * st.phi - st.phi_prev
    else:
        raise ValueError(p.scheme)
    phi, info = solve(-(4.0 * np.pi / p.h) * q, phi0, p.tol, p.solver, p.max_iter)
    return phi - phi.mean(), np.zeros_like(phi), info


def electrostatic_forces(pos, Q, phi, p: Params):
    if p.force == "cd":
        return gather_forces(pos, Q, phi, p.L, p.N, p.P)
    if p.force == "gradw":
        return gather_forces_tilde(pos, Q, phi, p.L, p.N, p.P)
    raise ValueError(p.force)


def kinetic(st: State, p: Params) -> float:
    m = _masses(st.types, p)[:, None]
    return 0.5 * float(np.sum(m * st.vel * st.vel)) / ACC


def momentum(st: State, p: Params) -> np.ndarray:
    m = _masses(st.types, p)[:, None]
    return (m * st.vel).sum(axis=0)


def energies(st: State, p: Params) -> dict:
    ke = kinetic(st, p)
    return dict(ke=ke, v_tf=st.V_tf, v_work=st.V_work, v_disc=st.V_disc,
                e_tot=ke + st.V_tf + st.V_work)


def exact_potential(pos, types, p: Params):
    """Zero-mean discrete potential of the current positions: the exact solution
    of M phi = -4 pi q / h (Eq. linearproblem) via the DFT."""
    q = spread(wrap(pos, p.L), _charges(types, p), p.L, p.N, p.P)
    return -(4.0 * np.pi / p.h) * solve_exact(q), q


def run(pos, vel, types, p: Params, tf, nsteps: int, record=None):
    st = init(pos, vel, types, p, tf)
    if record is not None:
        record.append(st)
    for _ in range(nsteps):
        st = step(st, p, tf)
        if record is not None:
            record.append(st)
    return st
