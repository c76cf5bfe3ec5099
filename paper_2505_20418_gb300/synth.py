"""Seeded synthetic inputs for molten-NaCl Poisson MaZe runs.

This module is the ONLY code shared by the CUDA path and the CPU oracle. It
holds no arithmetic of the method itself (no charge assignment, no Laplacian,
no solver, no force): it only draws the initial ionic configuration that both
sides receive as input, and it carries the molten-salt parameter table that
both sides receive as input.

Workload recipe (stands in for the paper's molten-NaCl box, Sec. III):
  * positions: rock-salt arrangement on an n^3 simple-cubic lattice of spacing
    d = L/n, site (a,b,c) at (a d, b d, c d), species Na where a+b+c is even
    and Cl otherwise; Gaussian noise of standard deviation ``sigma`` (Angstrom)
    per coordinate, wrapped into [0, L).
  * velocities: Maxwell-Boltzmann at temperature T for each species' mass,
    centre-of-mass velocity removed, rescaled so that the kinetic temperature
    with 3 N_p - 3 degrees of freedom is exactly T.
  * generator: numpy PCG64 seeded with ``seed``.

Units: Angstrom, fs, amu, elementary charge e, eV.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Conversion constants for input preparation only (temperature -> velocity).
# 1 eV / (amu * Angstrom) expressed in Angstrom / fs^2, and Boltzmann's
# constant in eV / K (CODATA 2018 exact/defined values).
_EV_PER_AMU_A2_FS2 = 1.602176634e-19 / (1.66053906660e-27 * 1e-10) * 1e10 / 1e30
_KB_EV = 1.380649e-23 / 1.602176634e-19

MASS_NA = 22.98977  # amu
MASS_CL = 35.453    # amu


@dataclasses.dataclass(frozen=True)
class TosiFumi:
    """Born-Mayer-Huggins parameters for the three pair kinds.

    Index 0 = Na-Na, 1 = Na-Cl, 2 = Cl-Cl. The pair energy is
    A exp(B (s - r)) - C / r^6 - D / r^8 (Sec. III, Tosi-Fumi form).
    A in eV, B in 1/Angstrom, s in Angstrom, C in eV Angstrom^6, D in eV
    Angstrom^8. Values: the Tosi-Fumi NaCl set (b = 0.338e-19 J, rho = 0.317
    Angstrom, sigma_Na = 1.170, sigma_Cl = 1.585 Angstrom, Pauling factors
    1.25 / 1.00 / 0.75, dispersion C = 1.68 / 11.2 / 116 x 1e-79 J m^6 and
    D = 0.8 / 13.9 / 233 x 1e-99 J m^8), converted to eV and Angstrom. The
    paper only cites this set; both the oracle and the CUDA path receive the
    same table as input, so parity does not depend on the values.
    """

    A: tuple
    B: float
    s: tuple
    C: tuple
    D: tuple


def tosi_fumi_nacl() -> TosiFumi:
    j_to_ev = 1.0 / 1.602176634e-19
    b = 0.338e-19 * j_to_ev
    rho = 0.317
    sig_na, sig_cl = 1.170, 1.585
    pauling = (1.25, 1.00, 0.75)
    c6 = tuple(v * 1e-79 * j_to_ev * 1e60 for v in (1.68, 11.2, 116.0))
    c8 = tuple(v * 1e-99 * j_to_ev * 1e80 for v in (0.8, 13.9, 233.0))
    s = (2 * sig_na, sig_na + sig_cl, 2 * sig_cl)
    return TosiFumi(A=tuple(c * b for c in pauling), B=1.0 / rho, s=s, C=c6, D=c8)


@dataclasses.dataclass
class Workload:
    """One molten-NaCl box: everything both sides need as input."""

    name: str
    n_side: int          # ions per lattice edge; N_p = n_side^3
    L: float             # cubic box edge, Angstrom
    N: int               # grid points per edge
    dt: float = 1.0      # fs
    tol: float = 1e-10   # constraint tolerance (infinity norm, units of e)
    T: float = 1200.0    # K
    sigma: float = 0.1   # lattice noise, Angstrom
    order: int = 4       # assignment order P (points per axis): 2 or 4
    r_cut: float | None = None
    seed: int = 0
    steps: int = 100

    @property
    def n_ions(self) -> int:
        return self.n_side ** 3

    @property
    def rc(self) -> float:
        return self.r_cut if self.r_cut is not None else min(self.L / 2, 9.0)


def rocksalt(n_side: int, L: float, sigma: float, rng: np.random.Generator):
    """Lattice + Gaussian noise. Returns pos (N_p,3) float64 and type (N_p,) int32."""
    if n_side % 2:
        raise ValueError("n_side must be even for a neutral rock-salt box")
    d = L / n_side
    a = np.arange(n_side)
    cz, cy, cx = np.meshgrid(a, a, a, indexing="ij")
    sites = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    types = ((sites.sum(axis=1).astype(np.int64)) % 2).astype(np.int32)
    pos = sites * d
    if sigma > 0:
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    pos = pos - L * np.floor(pos / L)
    pos[pos >= L] -= L  # guard the rounding edge of the wrap
    return np.ascontiguousarray(pos), types


def maxwell(types: np.ndarray, T: float, rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities (Angstrom/fs), COM removed, exactly at T."""
    m = np.where(types == 0, MASS_NA, MASS_CL)[:, None]
    if T <= 0:
        return np.zeros((types.size, 3))
    sd = np.sqrt(_KB_EV * T * _EV_PER_AMU_A2_FS2 / m)
    v = rng.normal(size=(types.size, 3)) * sd
    v -= (m * v).sum(axis=0) / m.sum()
    ke = 0.5 * (m * v * v).sum() / _EV_PER_AMU_A2_FS2
    dof = 3 * types.size - 3
    t_now = 2 * ke / (dof * _KB_EV)
    v *= math.sqrt(T / t_now)
    return np.ascontiguousarray(v)


def make_state(w: Workload):
    """(pos, vel, type) for a workload, drawn from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    pos, types = rocksalt(w.n_side, w.L, w.sigma, rng)
    vel = maxwell(types, w.T, rng)
    return pos, vel, types


def random_neutral(n_ions: int, L: float, seed: int, min_dist: float = 0.0):
    """Uniform random positions with alternating types (for tiny pin boxes).

    With ``min_dist`` > 0 positions are redrawn until every minimum-image pair
    distance is at least ``min_dist`` (rejection sampling, small n only).
    """
    if n_ions % 2:
        raise ValueError("need an even ion count for neutrality")
    rng = np.random.Generator(np.random.PCG64(seed))
    types = (np.arange(n_ions) % 2).astype(np.int32)
    for _ in range(10000):
        pos = rng.uniform(0.0, L, size=(n_ions, 3))
        if min_dist <= 0:
            return pos, types
        d = pos[:, None, :] - pos[None, :, :]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(-1)) + np.eye(n_ions) * 1e9
        if r.min() >= min_dist:
            return pos, types
    raise RuntimeError("rejection sampling failed")


# Named workloads: molten NaCl at 0.032 ions / Angstrom^3, 1200 K, dt = 1 fs.
def workload(name: str) -> Workload:
    if name == "nacl64":      # 64 ions, 16^3 grid, 100 steps, FP64 tol 1e-10
        return Workload("nacl64_L12.6_N16", 4, 12.6, 16, steps=100, seed=1000, r_cut=6.3)
    if name == "nacl1000":    # 1000 ions, 32^3 grid, 1000 steps
        return Workload("nacl1000_L31.5_N32", 10, 31.5, 32, steps=1000, seed=2000)
    if name == "nacl64000":   # 64000 ions, 128^3 grid (a profiling-size large box)
        return Workload("nacl64000_L126_N128", 40, 126.0, 128, steps=200, seed=4100)
    if name == "nacl8000":    # 8000 ions, 64^3 grid: 1/64 of the 512000-ion box (same density, spacing, T)
        return Workload("nacl8000_L63_N64", 20, 63.0, 64, steps=200, seed=4200)
    if name == "nacl512000":  # 512000 ions, 256^3 grid, 200 steps
        return Workload("nacl512000_L252_N256", 80, 252.0, 256, steps=200, seed=4000)
    raise KeyError(name)


# Replica sizes for batched / served boxes: (n_side, L, N) at ~1 Angstrom grid spacing.
REPLICA_SIZES = {
    216: (6, 18.9, 16),
    512: (8, 25.2, 24),
    1000: (10, 31.5, 32),
    1728: (12, 37.8, 40),
    4096: (16, 50.4, 48),
    13824: (24, 75.6, 64),
}


def replica(n_ions: int, seed: int, **kw) -> Workload:
    """One replica box of a standard size (see REPLICA_SIZES)."""
    n_side, L, N = REPLICA_SIZES[n_ions]
    return Workload(f"nacl{n_ions}_L{L}_N{N}", n_side, L, N, seed=seed, **kw)


BATCH_SIZES = (216, 512, 1000, 1728, 4096)


def batch_workloads(n_boxes: int, seed: int = 3000, sizes=BATCH_SIZES, **kw) -> list:
    """Replica boxes with ion counts drawn uniformly from ``sizes`` by
    PCG64(seed); replica r has its own seed, seed + 1 + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.choice(np.asarray(sizes), size=n_boxes)
    return [replica(int(n), seed + 1 + r, **kw) for r, n in enumerate(counts)]
