"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module makes inputs only.  It holds none of the method's arithmetic
(no spline, no density or force sum, no lattice-list logic): it tabulates the
analytic potential into knot values, lays atoms on a bcc crystal, draws
velocities and displacements, and picks knock-on energies and directions.
Both the CUDA library and the oracle receive what it returns; neither
imports the other.

Workload recipe (the shapes the paper's cascade runs have, Sec. 5.1):
  * bcc iron-like crystal, lattice constant a0 = 2.855 A, periodic box of
    nx x ny x nz cubic cells, 2 atoms per cell;
  * Finnis-Sinclair-form potential: f(r) = exp(-3 (r/2.47 - 1)),
    phi(r) = 0.4 [exp(-3.2 (r - 2.6)) - 2 exp(-1.6 (r - 2.6))] (a Morse pair
    term), F(rho) = -1.8 sqrt(rho); f and phi smoothly truncated at
    rc = 5.6 A (shifted-force form), tabulated on 5000 equidistant knots;
  * Maxwell velocities at temperature T (Philox counter-based normals),
    centre-of-mass motion removed, rescaled so that the kinetic energy is
    exactly 3/2 N kB T;
  * a primary knock-on atom (PKA) with energy E along a seeded direction;
  * for parity snapshots: Gaussian thermal displacements, plus "cascade"
    defects (interstitials dropped at random points, which leave vacancies
    and create run-away atoms, and close pairs down to ~1 A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Physical constants (CODATA 2018) used to turn temperatures and energies
# into velocities in Angstrom/fs for amu masses.
KB_EV = 8.617333262e-5  # eV/K
EV_PER_AMU_A2_FS2 = 1.0 / 9.6485332123310018e-3  # 1 amu A^2/fs^2 in eV

A0_FE = 2.855
MASS_FE = 55.845
RC = 5.6
N_KNOTS = 5000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


# ---------------------------------------------------------------------------
# analytic potential -> knot tables
# ---------------------------------------------------------------------------

def f_analytic(r):
    return np.exp(-3.0 * (np.asarray(r, dtype=np.float64) / 2.47 - 1.0))


def df_analytic(r):
    return -3.0 / 2.47 * f_analytic(r)


def phi_analytic(r):
    x = np.asarray(r, dtype=np.float64) - 2.6
    return 0.4 * (np.exp(-3.2 * x) - 2.0 * np.exp(-1.6 * x))


def dphi_analytic(r):
    x = np.asarray(r, dtype=np.float64) - 2.6
    return 0.4 * (-3.2 * np.exp(-3.2 * x) + 3.2 * np.exp(-1.6 * x))


def embed_analytic(rho):
    return -1.8 * np.sqrt(np.asarray(rho, dtype=np.float64))


def truncated(g, dg, rc=RC):
    """Shifted-force truncation: g(r) - g(rc) - (r - rc) g'(rc) below rc, 0 above."""

    def gs(r):
        r = np.asarray(r, dtype=np.float64)
        return np.where(r < rc, g(r) - g(rc) - (r - rc) * dg(rc), 0.0)

    def dgs(r):
        r = np.asarray(r, dtype=np.float64)
        return np.where(r < rc, dg(r) - dg(rc), 0.0)

    return gs, dgs


@dataclass
class Potential:
    n: int
    rc: float
    rho_max: float
    f: np.ndarray      # knots of f on r_k = k rc/(n-1)
    phi: np.ndarray    # knots of phi on the same grid
    F: np.ndarray      # knots of F on rho_k = k rho_max/(n-1)

    def scaled(self, eps_f, eps_phi, eps_F) -> "Potential":
        """Knots multiplied by (1 + eps) elementwise (a perturbed potential)."""
        return Potential(self.n, self.rc, self.rho_max, self.f * (1.0 + eps_f),
                         self.phi * (1.0 + eps_phi), self.F * (1.0 + eps_F))


def equilibrium_density(a0=A0_FE, rc=RC) -> float:
    """Host density of a perfect bcc crystal for the truncated analytic f (the
    sum over the neighbour shells), used to size the embedding table."""
    fs, _ = truncated(f_analytic, df_analytic, rc)
    m = int(math.ceil(2.0 * rc / a0)) + 1
    rho = 0.0
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                if (i % 2 == j % 2 == k % 2) and (i or j or k):
                    d = 0.5 * a0 * math.sqrt(i * i + j * j + k * k)
                    if d < rc:
                        rho += float(fs(d))
    return rho


def potential(n: int = N_KNOTS, rc: float = RC, a0: float = A0_FE) -> Potential:
    """Knot tables of the analytic Finnis-Sinclair/Morse potential; the
    embedding table spans [0, 4 rho_eq]."""
    fs, _ = truncated(f_analytic, df_analytic, rc)
    ps, _ = truncated(phi_analytic, dphi_analytic, rc)
    r = np.arange(n, dtype=np.float64) * (rc / (n - 1))
    rho_max = 4.0 * equilibrium_density(a0, rc)
    rho = np.arange(n, dtype=np.float64) * (rho_max / (n - 1))
    return Potential(n, rc, rho_max, fs(r), ps(r), embed_analytic(rho))


# ---------------------------------------------------------------------------
# alloys: per-species density and embedding functions, pair functions per
# unordered species pair (the paper's Fe-Cu-Ni tables are not available;
# these analytic forms stand in for them)
# ---------------------------------------------------------------------------

# species: density prefactor A and decay b of A exp(-b (r/2.47 - 1)), embedding
# strength c of -c sqrt(rho), Morse depth D and minimum r0 of the pair term;
# species 0 is the single-species potential above
SPECIES = (
    dict(A=1.0, b=3.0, c=1.8, D=0.40, r0=2.60),
    dict(A=0.8, b=3.4, c=1.5, D=0.35, r0=2.65),
    dict(A=1.1, b=3.2, c=1.6, D=0.45, r0=2.55),
    dict(A=0.9, b=2.8, c=1.7, D=0.38, r0=2.62),
)


def pair_index(a: int, b: int, nsp: int) -> int:
    """Row of pair (a, b) in the upper-triangle pair table (a <= b)."""
    a, b = min(a, b), max(a, b)
    return a * nsp - a * (a - 1) // 2 + (b - a)


def alloy_functions(nsp: int):
    """Analytic (untruncated) rho_a, rho_a', F_a, F_a', phi_ab, phi_ab' as callables."""
    sp = SPECIES[:nsp]

    def dens(a):
        A, b = sp[a]["A"], sp[a]["b"]
        g = lambda r: A * np.exp(-b * (np.asarray(r, dtype=np.float64) / 2.47 - 1.0))
        dg = lambda r: -b / 2.47 * g(r)
        return g, dg

    def emb(a):
        c = sp[a]["c"]
        return (lambda rho: -c * np.sqrt(np.asarray(rho, dtype=np.float64)),
                lambda rho: -0.5 * c / np.sqrt(np.asarray(rho, dtype=np.float64)))

    def pair(a, b):
        D = math.sqrt(sp[a]["D"] * sp[b]["D"])
        r0 = 0.5 * (sp[a]["r0"] + sp[b]["r0"])
        g = lambda r: D * (np.exp(-3.2 * (np.asarray(r, dtype=np.float64) - r0))
                           - 2.0 * np.exp(-1.6 * (np.asarray(r, dtype=np.float64) - r0)))
        dg = lambda r: D * (-3.2 * np.exp(-3.2 * (np.asarray(r, dtype=np.float64) - r0))
                            + 3.2 * np.exp(-1.6 * (np.asarray(r, dtype=np.float64) - r0)))
        return g, dg

    return dens, emb, pair


@dataclass
class AlloyPotential:
    nsp: int
    n: int
    rc: float
    rho_max: float
    f: np.ndarray    # (nsp, n): density function of each species on r_k
    F: np.ndarray    # (nsp, n): embedding function of each species on rho_k
    phi: np.ndarray  # (nsp (nsp + 1) / 2, n): pair functions, rows by pair_index

    def species(self, a: int) -> Potential:
        """The single-species potential of species a."""
        return Potential(self.n, self.rc, self.rho_max, self.f[a], self.phi[pair_index(a, a, self.nsp)], self.F[a])


def alloy_potential(nsp: int = 2, n: int = N_KNOTS, rc: float = RC, a0: float = A0_FE) -> AlloyPotential:
    """Knot tables of an nsp-species alloy (shifted-force truncated density
    and pair functions); the embedding tables span [0, 4 max_a rho_eq,a]."""
    if not 1 <= nsp <= len(SPECIES):
        raise ValueError("1 to 4 species")
    dens, emb, pair = alloy_functions(nsp)
    r = np.arange(n, dtype=np.float64) * (rc / (n - 1))
    rho_max = 4.0 * equilibrium_density(a0, rc) * max(s["A"] for s in SPECIES[:nsp]) * math.exp(
        max(s["b"] for s in SPECIES[:nsp]) - 3.0)
    rho = np.arange(n, dtype=np.float64) * (rho_max / (n - 1))
    f = np.stack([truncated(*dens(a), rc)[0](r) for a in range(nsp)])
    F = np.stack([emb(a)[0](rho) for a in range(nsp)])
    phi = np.stack([truncated(*pair(a, b), rc)[0](r) for a in range(nsp) for b in range(a, nsp)])
    return AlloyPotential(nsp, n, rc, rho_max, f, F, phi)


def random_types(n_atoms: int, fractions, seed: int) -> np.ndarray:
    """Species of each atom: i.i.d. draws with the given fractions (int8)."""
    g = _rng(seed)
    p = np.asarray(fractions, dtype=np.float64)
    return g.choice(len(p), size=n_atoms, p=p / p.sum()).astype(np.int8)


def knot_perturbation(n: int, sigma: float, seed: int):
    """Three arrays eps ~ N(0, sigma^2), one per table."""
    g = _rng(seed)
    return g.normal(0.0, sigma, n), g.normal(0.0, sigma, n), g.normal(0.0, sigma, n)


# ---------------------------------------------------------------------------
# crystal, velocities, knock-on atom
# ---------------------------------------------------------------------------

def box(nx, ny, nz, a0=A0_FE):
    return np.array([nx * a0, ny * a0, nz * a0], dtype=np.float64)


def bcc_positions(nx, ny, nz, a0=A0_FE) -> np.ndarray:
    """(2 nx ny nz, 3) atom positions of a perfect bcc crystal.  Atom q sits
    at cell (cx, cy, cz) with q = ((cz ny + cy) nx + cx) 2 + b; b = 0 is the
    cube corner, b = 1 the body centre."""
    cz, cy, cx, b = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), np.arange(2),
                                indexing="ij")
    half = 0.5 * b
    pos = np.stack([(cx + half) * a0, (cy + half) * a0, (cz + half) * a0], axis=-1)
    return pos.reshape(-1, 3).astype(np.float64)


def maxwell_velocities(n_atoms: int, T: float, mass: float, seed: int) -> np.ndarray:
    """(N, 3) velocities in A/fs at temperature T (K), zero total momentum,
    kinetic energy exactly 3/2 N kB T."""
    if n_atoms == 0 or T <= 0.0:
        return np.zeros((n_atoms, 3))
    g = _rng(seed)
    sigma = math.sqrt(KB_EV * T / (mass * EV_PER_AMU_A2_FS2))
    v = g.standard_normal((n_atoms, 3)) * sigma
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass * EV_PER_AMU_A2_FS2 * float(np.sum(v * v))
    target = 1.5 * n_atoms * KB_EV * T
    v *= math.sqrt(target / ke)
    return v


def random_direction(seed: int) -> np.ndarray:
    g = _rng(seed)
    while True:
        d = g.standard_normal(3)
        nrm = float(np.linalg.norm(d))
        if nrm > 1e-6:
            return d / nrm


def pka_atom(nx, ny, nz) -> int:
    """The atom at the box centre in bcc_positions order (cube corner of cell
    (nx//2, ny//2, nz//2)), the knock-on atom of the paper's cascade runs."""
    return ((nz // 2 * ny + ny // 2) * nx + nx // 2) * 2


# ---------------------------------------------------------------------------
# parity snapshots
# ---------------------------------------------------------------------------

def thermal_snapshot(nx, ny, nz, sigma: float, seed: int, a0=A0_FE) -> np.ndarray:
    """bcc positions with i.i.d. Gaussian displacements of std sigma (A) per
    component; the thermal snapshots of the potential-fitting workload use
    sigma = 0.1 sqrt(T / 600 K)."""
    g = _rng(seed)
    x = bcc_positions(nx, ny, nz, a0)
    return x + g.normal(0.0, sigma, x.shape)


def cascade_snapshot(nx, ny, nz, sigma: float, n_interstitial: int, n_close: int, seed: int,
                     a0=A0_FE, min_dist: float = 0.9) -> np.ndarray:
    """Thermal snapshot with cascade-like damage: n_interstitial atoms moved to
    uniformly random points (each leaves a vacancy behind and becomes a
    run-away atom; points closer than min_dist to another atom are redrawn),
    and n_close atoms pushed towards a neighbour so that the pair distance
    falls to 1.0-1.8 A."""
    g = _rng(seed)
    x = bcc_positions(nx, ny, nz, a0)
    x = x + g.normal(0.0, sigma, x.shape)
    L = box(nx, ny, nz, a0)
    n = x.shape[0]
    chosen = g.choice(n, size=min(n, n_interstitial + 2 * n_close), replace=False)
    movers = chosen[:n_interstitial]
    for q in movers:
        for _ in range(1000):
            p = g.uniform(0.0, 1.0, 3) * L
            d = x - p
            d -= L * np.round(d / L)
            r = np.sqrt(np.sum(d * d, axis=1))
            r[q] = np.inf
            if r.min() > min_dist:
                x[q] = p
                break
    pairs = chosen[n_interstitial:]
    for k in range(0, len(pairs) - 1, 2):
        a = pairs[k]
        d = x - x[a]
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        r[a] = np.inf
        b = int(np.argmin(r))
        target = g.uniform(1.0, 1.8)
        u = d[b] / r[b]
        x[a] = x[b] - u * target
    return np.mod(x, L)


def interstitial_snapshot(nx, ny, nz, sigma: float, n_interstitial: int, seed: int, a0=A0_FE) -> np.ndarray:
    """Thermal snapshot with n_interstitial atoms moved to distinct
    octahedral interstitial points (cube edge centres, a0/2 from two lattice
    atoms) of random cells: each leaves a vacancy and becomes a run-away.
    Needs no distance search, so it scales to millions of atoms and
    thousands of interstitials (a cascade's run-away load)."""
    g = _rng(seed)
    x = thermal_snapshot(nx, ny, nz, sigma, seed + 1, a0)
    n = x.shape[0]
    movers = g.choice(n, size=n_interstitial, replace=False)
    ncell = nx * ny * nz
    slots = g.choice(3 * ncell, size=n_interstitial, replace=False)  # (cell, axis of the edge)
    cell, axis = slots // 3, slots % 3
    cz, rest = cell // (nx * ny), cell % (nx * ny)
    cy, cx = rest // nx, rest % nx
    p = np.stack([cx, cy, cz], axis=1).astype(np.float64)
    p[np.arange(n_interstitial), axis] += 0.5
    x[movers] = p * a0
    return np.mod(x, box(nx, ny, nz, a0))


# ---------------------------------------------------------------------------
# batched cascades and fitting snapshots
# ---------------------------------------------------------------------------

@dataclass
class Replica:
    nx: int
    ny: int
    nz: int
    T: float
    pka_energy: float
    pka_dir: np.ndarray
    seed: int


def batch_replicas(n: int, seed: int, lo: int = 20, hi: int = 60) -> list:
    """Uneven replicas of the batched cascade workload: dims ~ U{lo..hi} each,
    T ~ U[300, 900] K, knock-on energy ~ U[1, 5] keV, isotropic direction."""
    g = _rng(seed)
    out = []
    for r in range(n):
        dims = g.integers(lo, hi + 1, size=3)
        T = float(g.uniform(300.0, 900.0))
        E = float(g.uniform(1000.0, 5000.0))
        out.append(Replica(int(dims[0]), int(dims[1]), int(dims[2]), T, E,
                           random_direction(seed * 1000 + r + 1), seed * 1000 + r + 7))
    return out


def fitting_snapshots(n_snap: int, nx: int, seed: int, a0=A0_FE):
    """Thermal snapshots of the potential-fitting workload: T_s ~ U[300, 1500] K,
    sigma_s = 0.1 A sqrt(T_s / 600 K)."""
    g = _rng(seed)
    temps = g.uniform(300.0, 1500.0, n_snap)
    snaps = [thermal_snapshot(nx, nx, nx, 0.1 * math.sqrt(T / 600.0), seed * 100 + s, a0)
             for s, T in enumerate(temps)]
    return temps, snaps
