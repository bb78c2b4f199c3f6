"""Seeded synthetic inputs for the short-range Lennard-Jones MD path.

This module is the one piece shared by the CUDA path's tests/bench and by the
CPU oracle: it only *generates inputs* (lattice sites, jitter, Maxwell
velocities, type assignments, pair parameters, ensemble box sizes).  It holds
none of the method's arithmetic (no binning, no neighbor search, no forces, no
integration).  Every random number comes from ``numpy.random.default_rng(seed)``
(PCG64), so a (recipe, seed) pair fixes the input bit for bit.

Workload recipes follow the classic LJ-melt benchmark that the paper's
CabanaMD proxy uses as its short-range kernel (Section "CabanaMD"): an FCC
crystal at reduced density rho*=0.8442, Gaussian velocities rescaled to
T*=1.44 with zero net momentum, eps=sigma=m=1, cutoff 2.5 sigma, skin 0.3 sigma,
dt=0.005.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RHO_MELT = 0.8442
T_MELT = 1.44
RC = 2.5
SKIN = 0.3
DT = 0.005
REBUILD_EVERY = 20

# FCC conventional-cell basis in units of the lattice constant a.
_FCC_BASIS = np.array([[0.0, 0.0, 0.0],
                       [0.5, 0.5, 0.0],
                       [0.5, 0.0, 0.5],
                       [0.0, 0.5, 0.5]], dtype=np.float64)


def fcc_lattice_constant(rho: float) -> float:
    """Edge a of the conventional FCC cell holding 4 atoms at number density rho."""
    return (4.0 / rho) ** (1.0 / 3.0)


def fcc_sites(nx: int, ny: int, nz: int, a: float) -> np.ndarray:
    """Sites of an nx*ny*nz FCC block, shape (4*nx*ny*nz, 3), float64.

    Order: cells by (iz, iy, ix) with ix fastest, then the 4 basis sites.
    """
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3)
    return sites * a


def maxwell_velocities(n: int, temperature: float, rng: np.random.Generator,
                       mass: np.ndarray | None = None) -> np.ndarray:
    """Gaussian velocities with the mean (mass-weighted) momentum removed and
    rescaled so that 2*KE/(3n-3) equals ``temperature`` exactly (k_B = 1)."""
    v = rng.standard_normal((n, 3))
    m = np.ones(n) if mass is None else np.asarray(mass, dtype=np.float64)
    v_cm = (m[:, None] * v).sum(axis=0) / m.sum()   # centre-of-mass velocity
    v -= v_cm[None, :]
    ke = 0.5 * float((m[:, None] * v * v).sum())
    t_now = 2.0 * ke / (3 * n - 3)
    v *= math.sqrt(temperature / t_now)
    return v


@dataclass
class LJSystem:
    """One periodic orthorhombic box (origin 0) with its pair parameters."""
    x: np.ndarray                 # (n, 3) float64, AoS
    v: np.ndarray                 # (n, 3) float64
    types: np.ndarray             # (n,) int32
    box: np.ndarray               # (3,) float64 edge lengths
    eps: np.ndarray = field(default_factory=lambda: np.ones((1, 1)))
    sigma: np.ndarray = field(default_factory=lambda: np.ones((1, 1)))
    mass: np.ndarray = field(default_factory=lambda: np.ones(1))
    rc: float = RC
    skin: float = SKIN
    dt: float = DT
    rebuild_every: int = REBUILD_EVERY

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def ntypes(self) -> int:
        return int(self.eps.shape[0])


def lj_melt(ncells: int, rho: float = RHO_MELT, temperature: float = T_MELT,
            seed: int = 1, jitter: float = 0.0) -> LJSystem:
    """FCC ncells^3 block (4*ncells^3 atoms) in a cubic periodic box.

    ``jitter`` > 0 adds an independent U(-jitter, +jitter) displacement to each
    coordinate (the 4M-atom workload uses 0.05 sigma).
    """
    rng = np.random.default_rng(seed)
    a = fcc_lattice_constant(rho)
    x = fcc_sites(ncells, ncells, ncells, a)
    if jitter > 0.0:
        x = x + rng.uniform(-jitter, jitter, size=x.shape)
    n = x.shape[0]
    v = maxwell_velocities(n, temperature, rng)
    box = np.full(3, ncells * a)
    return LJSystem(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v),
                    types=np.zeros(n, dtype=np.int32), box=box)


def random_pair_params(ntypes: int, rng: np.random.Generator, lo: float = 0.8,
                       hi: float = 1.2) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric (ntypes, ntypes) eps and sigma tables drawn from U[lo, hi]."""
    eps = np.zeros((ntypes, ntypes))
    sig = np.zeros((ntypes, ntypes))
    for a in range(ntypes):
        for b in range(a, ntypes):
            eps[a, b] = eps[b, a] = rng.uniform(lo, hi)
            sig[a, b] = sig[b, a] = rng.uniform(lo, hi)
    return eps, sig


def two_type_melt(ncells: int = 20, seed: int = 7, rho: float = RHO_MELT,
                  temperature: float = T_MELT, jitter: float = 0.05) -> LJSystem:
    """Force-matching workload: FCC ncells^3 box, two types assigned 50/50 at
    random, per-pair (eps, sigma) in U[0.8, 1.2]."""
    rng = np.random.default_rng(seed)
    a = fcc_lattice_constant(rho)
    x = fcc_sites(ncells, ncells, ncells, a)
    x = x + rng.uniform(-jitter, jitter, size=x.shape)
    n = x.shape[0]
    types = np.zeros(n, dtype=np.int32)
    types[rng.permutation(n)[: n // 2]] = 1
    v = maxwell_velocities(n, temperature, rng)
    eps, sig = random_pair_params(2, rng)
    return LJSystem(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), types=types,
                    box=np.full(3, ncells * a), eps=eps, sigma=sig, mass=np.ones(2))


def vacancy_box(n_atoms: int, rho: float, temperature: float,
                rng: np.random.Generator) -> LJSystem:
    """One ensemble member: the smallest FCC block with >= n_atoms sites, with
    random vacancies down to n_atoms, scaled to density rho."""
    nc = int(math.ceil((n_atoms / 4.0) ** (1.0 / 3.0) - 1e-12))
    edge = (n_atoms / rho) ** (1.0 / 3.0)
    a = edge / nc
    sites = fcc_sites(nc, nc, nc, a)
    keep = np.sort(rng.permutation(sites.shape[0])[:n_atoms])
    x = np.ascontiguousarray(sites[keep])
    v = maxwell_velocities(n_atoms, temperature, rng)
    return LJSystem(x=x, v=np.ascontiguousarray(v), types=np.zeros(n_atoms, dtype=np.int32),
                    box=np.full(3, edge))


def ensemble(nbox: int = 512, seed: int = 11, n_lo: int = 256, n_hi: int = 32768,
             rho_lo: float = 0.7, rho_hi: float = 0.9, t_lo: float = 0.8,
             t_hi: float = 1.6) -> list[LJSystem]:
    """Batched-ensemble workload: ``nbox`` independent boxes, atom counts
    log-uniform in [n_lo, n_hi], densities U[rho_lo, rho_hi], temperatures
    U[t_lo, t_hi], all drawn from one seed."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=nbox))
    counts = np.clip(np.round(counts).astype(np.int64), n_lo, n_hi)
    rhos = rng.uniform(rho_lo, rho_hi, size=nbox)
    temps = rng.uniform(t_lo, t_hi, size=nbox)
    return [vacancy_box(int(counts[b]), float(rhos[b]), float(temps[b]), rng)
            for b in range(nbox)]


def workload(name: str) -> LJSystem:
    """The named single-box workloads, by atom count and recipe."""
    if name == "lj_fcc10_4000":
        return lj_melt(10, seed=1)
    if name == "lj_fcc32_131072":
        return lj_melt(32, seed=2)
    if name == "lj_fcc100_4m":
        return lj_melt(100, seed=3, jitter=0.05)
    if name == "lj_fcc50_500k":         # same recipe at 1/8 size (profiling captures)
        return lj_melt(50, seed=3, jitter=0.05)
    if name == "lj_2type_fcc20_32000":
        return two_type_melt(20, seed=7)
    raise KeyError(name)


# ---- charged inputs (Ewald / SPME long-range path) ------------------------

def neutral_charges(n: int, rng: np.random.Generator, q: float = 1.0) -> np.ndarray:
    """n charges of +q and -q, floor(n/2) of each sign plus one 0 if n is odd,
    assigned to atoms in a random order (a neutral random ionic mixture)."""
    c = np.zeros(n)
    c[: n // 2] = q
    c[n // 2: 2 * (n // 2)] = -q
    return np.ascontiguousarray(c[rng.permutation(n)])


def rocksalt(nc: int, r0: float = 1.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Rock-salt (NaCl) crystal: a simple-cubic nc^3 lattice of spacing r0
    (nc even) with charges (-1)^(i+j+k).  Returns positions, charges, box."""
    if nc % 2:
        raise ValueError("nc must be even for a periodic rock-salt box")
    g = np.arange(nc)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) * float(r0)
    q = np.where((i + j + k).ravel() % 2 == 0, 1.0, -1.0)
    return np.ascontiguousarray(x, dtype=np.float64), q, np.full(3, nc * float(r0))


@dataclass
class ChargedSystem:
    """An LJ melt whose atoms also carry charges, with the Ewald parameters
    of the recipe (splitting alpha, real-space cutoff, grid, spline order)."""
    lj: LJSystem
    q: np.ndarray
    alpha: float
    rc: float
    K: tuple
    order: int


def charged_melt(ncells: int, seed: int, K: int, order: int = 4, jitter: float = 0.05,
                 alpha: float = 1.25, rc: float = RC) -> ChargedSystem:
    """The LJ melt recipe (FCC at rho 0.8442, T 1.44, jitter in sigma) with
    neutral random +-1 charges; alpha rc = 3.125 (erfc(alpha rc) ~ 1e-5)."""
    s = lj_melt(ncells, seed=seed, jitter=jitter)
    q = neutral_charges(s.n, np.random.default_rng(seed + 1000))
    return ChargedSystem(lj=s, q=q, alpha=alpha, rc=rc, K=(K, K, K), order=order)


def charged_workload(name: str) -> ChargedSystem:
    """The named charged workloads (grid K^3 chosen for ~0.44 sigma spacing)."""
    if name == "coulomb_fcc10_4000":
        return charged_melt(10, seed=21, K=40)
    if name == "coulomb_fcc50_500k":
        return charged_melt(50, seed=23, K=192)
    if name == "coulomb_fcc100_4m":
        return charged_melt(100, seed=25, K=384)
    raise KeyError(name)
