"""Seeded synthetic disk clusters and incidence angles.

This module only draws inputs: disk centres and radii, boundary-condition
flags, wavenumbers, truncation orders and angle grids.  It holds none of the
scattering arithmetic, so both the CUDA path and the CPU oracle can consume
what it produces without sharing any computation.

The shapes follow the paper's workloads: random clusters of non-overlapping
disks in a square (section 6.1, the ``CreateRandomDisks`` generator with a
minimal distance between disks), square lattices (``RectangularLattice``),
plane-wave incidences (Prop. 4.1) and far-field sample angles (section 4.4).

Readings fixed here (the paper leaves them open):
  * "density" of a random cluster is the area fraction of the disks;
  * random placement is random sequential addition with rejection of any
    centre closer than a_p + a_q + gap to an earlier disk;
  * far-field angles are theta_j = 2*pi*j/T, incidences beta_r = 2*pi*r/R;
  * wavenumbers of mixed Dirichlet/Neumann clusters are redrawn when k*a lies
    within 1e-4 (relative) of a zero of some J_m, m <= N, because the
    single-layer Neumann system has a pole there.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
NEUMANN = 1


@dataclass
class Cluster:
    """One scattering configuration: M disks, one wavenumber, one truncation."""

    centres: np.ndarray  # [M, 2] float64
    radii: np.ndarray  # [M] float64
    bc: np.ndarray  # [M] int8, 0 Dirichlet / 1 Neumann
    k: float
    N: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.radii.shape[0])

    @property
    def n(self) -> int:
        return 2 * self.N + 1

    @property
    def ntot(self) -> int:
        return self.M * self.n


def angles(count: int) -> np.ndarray:
    """Equally spaced angles 2*pi*j/count, j = 0..count-1."""
    return 2.0 * np.pi * np.arange(count, dtype=np.float64) / count


def random_disks(rng: np.random.Generator, M: int, half_side: float,
                 rmin: float, rmax: float, gap: float,
                 max_tries: int = 2_000_000) -> tuple[np.ndarray, np.ndarray]:
    """Random sequential addition of M disks with centres uniform in
    [-half_side, half_side]^2, radii uniform in [rmin, rmax], and pairwise
    clearance |O_p - O_q| >= a_p + a_q + gap."""
    centres = np.empty((M, 2))
    radii = np.empty(M)
    placed = 0
    tries = 0
    while placed < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_disks: could not place all disks")
        c = rng.uniform(-half_side, half_side, size=2)
        r = rng.uniform(rmin, rmax) if rmax > rmin else rmin
        if placed:
            d = np.hypot(centres[:placed, 0] - c[0], centres[:placed, 1] - c[1])
            if np.any(d < radii[:placed] + r + gap):
                continue
        centres[placed] = c
        radii[placed] = r
        placed += 1
    return centres, radii


def _near_bessel_zero(x: float, N: int, rel: float = 1e-4) -> bool:
    from scipy.special import jn_zeros

    for m in range(N + 1):
        zs = jn_zeros(m, 8)
        if np.any(np.abs(zs - x) <= rel * zs):
            return True
    return False


# --------------------------------------------------------------------------
# The five workload shapes (sizes as stated with each function).
# --------------------------------------------------------------------------

def four_disks() -> Cluster:
    """4 sound-soft unit disks at the corners (2,2),(-2,2),(-2,-2),(2,-2),
    k = 1, N = 12 (100 unknowns)."""
    O = np.array([[2.0, 2.0], [-2.0, 2.0], [-2.0, -2.0], [2.0, -2.0]])
    return Cluster(O, np.ones(4), np.zeros(4, np.int8), 1.0, 12, "four_disks")


def random_cluster_400(seed: int = 2, M: int = 400) -> Cluster:
    """M = 400 sound-soft disks, radii U[0.5, 1.5], centres U[-50, 50]^2,
    gap 0.2, k = 2*pi, N = ceil(k * a_max) + 10 (N = 20 for the seeded draw)."""
    rng = np.random.default_rng(seed)
    O, a = random_disks(rng, M, 50.0, 0.5, 1.5, 0.2)
    k = 2.0 * np.pi
    N = int(math.ceil(k * a.max())) + 10
    cl = Cluster(O, a, np.zeros(M, np.int8), k, N, f"random{M}_k2pi")
    cl.meta["beta"] = float(rng.uniform(0.0, 2.0 * np.pi))
    return cl


def batched_clusters(count: int = 256, seed: int = 3, m_lo: int = 50,
                     m_hi: int = 800) -> list[Cluster]:
    """`count` independent clusters: M ~ U{m_lo..m_hi}, unit radii, area
    fraction 0.2 in a square centred at the origin, gap 0.01, k ~ U[1, 8]
    (redrawn near Bessel zeros), N = ceil(k) + 8, Dirichlet/Neumann flag per
    disk ~ Bernoulli(1/2)."""
    out = []
    for i, ss in enumerate(np.random.SeedSequence(seed).spawn(count)):
        rng = np.random.default_rng(ss)
        M = int(rng.integers(m_lo, m_hi + 1))
        while True:
            k = float(rng.uniform(1.0, 8.0))
            N = int(math.ceil(k)) + 8
            if not _near_bessel_zero(k * 1.0, N):
                break
        half = 0.5 * math.sqrt(M * math.pi / 0.2)
        O, a = random_disks(rng, M, half, 1.0, 1.0, 0.01)
        bc = rng.integers(0, 2, size=M).astype(np.int8)
        out.append(Cluster(O, a, bc, k, N, f"batch{i}"))
    return out


def cluster_200(seed: int = 4) -> Cluster:
    """M = 200 sound-soft disks, radii U[0.8, 1.2], centres U[-30, 30]^2,
    gap 0.2, k = 10, N = 22."""
    rng = np.random.default_rng(seed)
    O, a = random_disks(rng, 200, 30.0, 0.8, 1.2, 0.2)
    return Cluster(O, a, np.zeros(200, np.int8), 10.0, 22, "random200_k10")


def perturbed_target(cl: Cluster, seed: int = 40) -> Cluster:
    """Target geometry for the far-field misfit: centres + 0.05*N(0,1),
    radii * (1 + 0.02*U[-1,1]), same k and N."""
    rng = np.random.default_rng(seed)
    O = cl.centres + 0.05 * rng.standard_normal(cl.centres.shape)
    a = cl.radii * (1.0 + 0.02 * rng.uniform(-1.0, 1.0, cl.M))
    return Cluster(O, a, cl.bc.copy(), cl.k, cl.N, cl.name + "_target")


def lattice_4000(seed: int = 5, M: int = 4000) -> Cluster:
    """First M sites (row-major) of a 64 x 63 square lattice of spacing 1,
    centred at the origin, Gaussian jitter sigma = 0.02 per coordinate,
    radius 0.3, sound-soft, k = 5, N = 15."""
    rng = np.random.default_rng(seed)
    nx, ny = 64, 63
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    sites = np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float64)[:M]
    sites -= np.array([(nx - 1) / 2.0, (ny - 1) / 2.0])
    sites += 0.02 * rng.standard_normal(sites.shape)
    return Cluster(sites, np.full(M, 0.3), np.zeros(M, np.int8), 5.0, 15, f"lattice{M}_k5")


def dort_three_disks(bc: int = DIRICHLET) -> Cluster:
    """Three small, well separated disks of the time-reversal example
    (section 7): centres (0, 20), (10, -10), (-10, -20), radii 0.02, 0.01,
    0.005, k = 2*pi (k a <= 0.126), N = 4, one boundary condition for all."""
    O = np.array([[0.0, 20.0], [10.0, -10.0], [-10.0, -20.0]])
    a = np.array([0.02, 0.01, 0.005])
    return Cluster(O, a, np.full(3, bc, np.int8), 2.0 * np.pi, 4, "dort3")


def penetrable_lattice(half: int = 10, spacing: float = 3.0) -> Cluster:
    """The penetrable example's geometry (section 7, Example II): unit disks
    on the (2 half + 1)^2 square lattice of the given spacing centred on the
    origin, without its middle row and column (400 disks for half = 10),
    exterior k = 1, N = 10 (the interior wavenumber 2 is set separately)."""
    idx = [i for i in range(-half, half + 1) if i != 0]
    O = np.array([[i * spacing, j * spacing] for j in idx for i in idx], dtype=np.float64)
    M = len(O)
    return Cluster(O, np.ones(M), np.zeros(M, np.int8), 1.0, 10, f"penetrable_lattice{M}")


def small_mixed(seed: int = 11, M: int = 6, N: int = 10, k: float = 2.3,
                half_side: float = 8.0) -> Cluster:
    """Small mixed Dirichlet/Neumann cluster for unit tests."""
    rng = np.random.default_rng(seed)
    O, a = random_disks(rng, M, half_side, 0.5, 1.0, 0.3)
    bc = rng.integers(0, 2, size=M).astype(np.int8)
    return Cluster(O, a, bc, k, N, f"small{M}")


def random_cluster(seed: int, M: int, half_side: float, rmin: float,
                   rmax: float, gap: float, k: float, N: int,
                   neumann_fraction: float = 0.0) -> Cluster:
    """Generic random cluster used for parity sweeps."""
    rng = np.random.default_rng(seed)
    O, a = random_disks(rng, M, half_side, rmin, rmax, gap)
    bc = (rng.uniform(size=M) < neumann_fraction).astype(np.int8)
    return Cluster(O, a, bc, k, N, f"rand{M}_s{seed}")
