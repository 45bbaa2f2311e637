"""Seeded synthetic inputs for the parallel orbital-updating solver.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no stencil, no density, no orthonormalisation), so the
GPU path and the CPU oracle can both be fed from it without sharing code.

Workloads stand in for the paper's molecules (Section 4): periodic cubic
boxes with Gaussian local wells V(r) = -Z exp(-|r-R|^2 / (2 sigma^2)),
sigma = 0.8 bohr, atoms placed uniformly with a minimum-image separation of
2 bohr, Z chosen so that sum(Z) is about 2N (a roughly neutral system), and
random initial orbitals with i.i.d. N(0,1) entries (the paper starts from
LCAO orbitals, which need atomic data that is not available here).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

WELL_WIDTH = 0.8  # bohr
MIN_SEPARATION = 2.0  # bohr


@dataclass(frozen=True)
class Workload:
    """One synthetic system: box, grid, stencil, atoms recipe and N."""

    name: str
    L: float  # cubic box edge, bohr
    n: int  # grid points per axis
    order: int  # 2 -> 7-point Laplacian, 4 -> 13-point Laplacian
    n_atoms: int
    z_recipe: str  # "const4", "set246" or "uniform26"
    N: int  # doubly occupied orbitals
    iterations: int
    seed: int
    hartree: int = 1
    exchange: int = 1
    width: float = WELL_WIDTH


WORKLOADS = {
    # plain method, FP64: L=10, 32^3, 7-point, 2 atoms Z=4, N=4, 200 iterations
    "l10_g32_n4": Workload("l10_g32_n4", 10.0, 32, 2, 2, "const4", 4, 200, 1),
    # differentiation: L=12, 64^3, 7-point, 4 atoms Z in {2,4,6}, N=8
    "l12_g64_n8": Workload("l12_g64_n8", 12.0, 64, 2, 4, "set246", 8, 300, 2),
    # precision form: L=20, 96^3, 7-point, 16 atoms Z~U[2,6], N=32
    "l20_g96_n32": Workload("l20_g96_n32", 20.0, 96, 2, 16, "uniform26", 32, 1000, 3),
    # headline: L=30, 160^3, 13-point, 64 atoms Z~U[2,6], N=128
    "l30_g160_n128": Workload("l30_g160_n128", 30.0, 160, 4, 64, "uniform26", 128, 2000, 4),
    # reduced headline system for hardware-counter captures (block > L2, a few GB on the device)
    "l24_g128_n64": Workload("l24_g128_n64", 24.0, 128, 4, 32, "uniform26", 64, 100, 6),
    # reduced 512-orbital system for hardware-counter captures of the several-block kernels
    # (block 226 MB > L2, under 3 GB on the device): L=12, 48^3, 13-point, 64 atoms Z~U[2,6], N=512
    "l12_g48_n512": Workload("l12_g48_n512", 12.0, 48, 4, 64, "uniform26", 512, 20, 7),
    # large: L=40, 192^3, 13-point, 256 atoms Z~U[2,6], N=512, 100 iterations
    "l40_g192_n512": Workload("l40_g192_n512", 40.0, 192, 4, 256, "uniform26", 512, 100, 5),
}


def _min_image_dist(a: np.ndarray, b: np.ndarray, L: float) -> float:
    d = a - b
    d -= L * np.round(d / L)
    return float(np.sqrt(np.sum(d * d)))


def atoms(seed: int, n_atoms: int, L: float, z_recipe: str,
          min_sep: float = MIN_SEPARATION) -> Tuple[np.ndarray, np.ndarray]:
    """Atom positions R (n_atoms x 3, bohr, in [0, L)) and charges Z.

    Positions are drawn uniformly in the box and rejected when closer than
    ``min_sep`` (minimum image) to an accepted atom.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R = np.zeros((n_atoms, 3))
    k = 0
    tries = 0
    while k < n_atoms:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("could not place atoms with the requested separation")
        p = rng.uniform(0.0, L, size=3)
        if all(_min_image_dist(p, R[j], L) >= min_sep for j in range(k)):
            R[k] = p
            k += 1
    if z_recipe == "const4":
        Z = np.full(n_atoms, 4.0)
    elif z_recipe == "set246":
        Z = rng.choice(np.array([2.0, 4.0, 6.0]), size=n_atoms)
    elif z_recipe == "uniform26":
        Z = rng.uniform(2.0, 6.0, size=n_atoms)
    else:
        raise ValueError(f"unknown z_recipe {z_recipe!r}")
    return R, Z


def random_orbitals(seed: int, N: int, n: Tuple[int, int, int], count: Optional[int] = None,
                    dtype=np.float64) -> np.ndarray:
    """Raw initial orbitals, i.i.d. N(0,1), shape (N, nz, ny, nx).

    They are not orthonormal: each solver orthonormalises them itself.
    ``count`` < N returns only the first ``count`` orbitals of the same draw
    (the generator fills the array in order, so they are identical).
    ``dtype=np.float32`` draws in single precision, orbital by orbital (a
    different draw from the float64 one, and half the host memory: for the
    largest workloads, whose float64 block would not be needed anyway).
    """
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    k = N if count is None else min(int(count), N)
    if dtype == np.float64:
        return rng.standard_normal((k, nz, ny, nx))
    out = np.empty((k, nz, ny, nx), dtype=np.float32)
    for i in range(k):
        out[i] = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    return out


def random_field(seed: int, n: Tuple[int, int, int], lo: float = 0.0,
                 hi: float = 1.0) -> np.ndarray:
    """A seeded uniform scalar field of shape (nz, ny, nx)."""
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.uniform(lo, hi, size=(nz, ny, nx))


def workload_inputs(name: str, dtype=None):
    """(workload, R, Z, U0_raw) for one named workload; U0 in float64, or in
    float32 for the workloads whose block exceeds 4 GB (unless ``dtype`` says)."""
    w = WORKLOADS[name]
    R, Z = atoms(w.seed, w.n_atoms, w.L, w.z_recipe)
    if dtype is None:
        dtype = np.float32 if w.N * w.n ** 3 * 8 > (4 << 30) else np.float64
    U0 = random_orbitals(w.seed, w.N, (w.n, w.n, w.n), dtype=dtype)
    return w, R, Z, U0
