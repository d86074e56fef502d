"""Plane-wave bases and grids (Sec. 2.3.1, eqs. fourier_bases and
Nb_Ng_definition; k-dependent sphere of Sec. 4.1.1).  Test infrastructure.

Conventions: ``lattice`` has the cell vectors as columns; the reciprocal
vectors b_i satisfy b_i . a_j = 2 pi delta_ij.  A Miller triple (j1,j2,j3)
stands for G = j1 b1 + j2 b2 + j3 b3 and lives at grid position
(j1 mod N1, j2 mod N2, j3 mod N3).  The grid frequency range is
-N/2 <= j < N/2 per axis (Sec. 2.3.1).
"""
from __future__ import annotations

import itertools

import numpy as np


def reciprocal_lattice(lattice: np.ndarray) -> np.ndarray:
    """Columns b_i with b_i . a_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def signed_index(n: int) -> np.ndarray:
    """Signed frequency j of each grid position p = 0..n-1 (j = p - n for p >= n/2)."""
    p = np.arange(n)
    return np.where(p < (n + 1) // 2 if n % 2 else p < n // 2, p, p - n)


def grid_millers(dims) -> np.ndarray:
    """(N1,N2,N3,3) integer Miller triples of the cubic basis G-box (all grid frequencies)."""
    j = [signed_index(n) for n in dims]
    m = np.stack(np.meshgrid(*j, indexing="ij"), axis=-1)
    return m


def grid_G(lattice, dims) -> np.ndarray:
    """(N1,N2,N3,3) Cartesian G vectors of all grid frequencies."""
    return grid_millers(dims) @ reciprocal_lattice(lattice).T


def sphere(lattice, dims, Ecut, kfrac):
    """The spherical basis G_k = {G : |k + G|^2 <= 2 Ecut} (Sec. 4.1.1).

    Returns (miller (Nb,3) int, flat grid index (Nb,) int, kinetic (Nb,) float
    = |k+G|^2 / 2), listed in lexicographic order of the signed (j1, j2, j3).
    Raises if the ball does not fit strictly inside the grid range.
    """
    B = reciprocal_lattice(lattice)
    k = B @ np.asarray(kfrac, dtype=np.float64)
    # bound |j_i| by the ball radius over the dual-lattice direction
    radius = np.sqrt(2.0 * Ecut)
    jmax = [int(np.ceil(radius * np.linalg.norm(np.linalg.inv(B)[i, :]) + 1)) for i in range(3)]
    rows = []
    for j in itertools.product(*[range(-m, m + 1) for m in jmax]):
        q = k + B @ np.array(j, dtype=np.float64)
        e = 0.5 * float(q @ q)
        if e <= Ecut:
            rows.append((j, e))
    miller = np.array([r[0] for r in rows], dtype=np.int64)
    kin = np.array([r[1] for r in rows], dtype=np.float64)
    for i, n in enumerate(dims):
        if miller[:, i].min() < -(n // 2) or miller[:, i].max() >= (n + 1) // 2:
            raise ValueError("plane-wave sphere does not fit inside the FFT grid")
    pos = np.mod(miller, np.array(dims))
    flat = (pos[:, 0] * dims[1] + pos[:, 1]) * dims[2] + pos[:, 2]
    return miller, flat, kin


def estimated_sizes(Ecut, volume):
    """The paper's asymptotic sizes (eq. Nb_Ng_definition):
    Nb ~ sqrt(2)/(3 pi^2) Ecut^{3/2} |Omega|, Ng ~ 16 sqrt(2)/pi^3 Ecut^{3/2} |Omega|."""
    Nb = np.sqrt(2.0) / (3.0 * np.pi ** 2) * Ecut ** 1.5 * volume
    Ng = 16.0 * np.sqrt(2.0) / np.pi ** 3 * Ecut ** 1.5 * volume
    return Nb, Ng
