"""Kleinman-Bylander nonlocal projectors of the synthetic systems.  Test
infrastructure: only tests/, the smoke check and bench.py's CPU baseline use
the oracle.

The paper's GTH pseudopotentials (Sec. 4) carry nonlocal projectors; the
large Gamma-point workload stands in for them with separable Gaussian s and p
channels on every pseudo-atom,

    V_nl = sum_j D_j |beta_j><beta_j|,

with unit-norm projectors centred at R (periodically repeated):

    beta_s(r)   = (pi sigma^2)^{-3/4} exp(-|r|^2 / (2 sigma^2)),
    beta_p,a(r) = sqrt(2)/sigma (pi sigma^2)^{-3/4} r_a exp(-|r|^2 / (2 sigma^2)).

In the normalised plane-wave basis e_q = e^{i q.r}/sqrt(Omega), q = k + G
(Sec. 2.3.1), a periodically repeated function has the coefficients

    <e_q | beta(. - R)> = e^{-i q.R} betahat(q) / sqrt(Omega),

with betahat the continuum Fourier transform, for these Gaussians

    betahat_s(q)   = (4 pi sigma^2)^{3/4} exp(-sigma^2 q^2 / 2),
    betahat_p,a(q) = -i sigma^2 q_a sqrt(2)/sigma (pi sigma^2)^{-3/4} (2 pi sigma^2)^{3/2}
                     exp(-sigma^2 q^2 / 2).

Projector order: for every centre s, p_x, p_y, p_z (4 per centre).
"""
from __future__ import annotations

import numpy as np

from . import basis


def projectors(lattice, miller, kfrac, centers, sigma) -> np.ndarray:
    """(Nb, 4 Ncentres) complex: column j = coefficients of beta_j on the sphere."""
    B = basis.reciprocal_lattice(lattice)
    q = (np.asarray(miller, dtype=np.float64) + np.asarray(kfrac, dtype=np.float64)) @ B.T
    q2 = np.einsum("gi,gi->g", q, q)
    omega = float(abs(np.linalg.det(lattice)))
    ss, sp = sigma
    gs = (4.0 * np.pi * ss * ss) ** 0.75 * np.exp(-0.5 * ss * ss * q2)
    cp = (np.sqrt(2.0) / sp) * (np.pi * sp * sp) ** -0.75 * (2.0 * np.pi * sp * sp) ** 1.5
    gp = -1j * sp * sp * cp * np.exp(-0.5 * sp * sp * q2)
    cols = []
    for R in np.atleast_2d(centers):
        ph = np.exp(-1j * (q @ R)) / np.sqrt(omega)
        cols.append(ph * gs)
        for a in range(3):
            cols.append(ph * gp * q[:, a])
    return np.stack(cols, axis=1)


def couplings(centers, D) -> np.ndarray:
    """(4 Ncentres,) D_j: D_s for the s channel, D_p for the three p channels."""
    n = len(np.atleast_2d(centers))
    return np.tile(np.array([D[0], D[1], D[1], D[1]], dtype=np.float64), n)


def nonlocal_matrix(lattice, miller, kfrac, centers, sigma, D) -> np.ndarray:
    """V_nl on the sphere: B diag(D) B^H."""
    Bm = projectors(lattice, miller, kfrac, centers, sigma)
    return (Bm * couplings(centers, D)) @ Bm.conj().T
