"""Naive discrete Fourier transforms between the sphere and the grid
(Sec. 2.3.1, eq. fft_ifft).  Test infrastructure.

With the unitary DFT W, (W x)_G = Ng^{-1/2} sum_r e^{-i G.r} x_r, and the
weight w = sqrt(|Omega|)/sqrt(Ng):
    F^{-1} c = w^{-1} W^{-1} Z c :  u(r) = |Omega|^{-1/2} sum_{G in sphere} c_G e^{i G.r}
    F x      = w Z^T W x          :  c_G = |Omega|^{1/2} / Ng  sum_r x_r e^{-i G.r}
Because G.r = 2 pi sum_a j_a i_a / N_a on the grid X, each transform is a sum
over one axis at a time (a separable naive DFT, O(Ng (N1+N2+N3)) work).
No FFT algorithm is used here.
"""
from __future__ import annotations

import numpy as np


def _axis_matrix(n: int, sign: int) -> np.ndarray:
    """E[i, p] = exp(sign * 2 pi i * i p / n) for grid position i and frequency slot p."""
    i = np.arange(n)
    # reduce i*p mod n before dividing, to keep the phase argument exact
    return np.exp(sign * 2j * np.pi * (np.outer(i, i) % n) / n)


def grid_synthesis(coef_grid: np.ndarray) -> np.ndarray:
    """sum_G c_G e^{+i G.r} for coefficients laid out on the full grid of
    frequency slots (shape (..., N1, N2, N3)); returns values on X."""
    out = coef_grid.astype(np.complex128)
    nd = out.ndim
    for ax in range(3):
        n = out.shape[nd - 3 + ax]
        E = _axis_matrix(n, +1)
        out = np.moveaxis(np.tensordot(out, E, axes=([nd - 3 + ax], [1])), -1, nd - 3 + ax)
    return out


def grid_analysis(values: np.ndarray) -> np.ndarray:
    """sum_r x_r e^{-i G.r} for every grid frequency slot (shape (..., N1, N2, N3))."""
    out = values.astype(np.complex128)
    nd = out.ndim
    for ax in range(3):
        n = out.shape[nd - 3 + ax]
        E = _axis_matrix(n, -1)
        out = np.moveaxis(np.tensordot(out, E, axes=([nd - 3 + ax], [1])), -1, nd - 3 + ax)
    return out


def F_inv(c: np.ndarray, flat_index: np.ndarray, dims, volume: float) -> np.ndarray:
    """F^{-1}: sphere coefficients (..., Nb) -> grid values (..., N1, N2, N3)."""
    lead = c.shape[:-1]
    pad = np.zeros(lead + (int(np.prod(dims)),), dtype=np.complex128)
    pad[..., flat_index] = c                 # zero padding Z
    pad = pad.reshape(lead + tuple(dims))
    return grid_synthesis(pad) / np.sqrt(volume)


def F(x: np.ndarray, flat_index: np.ndarray, dims, volume: float) -> np.ndarray:
    """F: grid values (..., N1, N2, N3) -> sphere coefficients (..., Nb)."""
    lead = x.shape[:-3]
    ng = int(np.prod(dims))
    full = grid_analysis(x).reshape(lead + (ng,))
    return full[..., flat_index] * (np.sqrt(volume) / ng)   # restriction Z^T


def unitary_dft_matrix(dims) -> np.ndarray:
    """The full Ng x Ng unitary DFT W (only for tiny grids, to pin the
    separable sums): W[G, r] = Ng^{-1/2} exp(-2 pi i sum_a p_a i_a / N_a)."""
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)        # (Ng, 3) positions
    phase = np.zeros((idx.shape[0], idx.shape[0]))
    for a, n in enumerate(dims):
        phase += np.outer(idx[:, a], idx[:, a]) / n
    return np.exp(-2j * np.pi * phase) / np.sqrt(idx.shape[0])
