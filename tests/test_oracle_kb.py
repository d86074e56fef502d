"""Pins of the oracle's Kleinman-Bylander projectors (oracle/kb.py)
against what does not depend on its closed forms: the plane-wave coefficients
equal a brute-force periodic quadrature of the real-space projectors on a fine
grid; Parseval gives unit norm once the sphere holds the Gaussian's transform;
V_nl = B diag(D) B^H is Hermitian, positive semidefinite for D > 0, of rank
4 per centre; the dense H_k of a KB system contains exactly that term."""
import itertools
import math

import numpy as np
import pytest

from oracle import basis, groundstate, kb


def _real_space(lattice, dims, R, sigma, chan, kcart):
    """Bloch sum sum_T e^{i k.T} beta(r - R - T) on the grid (the definitions
    in the oracle's docstring, written out in real space): the function whose
    coefficients in the Bloch basis e^{i(k+G).r}/sqrt(Omega) the oracle gives."""
    fr = [np.arange(n) / n for n in dims]
    f = np.stack(np.meshgrid(*fr, indexing="ij"), axis=-1)
    r = f @ lattice.T
    out = np.zeros(dims, dtype=complex)
    nimg = [int(math.ceil(10 * sigma / np.linalg.norm(lattice[:, i]))) + 1 for i in range(3)]
    norm = (np.pi * sigma * sigma) ** -0.75
    for n in itertools.product(*[range(-m, m + 1) for m in nimg]):
        d = r - (R + lattice @ np.array(n, dtype=float))
        T = lattice @ np.array(n, dtype=float)
        g = np.exp(-np.einsum("...i,...i->...", d, d) / (2 * sigma * sigma)) * norm * np.exp(1j * (kcart @ T))
        out = out + (g if chan == 0 else g * d[..., chan - 1] * math.sqrt(2.0) / sigma)
    return out


def test_coefficients_match_quadrature():
    lattice = np.diag([6.0, 6.5, 7.0])
    dims = (60, 64, 70)
    R = np.array([1.3, 2.9, 4.4])
    sigma = (0.8, 0.9)
    kfrac = np.array([-0.5, 0.25, 0.0])
    miller, _, _ = basis.sphere(lattice, (12, 12, 12), 3.0, kfrac)
    Bm = kb.projectors(lattice, miller, kfrac, R[None, :], sigma)
    Brec = basis.reciprocal_lattice(lattice)
    q = (miller + kfrac) @ Brec.T
    fr = [np.arange(n) / n for n in dims]
    r = np.stack(np.meshgrid(*fr, indexing="ij"), axis=-1) @ lattice.T
    omega = float(np.linalg.det(lattice))
    dV = omega / np.prod(dims)
    kcart = kfrac @ Brec.T
    for chan in range(4):
        beta = _real_space(lattice, dims, R, sigma[0] if chan == 0 else sigma[1], chan, kcart)
        for g in range(0, len(miller), 7):
            num = np.sum(np.exp(-1j * (r @ q[g])) * beta) * dV / math.sqrt(omega)
            assert abs(num - Bm[g, chan]) <= 1e-10 * max(1.0, abs(Bm[:, chan]).max())


def test_unit_norm_by_parseval():
    """Sum over G of |<e_G|beta>|^2 = the cell norm of the Bloch sum, 1 up to the
    overlap with the images (e^{-T^2/4 sigma^2} < 1e-15 here) and the tail outside
    the sphere (e^{-sigma^2 q^2} < 1e-13)."""
    lattice = np.diag([6.0, 6.5, 7.0])
    miller, _, _ = basis.sphere(lattice, (48, 48, 48), 70.0, np.zeros(3))
    Bm = kb.projectors(lattice, miller, np.zeros(3), np.array([[1.0, 2.0, 3.0]]), (0.5, 0.55))
    np.testing.assert_allclose(np.sum(np.abs(Bm) ** 2, axis=0), 1.0, atol=1e-10)


def test_nonlocal_matrix_hermitian_psd_rank():
    lattice = np.diag([6.0, 6.5, 7.0])
    miller, _, _ = basis.sphere(lattice, (12, 12, 12), 3.0, np.array([-0.5, 0, 0]))
    centres = np.array([[1.0, 2.0, 3.0], [4.0, 1.0, 5.5]])
    Vnl = kb.nonlocal_matrix(lattice, miller, np.array([-0.5, 0, 0]), centres, (0.8, 0.9), (1.0, 0.5))
    assert np.allclose(Vnl, Vnl.conj().T, atol=1e-14)
    w = np.linalg.eigvalsh(Vnl)
    assert w.min() > -1e-12
    assert np.sum(w > 1e-8 * w.max()) == 8
    neg = kb.nonlocal_matrix(lattice, miller, np.array([-0.5, 0, 0]), centres, (0.8, 0.9), (-1.0, 0.5))
    assert np.linalg.eigvalsh(neg).min() < -1e-3


def test_kb_system_hamiltonian_contains_the_term():
    from workloads import make_system
    s = make_system("tiny_kb")
    kf = s.kpoints[1]
    m, _, _, H0 = groundstate.hamiltonian(s.lattice, s.dims, s.Ecut, kf, s.V)
    m2, _, _, H1 = groundstate.hamiltonian(s.lattice, s.dims, s.Ecut, kf, s.V, (s.kb_centers, s.kb_sigma, s.kb_D))
    np.testing.assert_array_equal(m, m2)
    Bm = kb.projectors(s.lattice, m, kf, s.kb_centers, s.kb_sigma)
    np.testing.assert_allclose(H1 - H0, (Bm * kb.couplings(s.kb_centers, s.kb_D)) @ Bm.conj().T, atol=1e-14)
    gs = groundstate.solve(s)
    assert groundstate.gap(gs) > 0
