"""Pins for the oracle's Hamiltonian, occupations and density (eqs.
Hamiltonian, density, fprime; k-form of Sec. 4.1.1).  CPU only."""
import numpy as np
import pytest
from scipy.linalg import eigh_tridiagonal

from oracle import basis, dft, groundstate
from workloads import make_system

LAT = np.diag([5.0, 6.0, 7.0])
DIMS = (10, 12, 14)


def test_local_part_equals_explicit_transform_product():
    """Z^T W diag(V) W^{-1} Z built from the explicit matrix W equals the
    closed form Vhat(G-G')/Ng the oracle uses."""
    lat, dims = np.diag([4.0, 4.5, 5.0]), (6, 6, 8)
    rng = np.random.default_rng(0)
    V = rng.normal(size=dims)
    miller, flat, _ = basis.sphere(lat, dims, 1.5, (0.1, 0.2, -0.3))
    W = dft.unitary_dft_matrix(dims)
    full = W @ np.diag(V.ravel()) @ np.linalg.inv(W)
    np.testing.assert_allclose(groundstate.local_potential_matrix(V, miller, dims),
                               full[np.ix_(flat, flat)], atol=1e-12)


def test_hamiltonian_hermitian():
    s = make_system("tiny_ortho_k")
    for k in s.kpoints:
        _, _, _, H = groundstate.hamiltonian(s.lattice, s.dims, s.Ecut, k, s.V)
        np.testing.assert_allclose(H, H.conj().T, atol=1e-14)


def test_free_electrons():
    """V = 0: eigenvalues are exactly |k+G|^2/2."""
    k = (0.3, 0.0, -0.2)
    miller, flat, kin, H = groundstate.hamiltonian(LAT, DIMS, 3.0, k, np.zeros(DIMS))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), np.sort(kin), atol=1e-13)


def test_cosine_potential_reduces_to_tridiagonal_chains():
    """V(r) = 2 V0 cos(b1.r) couples only G and G +- b1: the spectrum is the union
    of tridiagonal chains with diagonal |k+G|^2/2 and off-diagonal V0
    (solved by LAPACK's tridiagonal eigensolver)."""
    V0 = 0.37
    k = np.array([0.1, 0.25, 0.0])
    i1 = np.arange(DIMS[0])[:, None, None] * np.ones(DIMS)
    V = 2 * V0 * np.cos(2 * np.pi * i1 / DIMS[0])
    miller, flat, kin, H = groundstate.hamiltonian(LAT, DIMS, 3.0, k, V)
    ref = []
    for j23 in sorted(set(map(tuple, miller[:, 1:]))):
        sel = np.all(miller[:, 1:] == j23, axis=1)
        order = np.argsort(miller[sel, 0])
        j1 = miller[sel, 0][order]
        assert np.all(np.diff(j1) == 1)      # chains are contiguous
        d = kin[sel][order]
        ref.extend(eigh_tridiagonal(d, np.full(len(d) - 1, V0), eigvals_only=True))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), np.sort(ref), atol=1e-12)


def test_fermi_dirac_derivative_and_level():
    x = np.linspace(-8, 8, 41)
    h = 1e-5
    fd = (groundstate.fermi_dirac(x + h) - groundstate.fermi_dirac(x - h)) / (2 * h)
    np.testing.assert_allclose(groundstate.fermi_dirac_derivative(x), fd, atol=1e-9)
    assert groundstate.fermi_dirac(0.0) == 1.0
    rng = np.random.default_rng(1)
    eps = [np.sort(rng.normal(size=12)) for _ in range(3)]
    w = [0.5, 0.25, 0.25]
    eF = groundstate.fermi_level(eps, w, 7, 0.05)
    total = sum(wk * groundstate.fermi_dirac((e - eF) / 0.05).sum() for e, wk in zip(eps, w))
    assert abs(total - 7) < 1e-10


@pytest.mark.parametrize("name", ["tiny_insulator", "tiny_ortho_k", "tiny_metal"])
def test_density_integrates_to_electron_count(name):
    s = make_system(name)
    gs = groundstate.solve(s)
    assert abs(gs.rho.sum() * gs.volume / gs.n_grid - s.n_electrons) < 1e-8
    assert gs.rho.min() >= 0.0
    for kb in gs.kblocks:
        # orthonormal eigenvectors, residual of the eigenpairs
        np.testing.assert_allclose(kb.vecs.conj().T @ kb.vecs, np.eye(len(kb.eps)), atol=1e-12)
        assert np.abs(kb.H @ kb.vecs[:, :5] - kb.vecs[:, :5] * kb.eps[:5]).max() < 1e-12


def test_insulators_have_a_gap():
    for name in ["tiny_insulator", "tiny_ortho_k"]:
        assert groundstate.gap(groundstate.solve(make_system(name))) > 1e-3
