"""Pins for the oracle's bases and transforms (Sec. 2.3.1, eqs. fourier_bases,
Nb_Ng_definition, fft_ifft; Prop. FinvPhi_bound).  CPU only."""
import numpy as np
import pytest

from oracle import basis, dft

LAT = np.array([[5.0, 0.0, 0.0], [0.3, 6.0, 0.0], [0.0, -0.4, 7.0]]).T   # non-orthogonal cell
DIMS = (6, 5, 8)                      # odd and even sizes


def _sphere(Ecut=1.2, k=(0.25, -0.1, 0.3)):
    return basis.sphere(LAT, DIMS, Ecut, k)


def test_sphere_is_exactly_the_ball():
    """Every frequency of the grid is in G_k iff |k+G|^2 <= 2 Ecut (brute force)."""
    Ecut, k = 1.2, np.array([0.25, -0.1, 0.3])
    miller, flat, kin = _sphere(Ecut, k)
    B = basis.reciprocal_lattice(LAT)
    allm = basis.grid_millers(DIMS).reshape(-1, 3)
    q = (allm + k) @ B.T
    inside = 0.5 * (q * q).sum(1) <= Ecut
    assert set(map(tuple, allm[inside])) == set(map(tuple, miller))
    qs = (miller + k) @ B.T
    np.testing.assert_allclose(kin, 0.5 * (qs * qs).sum(1), rtol=0, atol=1e-14)
    # lexicographic order of signed Miller triples
    assert [tuple(m) for m in miller] == sorted(tuple(m) for m in miller)


def test_reciprocal_duality():
    B = basis.reciprocal_lattice(LAT)
    np.testing.assert_allclose(B.T @ LAT, 2 * np.pi * np.eye(3), atol=1e-13)


def test_separable_sums_match_full_unitary_dft():
    """F^{-1} = w^{-1} W^{-1} Z and F = w Z^T W with the explicit Ng x Ng matrix W."""
    rng = np.random.default_rng(0)
    miller, flat, _ = _sphere()
    vol = abs(np.linalg.det(LAT))
    ng = int(np.prod(DIMS))
    W = dft.unitary_dft_matrix(DIMS)
    w = np.sqrt(vol) / np.sqrt(ng)
    Z = np.zeros((ng, len(flat)))
    Z[flat, np.arange(len(flat))] = 1.0
    c = rng.normal(size=len(flat)) + 1j * rng.normal(size=len(flat))
    ref = (np.linalg.inv(W) @ Z @ c) / w
    np.testing.assert_allclose(dft.F_inv(c, flat, DIMS, vol).ravel(), ref, atol=1e-12)
    x = rng.normal(size=ng) + 1j * rng.normal(size=ng)
    np.testing.assert_allclose(dft.F(x.reshape(DIMS), flat, DIMS, vol), w * Z.T @ W @ x, atol=1e-12)


def test_grid_sums_match_library_fft():
    """Special case reducing to a library routine: grid_analysis is numpy's
    unnormalised forward FFT and grid_synthesis is Ng times its inverse."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=DIMS) + 1j * rng.normal(size=DIMS)
    np.testing.assert_allclose(dft.grid_analysis(x), np.fft.fftn(x), atol=1e-11)
    np.testing.assert_allclose(dft.grid_synthesis(x), np.fft.ifftn(x) * x.size, atol=1e-11)


def test_plane_wave_maps_to_its_values():
    """F^{-1} e_G = e^{i G.r} / sqrt(|Omega|) with G.r from Cartesian vectors."""
    miller, flat, _ = _sphere()
    vol = abs(np.linalg.det(LAT))
    B = basis.reciprocal_lattice(LAT)
    fr = np.stack(np.meshgrid(*[np.arange(n) / n for n in DIMS], indexing="ij"), -1)
    r = fr @ LAT.T
    for idx in [0, len(flat) // 3, len(flat) - 1]:
        c = np.zeros(len(flat), dtype=complex)
        c[idx] = 1.0
        G = B @ miller[idx]
        ref = np.exp(1j * (r @ G)) / np.sqrt(vol)
        np.testing.assert_allclose(dft.F_inv(c, flat, DIMS, vol), ref, atol=1e-13)


def test_F_inverts_F_inv_on_the_sphere():
    rng = np.random.default_rng(2)
    miller, flat, _ = _sphere()
    vol = abs(np.linalg.det(LAT))
    c = rng.normal(size=(3, len(flat))) + 1j * rng.normal(size=(3, len(flat)))
    np.testing.assert_allclose(dft.F(dft.F_inv(c, flat, DIMS, vol), flat, DIMS, vol), c, atol=1e-12)


def test_real_space_orbitals_orthonormal_and_row_norm_bounds():
    """Prop. FinvPhi_bound: Phi_real = sqrt(|Omega|/Ng) F^{-1} Phi has orthonormal
    columns and sqrt(Nocc/|Omega|) <= ||F^{-1} Phi||_{2,inf} <= sqrt(Ng/|Omega|)."""
    rng = np.random.default_rng(3)
    miller, flat, _ = _sphere(Ecut=2.0, k=(0, 0, 0))
    vol = abs(np.linalg.det(LAT))
    ng = int(np.prod(DIMS))
    Phi, _ = np.linalg.qr(rng.normal(size=(len(flat), 4)) + 1j * rng.normal(size=(len(flat), 4)))
    psi = dft.F_inv(Phi.T, flat, DIMS, vol).reshape(4, -1).T          # (Ng, 4)
    Preal = np.sqrt(vol / ng) * psi
    np.testing.assert_allclose(Preal.conj().T @ Preal, np.eye(4), atol=1e-12)
    rown = np.sqrt((np.abs(psi) ** 2).sum(1)).max()
    assert np.sqrt(4 / vol) - 1e-12 <= rown <= np.sqrt(ng / vol) + 1e-12


@pytest.mark.parametrize("Ecut,L", [(15.0, 10.26), (10.0, 10.0)])
def test_sphere_size_matches_asymptotic_formula(Ecut, L):
    """eq. Nb_Ng_definition: Nb ~ sqrt(2)/(3 pi^2) Ecut^{3/2} |Omega| (within 3 %)."""
    lat = np.eye(3) * L
    miller, _, _ = basis.sphere(lat, (64, 64, 64), Ecut, (0, 0, 0))
    est, _ = basis.estimated_sizes(Ecut, L ** 3)
    assert abs(len(miller) - est) / est < 0.03


def test_paper_basis_ratio():
    """Golden: the paper's Ng ~ 16 Nb (Sec. 2.4) is the ratio 48/pi of the two
    asymptotic sizes, and its aluminium system prints Ng = 911,250 with
    Nb ~ 54,200 (tests/golden/paper_sizes.txt)."""
    rows = {}
    for line in open(__file__.replace("test_oracle_dft.py", "golden/paper_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            name, ng, nb = line.split()[:3]
            rows[name] = (float(ng), float(nb))
    nb_est, ng_est = basis.estimated_sizes(40.0, 1000.0)
    assert abs(ng_est / nb_est - 48 / np.pi) < 1e-12
    ng, nb = rows["Al40"]
    assert abs(ng / nb - 48 / np.pi) / (48 / np.pi) < 0.12
