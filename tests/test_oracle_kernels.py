"""Pins for K^H, K^xc and the Kerker preconditioner (Sec. 3.4.3; eqs.
precond_dyson, kerker; Lemma kerker_properties).  CPU only."""
import numpy as np

from oracle import basis, dft, response

LAT = np.diag([5.0, 6.0, 7.0])
DIMS = (10, 12, 14)


def _r():
    fr = np.stack(np.meshgrid(*[np.arange(n) / n for n in DIMS], indexing="ij"), -1)
    return fr @ LAT.T


def test_hartree_on_plane_waves():
    """K^H cos(G.r) = 4 pi/|G|^2 cos(G.r), K^H of a constant is 0."""
    B = basis.reciprocal_lattice(LAT)
    r = _r()
    for j in [(1, 0, 0), (0, 2, -1), (3, 1, 2)]:
        G = B @ np.array(j, float)
        v = np.cos(r @ G)
        np.testing.assert_allclose(response.hartree(v, LAT, DIMS), 4 * np.pi / (G @ G) * v,
                                   atol=1e-12)
    assert np.abs(response.hartree(np.full(DIMS, 2.5), LAT, DIMS)).max() < 1e-12


def test_hartree_solves_poisson():
    """-Laplace(K^H v) = 4 pi (v - mean v), Laplacian taken as -|G|^2 on the grid."""
    rng = np.random.default_rng(0)
    v = rng.normal(size=DIMS)
    vh = response.hartree(v, LAT, DIMS)
    G = basis.grid_G(LAT, DIMS)
    G2 = (G * G).sum(-1)
    lap = (dft.grid_synthesis(-G2 * dft.grid_analysis(vh)) / v.size).real
    np.testing.assert_allclose(-lap, 4 * np.pi * (v - v.mean()), atol=1e-10)


def test_exchange_kernel_is_derivative_of_exchange_potential():
    rho = np.geomspace(1e-6, 5.0, 50)
    h = 1e-6 * rho
    fd = (response.exchange_potential(rho + h) - response.exchange_potential(rho - h)) / (2 * h)
    np.testing.assert_allclose(response.exchange_kernel(rho), fd, rtol=1e-7)
    assert response.exchange_kernel(np.array([1e-12]))[0] == 0.0


def test_kerker_properties():
    """Lemma kerker_properties: T is Hermitian positive definite with ||T|| = 1,
    and eq. kerker (projected form with the unmodified D) equals D with D_11 := 1."""
    dims, lat, alpha = (4, 5, 6), np.diag([3.0, 3.5, 4.0]), 0.8
    ng = int(np.prod(dims))
    T = response.dense_operator(lambda v: response.kerker(v, lat, dims, alpha), dims)
    np.testing.assert_allclose(T, T.T, atol=1e-13)
    ev = np.linalg.eigvalsh(T)
    assert ev.min() > 0 and abs(ev.max() - 1.0) < 1e-12
    assert abs(np.linalg.norm(T, 2) - 1.0) < 1e-12
    # eq. kerker, built from the explicit DFT matrix and the unmodified D
    W = dft.unitary_dft_matrix(dims)
    G = basis.grid_G(lat, dims).reshape(-1, 3)
    G2 = (G * G).sum(-1)
    D = np.diag(G2 / (G2 + alpha ** 2))
    one = np.ones((ng, 1))
    T_paper = (np.eye(ng) - one @ one.T / ng) @ (np.linalg.inv(W) @ D @ W) + one @ one.T / ng
    np.testing.assert_allclose(T, T_paper.real, atol=1e-12)
    assert np.abs(T_paper.imag).max() < 1e-12
    # charge conservation
    rng = np.random.default_rng(1)
    v = rng.normal(size=dims)
    assert abs(response.kerker(v, lat, dims, alpha).sum() - v.sum()) < 1e-11
