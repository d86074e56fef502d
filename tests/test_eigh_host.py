"""The host Jacobi eigensolver of the Rayleigh-Ritz step (ikr_hermitian_eigh)
against LAPACK (numpy.linalg.eigh) on random Hermitian matrices, including
degenerate and diagonal ones: eigenvalues, A V = V diag(w), V^H V = 1."""
import numpy as np
import pytest


def _lib():
    pytest.importorskip("torch")
    from paper_2505_02319_gb300 import ikr
    return ikr


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (30, 3), (64, 4)])
def test_hermitian_eigh_matches_lapack(n, seed):
    ikr = _lib()
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a = a + a.conj().T
    w, v = ikr.hermitian_eigh(a)
    wr = np.linalg.eigvalsh(a)
    scale = max(1.0, np.abs(wr).max())
    assert np.max(np.abs(w - wr)) <= 1e-13 * scale
    assert np.linalg.norm(a @ v - v * w) <= 1e-12 * scale * n
    assert np.linalg.norm(v.conj().T @ v - np.eye(n)) <= 1e-12 * n


def test_hermitian_eigh_degenerate_and_diagonal():
    ikr = _lib()
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    lam = np.array([-2.0] * 4 + [0.5] * 3 + [1.0, 3.0, 3.0, 7.0, 9.0])
    a = (q * lam) @ q.conj().T
    w, v = ikr.hermitian_eigh(a)
    assert np.max(np.abs(w - np.sort(lam))) <= 1e-13 * 9
    assert np.linalg.norm(a @ v - v * w) <= 1e-12 * 9 * 12
    d = np.diag([3.0, -1.0, 2.0]).astype(complex)
    w, v = ikr.hermitian_eigh(d)
    np.testing.assert_array_equal(w, [-1.0, 2.0, 3.0])
