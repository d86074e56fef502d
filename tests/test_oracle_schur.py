"""Pins of the oracle's Schur-complement Sternheimer solve (oracle/schur.py)
against what holds independently of its formulas: the solution equals the
pseudo-inverse solution A^+ Q b of the plain equation (numpy.linalg.pinv) for
exact and for perturbed extra bands; for exact extra bands the smallest
eigenvalue of S on range(R) is eps_{Nocc+Nx+1} - eps_n; CG on S reaches the
tolerance in fewer iterations than the plain projected CG on the band with
the smallest gap."""
import numpy as np
import pytest

from oracle import gmres, groundstate, schur


@pytest.fixture(scope="module")
def block():
    from workloads import make_system
    gs = groundstate.solve(make_system("tiny_insulator"))
    return gs.kblocks[0]


def _setup(kb, nx, perturb, seed=0):
    rng = np.random.default_rng(seed)
    no = kb.nocc
    Phi = kb.vecs[:, :no]
    Psi = kb.vecs[:, no:no + nx].copy()
    if perturb:
        Psi = Psi + perturb * (rng.normal(size=Psi.shape) + 1j * rng.normal(size=Psi.shape))
        Psi = Psi - Phi @ (Phi.conj().T @ Psi)
        Psi = np.linalg.qr(Psi)[0]
    b = rng.normal(size=kb.H.shape[0]) + 1j * rng.normal(size=kb.H.shape[0])
    return Phi, Psi, b


@pytest.mark.parametrize("perturb", [0.0, 1e-2])
def test_schur_solution_equals_pseudo_inverse(block, perturb):
    kb = block
    Phi, Psi, b = _setup(kb, 6, perturb)
    Q = np.eye(kb.H.shape[0]) - Phi @ Phi.conj().T
    for n in range(kb.nocc):
        A = Q @ (kb.H - kb.eps[n] * np.eye(kb.H.shape[0])) @ Q
        x_ref = np.linalg.pinv(A, rcond=1e-12, hermitian=True) @ (Q @ b)
        x = schur.schur_solve(kb.H, kb.eps[n], Phi, Psi, b)
        assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_schur_spectrum_for_exact_extra_bands(block):
    kb = block
    nx = 6
    Phi, Psi, _ = _setup(kb, nx, 0.0)
    S, R = schur.schur_operator(kb.H, kb.eps[kb.nocc - 1], Phi, Psi)
    nb = kb.H.shape[0]
    U = np.linalg.qr(np.concatenate([Phi, Psi], axis=1), mode="complete")[0][:, kb.nocc + nx:]
    Smat = U.conj().T @ np.stack([S(U[:, j]) for j in range(U.shape[1])], axis=1)
    lam = np.linalg.eigvalsh(0.5 * (Smat + Smat.conj().T))
    assert abs(lam.min() - (kb.eps[kb.nocc + nx] - kb.eps[kb.nocc - 1])) <= 1e-10
    assert nb == U.shape[0]


def test_schur_cg_fewer_iterations_on_the_smallest_gap(block):
    kb = block
    n = kb.nocc - 1
    Phi, Psi, b = _setup(kb, 6, 0.0)
    Q = np.eye(kb.H.shape[0]) - Phi @ Phi.conj().T
    b = Q @ b
    b /= np.linalg.norm(b)
    kappa = 1.0
    x0, it0, r0 = gmres.sternheimer_cg(kb.H, kb.eps[n], Phi, b, 1e-10, kb.kinetic, kappa)
    x1, it1, r1 = schur.schur_cg(kb.H, kb.eps[n], Phi, Psi, b, 1e-10, kb.kinetic, kappa)
    assert r0 <= 1e-10 and r1 <= 1e-10
    assert it1 < it0
    A = Q @ (kb.H - kb.eps[n] * np.eye(kb.H.shape[0])) @ Q
    assert np.linalg.norm(A @ x1 - b) <= 1e-8
