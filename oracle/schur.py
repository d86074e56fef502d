"""Schur-complement form of the Sternheimer equation.  Test infrastructure:
only tests/, the smoke check and bench.py's CPU baseline use the oracle.

The paper solves every Sternheimer equation (eq. discretised_sternheimer) with
the Schur complement trick of its reference cances2023numerical (Sec. 3.4.2,
Sec. 4.1.2); it names the trick and states its effect (a larger smallest
eigenvalue of the operator actually iterated on, the same solution).  Written
out as block elimination:

With Q = 1 - Phi Phi^H (occupied orbitals Phi) and extra computed bands Psi
(orthonormal, orthogonal to Phi, approximate eigenvectors of H above the
occupied ones), range(Q) splits into span(Psi) and range(R), R = Q - Psi Psi^H.
For x = Psi a + y with y in range(R), Q(H - eps)Q x = Q b reads

    M a + W^H y = Psi^H b,               M = Psi^H (H - eps) Psi,
    W a + R (H - eps) R y = R b,         W = R (H - eps) Psi = R H Psi   (R Psi = 0),

and eliminating a gives the Schur complement on range(R):

    S y = R b - W M^{-1} Psi^H b,        S = R (H - eps) R - W M^{-1} W^H,
    a = M^{-1} (Psi^H b - W^H y).

S is the Schur complement of the positive definite Q(H - eps)Q on range(Q)
(eps an occupied eigenvalue below the gap), hence positive definite on range(R)
and solvable by CG; x equals the pseudo-inverse solution of the original
equation.  For exact eigenvectors W = 0 and S = R(H - eps)R, whose smallest
eigenvalue on range(R) is eps_{Nocc+Nx+1} - eps instead of eps_{Nocc+1} - eps.
"""
from __future__ import annotations

import numpy as np


def _parts(H, eps, Phi, Psi):
    def R(y):
        return y - Phi @ (Phi.conj().T @ y) - Psi @ (Psi.conj().T @ y)

    HPsi = H @ Psi
    M = Psi.conj().T @ HPsi - eps * np.eye(Psi.shape[1])
    W = R(HPsi)
    return R, M, W


def schur_operator(H, eps, Phi, Psi):
    """y -> S y on range(R), and the projector R."""
    R, M, W = _parts(H, eps, Phi, Psi)

    def S(y):
        return R(H @ y - eps * y) - W @ np.linalg.solve(M, W.conj().T @ y)

    return S, R


def schur_solve(H, eps, Phi, Psi, b):
    """x = Psi a + y from the Schur complement, solved directly in an
    orthonormal basis of range(R)."""
    R, M, W = _parts(H, eps, Phi, Psi)
    S, _ = schur_operator(H, eps, Phi, Psi)
    n = H.shape[0]
    basis = np.linalg.qr(np.concatenate([Phi, Psi], axis=1), mode="complete")[0][:, Phi.shape[1] + Psi.shape[1]:]
    rhs = R(b) - W @ np.linalg.solve(M, Psi.conj().T @ b)
    SU = np.stack([S(basis[:, j]) for j in range(basis.shape[1])], axis=1)
    y = basis @ np.linalg.solve(basis.conj().T @ SU, basis.conj().T @ rhs)
    a = np.linalg.solve(M, Psi.conj().T @ b - W.conj().T @ y)
    assert n == b.shape[0]
    return Psi @ a + y


def schur_cg(H, eps, Phi, Psi, b, tol, kinetic, kappa, maxiter=500):
    """Preconditioned CG on S y = rhs in range(R) (preconditioner
    R diag(1/(kappa + |k+G|^2/2)) R, the kinetic one of the plain CG), then
    x = Psi a + y.  Stops at ||rhs - S y|| <= tol after at least one iteration.
    Returns (x, iterations, final recursive residual norm)."""
    R, M, W = _parts(H, eps, Phi, Psi)
    S, _ = schur_operator(H, eps, Phi, Psi)
    Minv = 1.0 / (kappa + kinetic)
    rhs = R(b) - W @ np.linalg.solve(M, Psi.conj().T @ b)
    y = np.zeros_like(b)
    r = rhs.copy()
    z = R(Minv * r)
    p = z.copy()
    rz = np.vdot(r, z).real
    it = 0
    rnorm = np.linalg.norm(r)
    while it < maxiter:
        Sp = S(p)
        alpha = rz / np.vdot(p, Sp).real
        y = y + alpha * p
        r = r - alpha * Sp
        it += 1
        rnorm = np.linalg.norm(r)
        if rnorm <= tol:
            break
        z = R(Minv * r)
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    y = R(y)
    a = np.linalg.solve(M, Psi.conj().T @ b - W.conj().T @ y)
    return Psi @ a + y, it, rnorm
