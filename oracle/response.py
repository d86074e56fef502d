"""Exact chi0, K^Hxc, Kerker and the dielectric adjoint E.  Test infrastructure.

All densities/potentials are real vectors of grid values (Sec. 2.3.2); norms
are the plain (unweighted) l2 norms of those vectors, as in eq. op_discretised.
"""
from __future__ import annotations

import numpy as np

from . import basis, dft

RHO_MIN = 1e-10          # below this density the exchange kernel is set to 0
DEGENERATE = 1e-10       # |eps_n - eps_m| below which the f' limit is taken


# ----------------------------------------------------------------- kernels ---

def hartree(v: np.ndarray, lattice, dims) -> np.ndarray:
    """K^H v = W^{-1} diag(4 pi/|G|^2, G=0 -> 0) W v  (Sec. 3.4.3: diagonal in
    the plane-wave basis with the G = 0 entry zero)."""
    G = basis.grid_G(lattice, dims)
    G2 = np.einsum("...i,...i->...", G, G)
    kern = np.zeros_like(G2)
    nz = G2 > 0
    kern[nz] = 4.0 * np.pi / G2[nz]
    vh = dft.grid_analysis(v)
    return (dft.grid_synthesis(kern * vh) / v.size).real


def exchange_kernel(rho: np.ndarray) -> np.ndarray:
    """LDA (Slater) exchange kernel of a spin-paired density:
    V_x = -(3 rho / pi)^{1/3},  K_x = dV_x/drho = -(1/3)(3/pi)^{1/3} rho^{-2/3};
    set to 0 where rho < RHO_MIN (reading A8)."""
    out = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    out[ok] = -(1.0 / 3.0) * (3.0 / np.pi) ** (1.0 / 3.0) * rho[ok] ** (-2.0 / 3.0)
    return out


def exchange_potential(rho: np.ndarray) -> np.ndarray:
    return -(3.0 * np.maximum(rho, 0.0) / np.pi) ** (1.0 / 3.0)


def apply_K(v, gs, kxc=None):
    """K = K^H + K^xc, K^xc acting pointwise in real space (Sec. 2.2)."""
    if kxc is None:
        kxc = exchange_kernel(gs.rho)
    return hartree(v, gs.lattice, gs.dims) + kxc * v


def kerker(v: np.ndarray, lattice, dims, alpha: float) -> np.ndarray:
    """T v with T = W^{-1} (D + (1 - D_11) e1 e1^T) W, D = |G|^2/(|G|^2 + alpha^2):
    the charge-conserving Kerker preconditioner of eq. kerker in the form the
    proof of Lemma kerker_properties reduces it to."""
    G = basis.grid_G(lattice, dims)
    G2 = np.einsum("...i,...i->...", G, G)
    D = G2 / (G2 + alpha * alpha)
    D[0, 0, 0] = 1.0
    return (dft.grid_synthesis(D * dft.grid_analysis(v)) / v.size).real


# -------------------------------------------------------------------- chi0 ---

def _delta_coeff(fn, fm, en, em, fpn, fpm):
    """(f_n - f_m)/(eps_n - eps_m), with the derivative limit for degenerate pairs
    (eq. fprime reading A3: the mean of f'_n and f'_m)."""
    if abs(en - em) < DEGENERATE:
        return 0.5 * (fpn + fpm)
    return (fn - fm) / (en - em)


def dphiP_coefficient(fn, fm, delta):
    """c_nm of dphi^P_n = sum_m c_nm <phi_m, dV phi_n> phi_m (reading A1):
    f_n/(f_n^2+f_m^2) * (f_n-f_m)/(eps_n-eps_m)."""
    return fn / (fn * fn + fm * fm) * delta


def chi0(gs, dV: np.ndarray, return_parts: bool = False):
    """chi0 dV of eq. kchi0 (eq. chi0 for a single k-point):

      sum_k w_k sum_{n<=Nocc_k} 2 f_nk Re(conj(F^-1 phi_nk) . F^-1 dphi_nk)
                                 + df_nk |F^-1 phi_nk|^2,

    dphi = dphi^P + dphi^Q with
      * dphi^Q_n = A_n^+ b_n, b_n = -Q F(dV . F^-1 phi_n), A_n = Q(H - eps_n)Q,
        A_n^+ = Phi_perp D_n^{-1} Phi_perp^H from the full eigendecomposition
        (proof of Lemma cgtol_E; the unique solution in range(Q));
      * dphi^P_n = sum_{m<=Nocc, m != n} c_nm <phi_m, dV phi_n> phi_m with
        c_nm = f_n/(f_n^2+f_m^2) (f_n-f_m)/(eps_n-eps_m)  (eq. delta_phi_P as
        read in A1/A2: the printed coefficient carries one more factor f_n,
        which belongs to the f_n in eq. chi0; the m = n term is left to df_n);
      * df_n = f'_n (deps_n - deps_F), deps_n = <phi_n, dV phi_n>, and deps_F
        fixed by sum_k w_k sum_n df_nk = 0 (eq. delta_f; deps_F = 0 when
        sum w f' = 0).
    """
    dims, vol = gs.dims, gs.volume
    out = np.zeros(dims)
    parts = []
    num = 0.0
    den = 0.0
    for kb in gs.kblocks:
        no = kb.nocc
        psi = dft.F_inv(kb.vecs[:, :no].T, kb.flat, dims, vol)              # (no, grid)
        y = dft.F(dV[None] * psi, kb.flat, dims, vol)                       # (no, Nb)
        a = y @ kb.vecs.conj()          # a[n, m] = <phi_m, y_n> = <phi_m, dV phi_n>
        deps = a[np.arange(no), np.arange(no)].real
        e = kb.eps
        dphi = np.zeros((no, kb.vecs.shape[0]), dtype=np.complex128)
        for n in range(no):
            # Q part: sum over unoccupied eigenvectors m > Nocc of (-a_m)/(eps_m - eps_n)
            coef = np.zeros(kb.vecs.shape[1], dtype=np.complex128)
            coef[no:] = -a[n, no:] / (e[no:] - e[n])
            # P part
            for m in range(no):
                if m == n:
                    continue
                fn, fm = kb.f[n], kb.f[m]
                if fn * fn + fm * fm == 0.0:
                    continue
                d = _delta_coeff(fn, fm, e[n], e[m], kb.fprime[n], kb.fprime[m])
                coef[m] = dphiP_coefficient(fn, fm, d) * a[n, m]
            dphi[n] = kb.vecs @ coef
        dpsi = dft.F_inv(dphi, kb.flat, dims, vol)
        out += kb.weight * np.einsum("n,nxyz->xyz", 2.0 * kb.f[:no],
                                     (psi.conj() * dpsi).real)
        num += kb.weight * float(np.dot(kb.fprime[:no], deps))
        den += kb.weight * float(kb.fprime[:no].sum())
        parts.append((psi, deps, dphi))
    deF = num / den if den != 0.0 else 0.0
    for kb, (psi, deps, _) in zip(gs.kblocks, parts):
        df = kb.fprime[:kb.nocc] * (deps - deF)
        out += kb.weight * np.einsum("n,nxyz->xyz", df, np.abs(psi) ** 2)
    if return_parts:
        return out, dict(deF=deF, parts=parts)
    return out


def dielectric(gs, v: np.ndarray, kxc=None) -> np.ndarray:
    """E v = v - ||K v|| chi0(K v / ||K v||)  (eq. op_discretised, reading A4)."""
    Kv = apply_K(v, gs, kxc)
    nrm = float(np.linalg.norm(Kv))
    if nrm == 0.0:
        return v.copy()
    return v - nrm * chi0(gs, Kv / nrm)


def dielectric_adjoint(gs, v: np.ndarray, kxc=None) -> np.ndarray:
    """E^T v = v - K chi0 v: the dielectric operator, the transpose of E = 1 - chi0 K
    for symmetric chi0 and K (Sec. 2.2)."""
    return v - apply_K(chi0(gs, v), gs, kxc)


def dense_operator(apply, dims) -> np.ndarray:
    """Columns apply(e_j) for every grid point (tiny grids only)."""
    ng = int(np.prod(dims))
    M = np.zeros((ng, ng))
    for j in range(ng):
        e = np.zeros(ng)
        e[j] = 1.0
        M[:, j] = apply(e.reshape(dims)).ravel()
    return M
