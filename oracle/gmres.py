"""GMRES for the Dyson equation: exact products, and Algorithm 1 (inexact
GMRES) with the adaptive Sternheimer tolerances.  Test infrastructure.

``gmres`` is textbook restarted GMRES(m) (Sec. 3.1: x_i = x_0 + V_i y_i with
y_i the minimiser of the small least-squares problem eq. small_ls), with
modified Gram-Schmidt Arnoldi and Givens rotations.

``inexact_gmres`` follows Algorithm 1 step by step: the first residual is
formed with an inexact product accurate to tau/3, step i uses the tolerance
s/(3m) * tau/||r~_{i-1}||, termination when ||r~_i|| <= tau/3, then a
restart with s = sigma_i(H_i) if s > sigma_i(H_i), and after m steps a
restart with s = sigma_m(H_m).  The per-Sternheimer CG tolerances come from
``cg_tolerances`` (Table strategies; k-form Table strategies_k).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import basis, dft, response, schur


# ------------------------------------------------------------ plain GMRES ---

def gmres(apply, b, x0=None, tol=1e-12, m=20, max_restarts=50):
    """Restarted GMRES(m) with exact products; absolute tolerance on ||b - A x||."""
    shape = b.shape
    b = b.ravel()
    x = np.zeros_like(b) if x0 is None else x0.ravel().copy()
    history = []
    for _ in range(max_restarts):
        r = b - apply(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        history.append(beta)
        if beta <= tol:
            break
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k_used = 0
        for i in range(m):
            w = apply(V[i].reshape(shape)).ravel()
            for j in range(i + 1):
                H[j, i] = V[j] @ w
                w = w - H[j, i] * V[j]
            H[i + 1, i] = np.linalg.norm(w)
            if H[i + 1, i] > 0:
                V[i + 1] = w / H[i + 1, i]
            for j in range(i):
                t = cs[j] * H[j, i] + sn[j] * H[j + 1, i]
                H[j + 1, i] = -sn[j] * H[j, i] + cs[j] * H[j + 1, i]
                H[j, i] = t
            rho = np.hypot(H[i, i], H[i + 1, i])
            cs[i], sn[i] = H[i, i] / rho, H[i + 1, i] / rho
            H[i, i] = rho
            H[i + 1, i] = 0.0
            g[i + 1] = -sn[i] * g[i]
            g[i] = cs[i] * g[i]
            k_used = i + 1
            if abs(g[i + 1]) <= tol:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
    return x.reshape(shape), history


# ---------------------------------------------------- Sternheimer by CG ---

def sternheimer_cg(H, eps_n, Phi, b, tol, kinetic, kappa, maxiter=500):
    """Preconditioned CG on A_n = Q(H - eps_n)Q, Q = 1 - Phi Phi^H, from x0 = 0,
    stopping at ||b - A x|| <= tol after at least one iteration (Sec. 4.1.2).
    Every iterate is re-projected onto range(Q) (Remark rmk:sternheimer_solution).
    Preconditioner: Q diag(1/(kappa + |k+G|^2/2)) (kinetic, diagonal in Fourier).
    Returns (x, iterations, final recursive residual norm)."""
    def Q(y):
        return y - Phi @ (Phi.conj().T @ y)

    def A(y):
        return Q(H @ y - eps_n * y)

    Minv = 1.0 / (kappa + kinetic)
    x = np.zeros_like(b)
    r = Q(b)
    z = Q(Minv * r)
    p = z.copy()
    rz = np.vdot(r, z).real
    it = 0
    rnorm = np.linalg.norm(r)
    while it < maxiter:
        Ap = A(p)
        alpha = rz / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        rnorm = np.linalg.norm(r)
        if rnorm <= tol:
            break
        z = Q(Minv * r)
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    return Q(x), it, rnorm


def chi0_inexact(gs, u, tolerances, kxc=None, schur_nbands=0):
    """chi0 u with dphi^Q from CG at the per-(n,k) tolerances (a dict or array
    indexed like ``systems(gs)``); same formula as response.chi0 otherwise.
    schur_nbands > 0: the Sternheimer equations in their Schur-complement form
    (Sec. 3.4.2, oracle/schur.py) with the bands N_occ,k + 1 .. schur_nbands as
    the extra computed bands.  Returns (chi0 u, number of Hamiltonian applications)."""
    dims, vol = gs.dims, gs.volume
    out = np.zeros(dims)
    nham = 0
    num = den = 0.0
    cache = []
    s = 0
    for kb in gs.kblocks:
        no = kb.nocc
        Phi = kb.vecs[:, :no]
        psi = dft.F_inv(Phi.T, kb.flat, dims, vol)
        y = dft.F(u[None] * psi, kb.flat, dims, vol)
        a = y @ Phi.conj()
        deps = a[np.arange(no), np.arange(no)].real
        kappa = np.einsum("gn,g,gn->n", Phi.conj(), kb.kinetic, Phi).real
        dphi = np.zeros((no, Phi.shape[0]), dtype=np.complex128)
        Psi = kb.vecs[:, no:schur_nbands] if schur_nbands > no else None
        for n in range(no):
            b = -(y[n] - Phi @ a[n])
            if Psi is not None:
                xq, it, _ = schur.schur_cg(kb.H, kb.eps[n], Phi, Psi, b, tolerances[s], kb.kinetic,
                                           max(1.0, kappa[n]))
            else:
                xq, it, _ = sternheimer_cg(kb.H, kb.eps[n], Phi, b, tolerances[s], kb.kinetic,
                                           max(1.0, kappa[n]))
            nham += it
            s += 1
            coef = np.zeros(no, dtype=np.complex128)
            for m in range(no):
                if m == n:
                    continue
                fn, fm = kb.f[n], kb.f[m]
                if fn * fn + fm * fm == 0.0:
                    continue
                d = response._delta_coeff(fn, fm, kb.eps[n], kb.eps[m], kb.fprime[n], kb.fprime[m])
                coef[m] = response.dphiP_coefficient(fn, fm, d) * a[n, m]
            dphi[n] = xq + Phi @ coef
        dpsi = dft.F_inv(dphi, kb.flat, dims, vol)
        out += kb.weight * np.einsum("n,nxyz->xyz", 2.0 * kb.f[:no], (psi.conj() * dpsi).real)
        num += kb.weight * float(np.dot(kb.fprime[:no], deps))
        den += kb.weight * float(kb.fprime[:no].sum())
        cache.append((psi, deps))
    deF = num / den if den != 0.0 else 0.0
    for kb, (psi, deps) in zip(gs.kblocks, cache):
        df = kb.fprime[:kb.nocc] * (deps - deF)
        out += kb.weight * np.einsum("n,nxyz->xyz", df, np.abs(psi) ** 2)
    return out, nham


def dielectric_inexact(gs, v, tol_fn, kxc=None, schur_nbands=0):
    """E~ v = v - ||Kv|| chi0~(Kv/||Kv||) with CG tolerances tol_fn(||Kv||)."""
    Kv = response.apply_K(v, gs, kxc)
    nrm = float(np.linalg.norm(Kv))
    if nrm == 0.0:
        return v.copy(), 0
    c, nham = chi0_inexact(gs, Kv / nrm, tol_fn(nrm), kxc, schur_nbands)
    return v - nrm * c, nham


def kernel_norm_bound(gs, kxc):
    """||K|| <= max_{G != 0} 4 pi/|G|^2 + max_r |K^xc(r)| (K^H and K^xc symmetric)."""
    G = basis.grid_G(gs.lattice, gs.dims)
    g2 = np.sum(G * G, axis=-1)
    return float(4.0 * np.pi / g2[g2 > 0].min() + np.abs(kxc).max())


def dielectric_adjoint_inexact(gs, v, tol_fn, kxc, knorm, schur_nbands=0):
    """E~^T v = v - ||v|| K chi0~(v/||v||) (the transpose of eq. op_discretised):
    the Sternheimer error enters through K after chi0, so the tolerances take
    ||K|| (its bound) where the forward application takes ||K v||."""
    nrm = float(np.linalg.norm(v))
    if nrm == 0.0:
        return v.copy(), 0
    c, nham = chi0_inexact(gs, v / nrm, tol_fn(knorm), kxc, schur_nbands)
    return v - nrm * response.apply_K(c, gs, kxc), nham


# ------------------------------------------------------------- strategies ---

def systems(gs):
    """(k index, band index) of every Sternheimer system, k-major."""
    return [(ik, n) for ik, kb in enumerate(gs.kblocks) for n in range(kb.nocc)]


def orbital_row_norm(gs, kb, real_part):
    """||F_k^{-1} Phi_k||_{2,inf} (or of its real part): the largest row norm.

    The real part is taken in the gauge in which each orbital is as real as
    possible (Sec. "Dropping the imaginary part of the orbitals": where a
    real representation exists the real part loses nothing).  Multiplying
    u_n by e^{-i theta} gives sum_r (Re)^2 = (sum |u|^2 + Re(e^{-2i theta}
    sum u^2))/2, largest at theta = arg(sum_r u_n(r)^2)/2; the result no
    longer depends on the phases the eigensolver returned."""
    psi = dft.F_inv(kb.vecs[:, :kb.nocc].T, kb.flat, gs.dims, gs.volume)
    if real_part:
        sq = (psi * psi).reshape(psi.shape[0], -1).sum(axis=1)
        theta = 0.5 * np.angle(sq)
        psi = (psi * np.exp(-1j * theta).reshape((-1,) + (1,) * (psi.ndim - 1))).real
    return float(np.sqrt((np.abs(psi) ** 2).sum(axis=0)).max())


def prefactors(gs, strategy, Kv_norm):
    """The prefactor pi_nk of the CG tolerance for each system.

    Gamma-point forms are Table strategies; with k-points Table strategies_k
    with N_occ,k * N_mp replaced by N_occ = sum_k N_occ,k (bal) and
    sqrt(N_occ,k) N_mp by sqrt(N_occ) (grt), as the paper does in App. F.
    'grt_exact' is the prefactor C_{i,nk} of Theorem inexact_gmres_dyson in its
    k-form (App. F), gaps and complex orbital norm kept.
    """
    vol, ng = gs.volume, gs.n_grid
    nocc_tot = sum(kb.nocc for kb in gs.kblocks)
    nmp = len(gs.kblocks)
    out = []
    for kb in gs.kblocks:
        if strategy == "grt":
            orb = orbital_row_norm(gs, kb, True)
        elif strategy == "grt_exact":
            orb = orbital_row_norm(gs, kb, False)
        for n in range(kb.nocc):
            f, w = kb.f[n], kb.weight
            if strategy == "agr":
                p = 1.0
            elif strategy == "bal":
                p = vol / (2.0 * f * w * nocc_tot * np.sqrt(ng))
            elif strategy == "grt":
                p = np.sqrt(vol) / (2.0 * f * w * np.sqrt(ng) * np.sqrt(nocc_tot) * Kv_norm * orb)
            elif strategy == "grt_exact":
                gapn = kb.eps[kb.nocc] - kb.eps[n]
                p = (np.sqrt(vol) * gapn /
                     (2.0 * f * w * Kv_norm * orb * nmp * np.sqrt(ng * kb.nocc)))
            else:
                raise ValueError(strategy)
            out.append(p)
    return np.array(out)


def cg_tolerances(gs, strategy, tau, i, m, s, rprev, Kv_norm, b_norm):
    """tau^CG_{i,nk} for GMRES step i (i = 0: the restart residual, C_{0,n} tau/3)."""
    nsys = sum(kb.nocc for kb in gs.kblocks)
    if strategy == "D10":
        return np.full(nsys, tau / 10.0)
    if strategy == "D100":
        return np.full(nsys, tau / 100.0)
    if strategy == "D10n":
        return np.full(nsys, tau / (10.0 * b_norm))
    pf = prefactors(gs, strategy, Kv_norm)
    if i == 0:
        return pf * tau / 3.0
    return pf * s / (3.0 * m) * tau / rprev


# -------------------------------------------------------------- Algorithm 1 ---

@dataclasses.dataclass
class InexactResult:
    x: np.ndarray
    estimated: list          # ||r~_i|| of every step, all cycles
    sigmas: list             # sigma_i(H_i) whenever computed
    nham: int                # Hamiltonian applications (= CG iterations)
    restarts: int
    steps: int               # GMRES steps (E applications, restart residuals excluded)
    converged: bool
    # data of the last cycle, for the checks of Lemmas inexact_residual_norm
    # and gmres_y_k_bound
    cycle_x0: np.ndarray = None
    cycle_err0: float = 0.0  # ||(E - E~(0)) x0||
    cycle_errs: list = None  # ||(E - E~(i)) v_i||, i = 1..k
    cycle_res: list = None   # ||r~_0|| = beta, ||r~_1||, ..., ||r~_k||
    cycle_y: np.ndarray = None
    cycle_H: np.ndarray = None


def inexact_gmres(gs, b, tau, m, strategy, x0=None, s=1.0, kxc=None,
                  max_restarts=20, track_errors=False, kerker_alpha=0.0, schur_nbands=0, adjoint=False):
    """Algorithm 1 with CG-solved Sternheimer equations (emulation on the CPU).

    kerker_alpha > 0: Algorithm 1 on the left-preconditioned system T E x = T b
    of eq. precond_dyson with the Kerker T of eq. kerker; the tolerance rules
    are unchanged (||T|| = 1, Lemma kerker_properties), the stopping rule and
    the reported residuals are those of T r, and b_norm stays ||b||.
    schur_nbands > 0: Schur-complement Sternheimer solves (see chi0_inexact).
    adjoint: Algorithm 1 on E^T lambda = b (dielectric_adjoint_inexact, the
    tolerance rules with ||K|| for ||K v_i||)."""
    if kxc is None:
        kxc = response.exchange_kernel(gs.rho)
    shape = b.shape
    b_norm = float(np.linalg.norm(b))

    def T(v):
        return response.kerker(v, gs.lattice, gs.dims, kerker_alpha) if kerker_alpha > 0 else v

    knorm = kernel_norm_bound(gs, kxc)

    def apply_E(v, tol_fn):
        if adjoint:
            return dielectric_adjoint_inexact(gs, v, tol_fn, kxc, knorm, schur_nbands)
        return dielectric_inexact(gs, v, tol_fn, kxc, schur_nbands)

    def exact_E(v):
        return response.dielectric_adjoint(gs, v, kxc) if adjoint else response.dielectric(gs, v, kxc)
    x0 = np.zeros_like(b) if x0 is None else x0.copy()
    est, sig = [], []
    nham = 0
    restarts = 0
    steps = 0
    while True:
        # Line 1: r~0 = b - E~(0) x0 with error <= tau/3 (free when x0 = 0)
        err0 = 0.0
        if np.linalg.norm(x0) > 0:
            def tol0(kvn):
                return cg_tolerances(gs, strategy, tau, 0, m, s, 1.0, kvn, b_norm)
            Ex0, nh = apply_E(x0, tol0)
            nham += nh
            if track_errors:
                err0 = float(np.linalg.norm(T(Ex0 - exact_E(x0))))
            r0 = T(b - Ex0)
        else:
            r0 = T(b)
        beta = float(np.linalg.norm(r0))
        V = [r0.ravel() / beta]
        H = np.zeros((m + 1, m))
        res = [beta]
        errs = []
        rprev = beta
        finished = False
        for i in range(1, m + 1):
            def toli(kvn, i=i, rprev=rprev):
                return cg_tolerances(gs, strategy, tau, i, m, s, rprev, kvn, b_norm)
            w, nh = apply_E(V[-1].reshape(shape), toli)
            nham += nh
            steps += 1
            if track_errors:
                errs.append(float(np.linalg.norm(T(w - exact_E(V[-1].reshape(shape))))))
            w = T(w).ravel()
            for j in range(i):                       # MGS Arnoldi
                H[j, i - 1] = V[j] @ w
                w = w - H[j, i - 1] * V[j]
            H[i, i - 1] = np.linalg.norm(w)
            V.append(w / H[i, i - 1] if H[i, i - 1] > 0 else w)
            Hi = H[:i + 1, :i]
            e1 = np.zeros(i + 1)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hi, e1, rcond=None)
            rnorm = float(np.linalg.norm(e1 - Hi @ y))
            est.append(rnorm)
            res.append(rnorm)
            rprev = rnorm
            if rnorm <= tau / 3.0 or i == m:
                sigma = float(np.linalg.svd(Hi, compute_uv=False)[-1])
                sig.append(sigma)
                x = x0 + (np.array(V[:i]).T @ y).reshape(shape)
                result = InexactResult(x, est, sig, nham, restarts, steps, False,
                                       x0, err0, errs, res, y, Hi.copy())
                if rnorm <= tau / 3.0 and s <= sigma:
                    result.converged = True
                    return result
                s = sigma                 # restart (line s_update, or after m steps)
                x0 = x
                restarts += 1
                finished = True
                break
        assert finished
        if restarts > max_restarts:
            return result
