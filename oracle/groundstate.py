"""Dense ground state of the synthetic systems.  Test infrastructure.

The paper obtains its ground states from a DFTK SCF (Sec. 4.1.2), which is out
of scope here; the synthetic systems use a fixed local potential V and the
eigenpairs of the discretised k-point Hamiltonian (eq. Hamiltonian with the
k-form of Sec. 4.1.1)

    H_k = diag(|k+G|^2 / 2) + Z^T W diag(V) W^{-1} Z      on the sphere G_k,

(plus the nonlocal B diag(D) B^H of oracle/kb.py for systems with
Kleinman-Bylander projectors),

obtained by dense diagonalisation.  Because W is the unitary DFT, the local
part has the plain closed form (W diag(V) W^{-1})_{G,G'} = Vhat(G - G') / Ng
with Vhat(q) = sum_r V(r) e^{-i q.r}, the difference G - G' taken modulo the
grid.  Occupations follow eq. density with the Fermi-Dirac function
f(x) = 2/(1+e^x) and the Fermi level fixed by sum_k w_k sum_n f_nk = N; for
T = 0 ("insulator") the lowest N/2 bands of every k-point carry f = 2.
N_occ,k = max{n : f_nk > eps_occ} (Sec. 2.2) with eps_occ = 1e-10 (the
paper leaves eps_occ unspecified).
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.special import expit

from . import basis, dft, kb as kbproj

EPS_OCC = 1e-10


@dataclasses.dataclass
class KBlock:
    kfrac: np.ndarray
    weight: float
    miller: np.ndarray      # (Nb,3)
    flat: np.ndarray        # (Nb,) flat grid index
    kinetic: np.ndarray     # (Nb,) |k+G|^2/2
    H: np.ndarray           # (Nb,Nb) dense Hamiltonian
    eps: np.ndarray         # all eigenvalues (ascending)
    vecs: np.ndarray        # all eigenvectors (columns)
    f: np.ndarray = None
    fprime: np.ndarray = None
    nocc: int = 0


@dataclasses.dataclass
class GroundState:
    lattice: np.ndarray
    dims: tuple
    volume: float
    Ecut: float
    V: np.ndarray
    temperature: float
    n_electrons: int
    kblocks: list
    eF: float
    rho: np.ndarray

    @property
    def n_grid(self):
        return int(np.prod(self.dims))


def local_potential_matrix(V: np.ndarray, miller: np.ndarray, dims) -> np.ndarray:
    """Z^T W diag(V) W^{-1} Z on the sphere: entries Vhat(G-G')/Ng."""
    ng = int(np.prod(dims))
    Vhat = dft.grid_analysis(V) / ng
    d = miller[:, None, :] - miller[None, :, :]
    pos = np.mod(d, np.array(dims))
    return Vhat[pos[..., 0], pos[..., 1], pos[..., 2]]


def hamiltonian(lattice, dims, Ecut, kfrac, V, kb=None):
    """Dense H_k; kb = (centres, sigma, D) adds the nonlocal B diag(D) B^H."""
    miller, flat, kin = basis.sphere(lattice, dims, Ecut, kfrac)
    H = local_potential_matrix(V, miller, dims)
    H[np.diag_indices_from(H)] += kin
    if kb is not None:
        H = H + kbproj.nonlocal_matrix(lattice, miller, kfrac, *kb)
    return miller, flat, kin, H


def fermi_dirac(x):
    """f(x) = 2 / (1 + e^x)."""
    return 2.0 * expit(-x)


def fermi_dirac_derivative(x):
    """f'(x) = -2 e^x / (1+e^x)^2."""
    return -2.0 * expit(x) * expit(-x)


def fermi_level(eps_list, weights, n_electrons, T):
    """Bisection on sum_k w_k sum_n f((eps_nk - eF)/T) = N (Sec. 2.1)."""
    lo = min(e.min() for e in eps_list) - 50 * T - 1.0
    hi = max(e.max() for e in eps_list) + 50 * T + 1.0

    def count(eF):
        return sum(w * fermi_dirac((e - eF) / T).sum() for e, w in zip(eps_list, weights))

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def occupations(eps_list, weights, n_electrons, T):
    """Returns (f list, f' list, eF).  f'_n = (1/T) f'((eps_n - eF)/T) (eq. fprime)."""
    if T == 0.0:
        nb = n_electrons // 2
        fs = [np.where(np.arange(len(e)) < nb, 2.0, 0.0) for e in eps_list]
        fps = [np.zeros(len(e)) for e in eps_list]
        homo = max(e[nb - 1] for e in eps_list)
        lumo = min(e[nb] for e in eps_list)
        return fs, fps, 0.5 * (homo + lumo)
    eF = fermi_level(eps_list, weights, n_electrons, T)
    fs = [fermi_dirac((e - eF) / T) for e in eps_list]
    fps = [fermi_dirac_derivative((e - eF) / T) / T for e in eps_list]
    return fs, fps, eF


def density(gs_kblocks, dims, volume):
    """rho = sum_k w_k sum_{n <= Nocc_k} f_nk |F_k^{-1} phi_nk|^2 (eq. discretised_KS)."""
    rho = np.zeros(dims)
    for kb in gs_kblocks:
        psi = dft.F_inv(kb.vecs[:, :kb.nocc].T, kb.flat, dims, volume)
        rho += kb.weight * np.einsum("n,nxyz->xyz", kb.f[:kb.nocc], np.abs(psi) ** 2)
    return rho


def solve(system, V=None) -> GroundState:
    """Dense ground state of a workloads.System (optionally with a replaced V)."""
    V = system.V if V is None else V
    lattice, dims = system.lattice, tuple(system.dims)
    volume = float(abs(np.linalg.det(lattice)))
    blocks = []
    kb = None
    if getattr(system, "kb_centers", None) is not None:
        kb = (system.kb_centers, system.kb_sigma, system.kb_D)
    for kf, w in zip(system.kpoints, system.kweights):
        miller, flat, kin, H = hamiltonian(lattice, dims, system.Ecut, kf, V, kb)
        eps, vecs = np.linalg.eigh(H)
        blocks.append(KBlock(kfrac=np.array(kf), weight=float(w), miller=miller, flat=flat,
                             kinetic=kin, H=H, eps=eps, vecs=vecs))
    fs, fps, eF = occupations([b.eps for b in blocks], [b.weight for b in blocks],
                              system.n_electrons, system.temperature)
    for b, f, fp in zip(blocks, fs, fps):
        b.f, b.fprime = f, fp
        b.nocc = int(np.max(np.nonzero(f > EPS_OCC)[0]) + 1)
    rho = density(blocks, dims, volume)
    return GroundState(lattice=lattice, dims=dims, volume=volume, Ecut=system.Ecut, V=V,
                       temperature=system.temperature, n_electrons=system.n_electrons,
                       kblocks=blocks, eF=eF, rho=rho)


def gap(gs: GroundState) -> float:
    """min_k (eps_{Nocc+1,k} - eps_{Nocc,k}) (the Sternheimer gap of Lemma cgtol_E)."""
    return min(b.eps[b.nocc] - b.eps[b.nocc - 1] for b in gs.kblocks)
