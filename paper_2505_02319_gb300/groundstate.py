"""Ground state for the response solver from the library's own H_k.

The response method takes the ground state (eq. discretised_KS) as its input;
the paper obtains it from an SCF, which is out of scope here.  For the fixed
synthetic potentials the ground state comes either from the library's GPU
eigensolver (ikr_compute_eigenpairs: Chebyshev-filtered subspace iteration on
its own H_k applications, any basis size) or, for small bases, from every
H_k assembled column by column from ikr_apply_hamiltonian and diagonalised
densely (torch.linalg.eigh).  This is setup, outside the solver.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ikr


def dense_eigenpairs(ctx: ikr.Context, nbands: int, batch: int = 512):
    """Lowest ``nbands`` eigenpairs of every H_k: (eigenvalues (nk, nbands)
    float64 numpy, list of (nbands, Nb_k) complex128 CUDA tensors)."""
    evals, evecs = [], []
    for k in range(ctx.nkpt):
        nb = ctx.basis_size(k)
        cols = torch.empty((nb, nb), dtype=torch.complex128, device="cuda")
        for j0 in range(0, nb, batch):
            jb = min(batch, nb - j0)
            e = torch.zeros((jb, nb), dtype=torch.complex128, device="cuda")
            e[torch.arange(jb), j0 + torch.arange(jb)] = 1.0
            cols[j0:j0 + jb] = ctx.apply_hamiltonian(k, e)     # row j = H e_j
        H = cols.transpose(0, 1)
        H = 0.5 * (H + H.conj().transpose(0, 1))
        w, v = torch.linalg.eigh(H)
        evals.append(w[:nbands].cpu().numpy())
        evecs.append(v[:, :nbands].transpose(0, 1).contiguous())
        del cols, H, w, v
    return np.array(evals), evecs


def context_for(system, nbands=None, eigensolver="dense", eig_tol=1e-10, schur=False) -> ikr.Context:
    """Context with ground state for a workloads.System.  ``eigensolver``:
    "dense" (H_k assembled and diagonalised, small bases) or "chfsi" (the
    library's GPU Chebyshev-filtered subspace iteration, any basis size).
    ``schur``: Schur-complement Sternheimer solves over the bands above N_occ,k."""
    ctx = ikr.Context.setup_groundstate(system.lattice, system.dims, system.Ecut, system.kpoints,
                                        system.kweights, system.V, system.temperature,
                                        system.n_electrons)
    nb = nbands or system.nbands
    if getattr(system, "kb_centers", None) is not None:
        ctx.set_nonlocal(system.kb_centers, system.kb_sigma, system.kb_D)
    if eigensolver == "chfsi":
        ctx.compute_eigenpairs(nb, tol=eig_tol)
    elif eigensolver == "dense":
        ev, vecs = dense_eigenpairs(ctx, nb)
        ctx.set_eigenpairs(ev, vecs)
    else:
        raise ValueError(f"unknown eigensolver {eigensolver!r}")
    ctx.nbands = nb
    ctx.ngrid = int(np.prod(system.dims))
    ctx.groundstate_nsys = int(ctx.groundstate_info(nb, ctx.ngrid)["nocc"].sum())
    if schur:
        ctx.set_schur(True)
    return ctx
