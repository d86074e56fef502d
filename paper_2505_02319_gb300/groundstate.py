"""Ground state for the response solver from the library's own eigensolver.

The response method takes the ground state (eq. discretised_KS) as its input;
the paper obtains it from an SCF, which is out of scope here.  For the fixed
synthetic potentials the ground state comes from the library's GPU eigensolver
(ikr_compute_eigenpairs: Chebyshev-filtered subspace iteration on its own H_k
applications, any basis size), or from eigenpairs a caller supplies (for
instance its own SCF).  This is setup, outside the solver.
"""
from __future__ import annotations

import numpy as np

from . import ikr


def context_for(system, nbands=None, eig_tol=1e-10, schur=False, eigenpairs=None) -> ikr.Context:
    """Context with ground state for a workloads.System.  The eigenpairs come
    from the library's GPU eigensolver to residual ``eig_tol`` (Ha), or from
    ``eigenpairs(ctx, nbands) -> (eigenvalues (nk, nbands), [per k-point a
    (nbands, Nb_k) complex128 CUDA tensor, row n = band n])`` when given.  ``schur``: Schur-complement Sternheimer
    solves over the bands above N_occ,k."""
    ctx = ikr.Context.setup_groundstate(system.lattice, system.dims, system.Ecut, system.kpoints,
                                        system.kweights, system.V, system.temperature,
                                        system.n_electrons)
    nb = nbands or system.nbands
    if getattr(system, "kb_centers", None) is not None:
        ctx.set_nonlocal(system.kb_centers, system.kb_sigma, system.kb_D)
    if eigenpairs is None:
        ctx.compute_eigenpairs(nb, tol=eig_tol)
    else:
        ev, vecs = eigenpairs(ctx, nb)
        ctx.set_eigenpairs(ev, vecs)
    ctx.nbands = nb
    ctx.ngrid = int(np.prod(system.dims))
    ctx.groundstate_nsys = int(ctx.groundstate_info(nb, ctx.ngrid)["nocc"].sum())
    if schur:
        ctx.set_schur(True)
    return ctx
