"""Shared helpers of the GPU parity tests (systems, contexts, oracle states)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def system(name):
    from workloads import make_system
    return make_system(name)


@functools.lru_cache(maxsize=None)
def oracle_state(name):
    from oracle import groundstate
    return groundstate.solve(system(name))


def dense_eigenpairs(ctx, nbands, batch=512):
    """Test-side cross-check of the ground state: every H_k assembled column by
    column from the library's ikr_apply_hamiltonian and diagonalised densely
    (torch.linalg.eigh).  Returns (eigenvalues (nk, nbands) numpy, list of
    (nbands, Nb_k) complex128 CUDA tensors)."""
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


def dense_context_for(s, **kw):
    """A context whose ground state is the dense diagonalisation (exact to
    rounding, as the oracle's), for the parity tests at 1e-10."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import groundstate
    return groundstate.context_for(s, eigenpairs=dense_eigenpairs, **kw)


@functools.lru_cache(maxsize=None)
def context(name):
    return dense_context_for(system(name))


def dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
