"""Kleinman-Bylander nonlocal projectors on the GPU (ikr_set_nonlocal): the
FP32 H_k against the oracle's dense H_k with B diag(D) B^H, the GPU
eigensolver on a system with projectors against the oracle's eigenvalues, and
the mixed-precision Dyson solve (whose CG adds <p, V_nl p> to <p, Ap>)
against the oracle's E.  The FP64 H_k, density and chi0 parity of the same
system run in test_gpu_parity.py (tiny_kb)."""
import numpy as np
import pytest

from gpu_common import context, dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu


def test_kb_hamiltonian_fp32():
    from paper_2505_02319_gb300 import ikr
    gs, ctx = oracle_state("tiny_kb"), context("tiny_kb")
    rng = np.random.default_rng(3)
    for k, kb in enumerate(gs.kblocks):
        nb = len(kb.eps)
        psi = (rng.normal(size=(3, nb)) + 1j * rng.normal(size=(3, nb))).astype(np.complex64)
        out = ctx.apply_hamiltonian(k, torch.tensor(psi, device="cuda"), precision=ikr.MIXED).cpu().numpy()
        assert rel(out, (kb.H @ psi.T.astype(np.complex128)).T) < 2e-6


def test_kb_eigensolver_matches_oracle():
    from paper_2505_02319_gb300 import groundstate
    s, gs = system("tiny_kb"), oracle_state("tiny_kb")
    ctx = groundstate.context_for(s, eig_tol=1e-11)
    for k, kb in enumerate(gs.kblocks):
        assert np.max(np.abs(ctx.eigenvalues[k] - kb.eps[:ctx.nbands])) < 1e-10


def test_kb_mixed_solve_reaches_tau():
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = system("tiny_kb"), oracle_state("tiny_kb"), context("tiny_kb")
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))) <= 1e-8


def test_kb_noalloc_rejected():
    from paper_2505_02319_gb300 import ikr
    ctx = context("tiny_kb")
    psi = torch.zeros((1, ctx.basis_size(0)), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    import ctypes as ct
    st = ikr._LIB.ikr_apply_hamiltonian_noalloc(ctx._h, 0, ct.c_void_p(psi.data_ptr()), ct.c_void_p(out.data_ptr()), 1,
                                                ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == ikr.IKR_ERR_ARG
