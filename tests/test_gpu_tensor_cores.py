"""Tensor-core projection coefficients (tcgen05 kind::tf32, three-term split).

<phi_m, y_s> on the tensor cores against the CUDA-core kernels and against
numpy on the same FP32 inputs, the known answer <phi_m, phi_n> = delta_mn, and
the mixed-precision Dyson solve with the tensor-core projections reaching tau."""
import numpy as np
import pytest

import gpu_common
from gpu_common import context, dev, oracle_state, system, torch

pytestmark = pytest.mark.gpu


def _orbitals(ctx, name):
    _, vecs = gpu_common.dense_eigenpairs(ctx, ctx.nbands)
    return vecs


@pytest.mark.parametrize("name,nvec", [("tiny_insulator", 3), ("tiny_metal", 24), ("tiny_kb", 40)])
def test_tensor_core_coefficients_match_cuda_cores(name, nvec):
    ctx = context(name)
    rng = np.random.default_rng(7)
    vecs = _orbitals(ctx, name)
    for k in range(len(vecs)):
        nb = ctx.basis_size(k)
        y = (rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb))).astype(np.complex64)
        yt = torch.tensor(y, device="cuda")
        c0 = ctx.projection_coefficients(k, yt, method=0)
        c1 = ctx.projection_coefficients(k, yt, method=1)
        # rows of vecs[k] are the orbitals; the library holds their complex64 rounding
        phi = vecs[k].cpu().numpy()[:c0.shape[1]].astype(np.complex64).astype(np.complex128)
        ref = y.astype(np.complex128) @ phi.conj().T
        scale = np.abs(ref).max()
        assert np.abs(c0 - ref).max() < 2e-6 * scale * np.sqrt(nb)
        assert np.abs(c1 - ref).max() < 2e-6 * scale * np.sqrt(nb)
        assert np.abs(c1 - c0).max() < 2e-6 * scale * np.sqrt(nb)


@pytest.mark.parametrize("name,nvec", [("tiny_insulator", 3), ("tiny_metal", 24), ("tiny_kb", 40)])
def test_tensor_core_projection_matches_cuda_cores(name, nvec):
    ctx = context(name)
    rng = np.random.default_rng(8)
    vecs = _orbitals(ctx, name)
    for k in range(len(vecs)):
        nb = ctx.basis_size(k)
        y = (rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb))).astype(np.complex64)
        q0 = ctx.project_out(k, torch.tensor(y, device="cuda"), method=0).cpu().numpy()
        q1 = ctx.project_out(k, torch.tensor(y, device="cuda"), method=1).cpu().numpy()
        nocc = ctx.projection_coefficients(k, torch.tensor(y, device="cuda"), method=0).shape[1]
        phi = vecs[k].cpu().numpy()[:nocc].astype(np.complex64).astype(np.complex128)
        ref = y - (y.astype(np.complex128) @ phi.conj().T) @ phi
        scale = np.abs(y).max()
        assert np.abs(q0 - ref).max() < 1e-5 * scale
        assert np.abs(q1 - ref).max() < 1e-5 * scale
        assert np.abs(q1.astype(np.complex128) @ phi.conj().T).max() < 1e-5 * scale * np.sqrt(nb)


def test_tensor_core_coefficients_of_the_orbitals_are_the_identity():
    ctx = context("tiny_metal")
    vecs = _orbitals(ctx, "tiny_metal")
    for k in range(len(vecs)):
        c = ctx.projection_coefficients(k, vecs[k].to(torch.complex64).contiguous(), method=1)
        n = c.shape[1]
        assert np.abs(c[:n, :n] - np.eye(n)).max() < 1e-5


def test_tensor_core_projections_in_the_mixed_solve():
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = system("tiny_metal"), oracle_state("tiny_metal"), context("tiny_metal")
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    ctx.set_tensor_cores(True)
    try:
        x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    finally:
        ctx.set_tensor_cores(False)
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))) <= 1e-8


def test_tensor_cores_with_schur_sets_in_chi0():
    """The Schur-complement solves project on [Phi Psi] and Psi: with the tensor
    cores on, the mixed-precision chi0 of the metal still matches the oracle."""
    from oracle import response
    from workloads import perturbation
    s, gs = system("tiny_metal"), oracle_state("tiny_metal")
    from paper_2505_02319_gb300 import groundstate
    ctx = gpu_common.dense_context_for(s, schur=True)
    ctx.set_tensor_cores(True)
    dV = perturbation(s)
    nsys = ctx.groundstate_nsys
    from paper_2505_02319_gb300 import ikr
    d, _ = ctx.apply_chi0(dev(dV), tol=np.full(nsys, 1e-11), precision=ikr.MIXED)
    ref = response.chi0(gs, dV)
    assert np.linalg.norm(d.cpu().numpy() - ref.ravel()) < 1e-9 * np.linalg.norm(ref)
    ctx.destroy()


def test_tensor_core_nonlocal_projectors():
    """The Kleinman-Bylander term B diag(D) B^H of H_k runs on the projection
    kernels with the projectors as the vector set: in FP32 on the CUDA cores and
    on the tensor cores (tcgen05, three-term TF32 split) it matches the oracle's
    dense H_k to the FP32 tolerance of the other H_k tests."""
    from paper_2505_02319_gb300 import ikr
    gs, ctx = oracle_state("tiny_kb"), context("tiny_kb")
    rng = np.random.default_rng(29)
    for k, kb in enumerate(gs.kblocks):
        nb = len(kb.eps)
        psi = (rng.normal(size=(5, nb)) + 1j * rng.normal(size=(5, nb))).astype(np.complex64)
        ref = psi.astype(np.complex128) @ kb.H.T
        outs = []
        for tc in (False, True):
            ctx.set_tensor_cores(tc)
            try:
                outs.append(ctx.apply_hamiltonian(k, torch.tensor(psi, device="cuda"), precision=ikr.MIXED)
                            .cpu().numpy())
            finally:
                ctx.set_tensor_cores(False)
        for out in outs:
            assert np.linalg.norm(out - ref) < 2e-6 * np.linalg.norm(ref), k
