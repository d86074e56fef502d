"""Tensor-core projection coefficients (tcgen05 kind::f16, every FP32 operand
split exactly into three bf16 pieces, six products per step).

<phi_m, y_s> on the tensor cores against the CUDA-core kernels and against
numpy on the same FP32 inputs (as accurate as the FP32 CUDA-core products), the
known answer <phi_m, phi_n> = delta_mn, in both operand layouts, and the
mixed-precision Dyson solve with the tensor-core projections reaching tau with
the CUDA-core solve's work."""
import numpy as np
import pytest

import gpu_common
from gpu_common import context, dev, oracle_state, system, torch

pytestmark = pytest.mark.gpu


def _orbitals(ctx, name):
    _, vecs = gpu_common.dense_eigenpairs(ctx, ctx.nbands)
    return vecs


# nvec 3 and 24: one 32-system tile; 40: 64 systems; 100: 128 systems; 150: two 128-system tiles;
# cfg2: 2 Nb_k ~ 6,000 reals, several split-K chunks per k-point
@pytest.mark.parametrize("name,nvec", [("tiny_insulator", 3), ("tiny_metal", 24), ("tiny_kb", 40),
                                       ("tiny_metal", 100), ("tiny_kb", 150), ("cfg2", 40)])
def test_tensor_core_coefficients_match_cuda_cores(name, nvec):
    ctx = context(name)
    rng = np.random.default_rng(7)
    vecs = _orbitals(ctx, name)
    for k in range(len(vecs)):
        nb = ctx.basis_size(k)
        y = (rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb))).astype(np.complex64)
        yt = torch.tensor(y, device="cuda")
        c0 = ctx.projection_coefficients(k, yt, method=0)
        # rows of vecs[k] are the orbitals; the library holds their complex64 rounding
        phi = vecs[k].cpu().numpy()[:c0.shape[1]].astype(np.complex64).astype(np.complex128)
        ref = y.astype(np.complex128) @ phi.conj().T
        scale = np.abs(ref).max()
        e0 = np.abs(c0 - ref).max()
        assert e0 < 2e-6 * scale * np.sqrt(nb)
        for method in (1, 2):   # swizzled and canonical operand layouts
            e1 = np.abs(ctx.projection_coefficients(k, yt, method=method) - ref).max()
            # the three-piece split makes the products FP32-exact: the tensor cores are as
            # accurate as the CUDA cores (a two-piece TF32 split is ~50x worse here)
            assert e1 < 4 * e0 + 1e-9 * scale, (method, e1, e0)


# nvec 3 and 24: one 32-system tile; 40: 64 systems; 100: 128 systems; 150: two 128-system tiles
@pytest.mark.parametrize("name,nvec", [("tiny_insulator", 3), ("tiny_metal", 24), ("tiny_kb", 40),
                                       ("tiny_metal", 100), ("tiny_kb", 150)])
def test_tensor_core_projection_matches_cuda_cores(name, nvec):
    ctx = context(name)
    rng = np.random.default_rng(8)
    vecs = _orbitals(ctx, name)
    for k in range(len(vecs)):
        nb = ctx.basis_size(k)
        y = (rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb))).astype(np.complex64)
        q0 = ctx.project_out(k, torch.tensor(y, device="cuda"), method=0).cpu().numpy()
        nocc = ctx.projection_coefficients(k, torch.tensor(y, device="cuda"), method=0).shape[1]
        phi = vecs[k].cpu().numpy()[:nocc].astype(np.complex64).astype(np.complex128)
        ref = y - (y.astype(np.complex128) @ phi.conj().T) @ phi
        scale = np.abs(y).max()
        e0 = np.abs(q0 - ref).max()
        assert e0 < 1e-5 * scale
        for method in (1, 2):
            q1 = ctx.project_out(k, torch.tensor(y, device="cuda"), method=method).cpu().numpy()
            e1 = np.abs(q1 - ref).max()
            # FP32 rounding level (the tensor cores' accumulation order differs); the precision
            # of the products themselves is checked on the coefficients above
            assert e1 < 8 * e0 + 1e-7 * scale, (method, e1, e0)
            assert np.abs(q1.astype(np.complex128) @ phi.conj().T).max() < 1e-5 * scale * np.sqrt(nb)


def test_tensor_core_coefficients_of_the_orbitals_are_the_identity():
    ctx = context("tiny_metal")
    vecs = _orbitals(ctx, "tiny_metal")
    for k in range(len(vecs)):
        for method in (1, 2):
            c = ctx.projection_coefficients(k, vecs[k].to(torch.complex64).contiguous(), method=method)
            n = c.shape[1]
            assert np.abs(c[:n, :n] - np.eye(n)).max() < 1e-6


def test_tensor_core_projections_in_the_mixed_solve():
    """The mixed solve with the tensor-core projections reaches tau and needs the
    CUDA-core solve's Hamiltonian applications to within 2 % (the products are
    FP32-accurate, so only rounding order differs)."""
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = system("tiny_metal"), oracle_state("tiny_metal"), context("tiny_metal")
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    _, rep0 = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    ctx.set_tensor_cores(True)
    try:
        x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    finally:
        ctx.set_tensor_cores(False)
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))) <= 1e-8
    assert abs(rep[0]["n_ham"] - rep0[0]["n_ham"]) <= 0.02 * rep0[0]["n_ham"], (rep[0]["n_ham"], rep0[0]["n_ham"])


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
    on the tensor cores (tcgen05, three-piece bf16 split) it matches the oracle's
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
