"""Oracle parity at the FFT grids of the large workloads.

The plane, density and z-pass kernels are compiled per grid shape, so the
40 x 40 (x 216) instances that the metallic slab runs and the 96 x 96 (x 96)
instances of the 64-atom projector cell need their own oracle comparison.
The oracle cannot diagonalise those systems at their full cut-offs, but the
instances depend only on the grid: the same cells, atoms, k-points and grids
at a reduced cut-off (the slab at 2.5 Ha with 2 x 2 x 1 k-points, N_b,k about
1,100; the projector cell at 1.5 Ha with its 256 Kleinman-Bylander projectors,
N_b = 739, still an insulator: eps_129 - eps_128 = 8e-4 Ha) run exactly the
kernels of the full-size runs.  Checks: H_k in FP64 (1e-12)
and FP32 (2e-6) against the oracle's dense H_k, chi0 with dense ground states
against the oracle's (1e-10), and for the slab the mixed-precision Kerker solve
with the guaranteed rule reaching tau on ||T (b - E x)|| with the oracle's E
(reading A10).  The slab's own reduced grid (12 x 12 x 64), which the oracle
strategy study uses, gets the same solve check."""
import functools

import numpy as np
import pytest

import gpu_common
from gpu_common import dev, rel, torch

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def reduced(name):
    from workloads import make_system, with_cutoff, with_kgrid
    if name == "slab_full_grid":
        s = with_kgrid(with_cutoff(make_system("cfg3"), 2.5, (40, 40, 216)), (2, 2, 1))
    elif name == "slab_study_grid":
        s = with_kgrid(with_cutoff(make_system("cfg3"), 2.5, (12, 12, 64)), (2, 2, 1))
    elif name == "kb_cell_full_grid":
        s = with_cutoff(make_system("cfg4"), 1.5, (96, 96, 96))
    else:
        raise ValueError(name)
    return s


@functools.lru_cache(maxsize=None)
def oracle_gs(name):
    from oracle import groundstate
    return groundstate.solve(reduced(name))


@functools.lru_cache(maxsize=None)
def ctx_of(name):
    return gpu_common.dense_context_for(reduced(name))


@pytest.mark.parametrize("name", ["slab_full_grid", "kb_cell_full_grid"])
def test_hamiltonian_on_the_large_grids(name):
    from paper_2505_02319_gb300 import ikr
    gs, ctx = oracle_gs(name), ctx_of(name)
    assert tuple(ctx.fft_geometry()["dims"]) == tuple(reduced(name).dims)
    rng = np.random.default_rng(31)
    for k, kb in enumerate(gs.kblocks):
        nb = ctx.basis_size(k)
        assert nb == kb.vecs.shape[0]
        np.testing.assert_array_equal(ctx.basis_millers(k), kb.miller)
        psi = rng.normal(size=(3, nb)) + 1j * rng.normal(size=(3, nb))
        ref = psi @ kb.H.T
        out = ctx.apply_hamiltonian(k, torch.tensor(psi, device="cuda")).cpu().numpy()
        assert rel(out, ref) < 1e-12, k
        out32 = ctx.apply_hamiltonian(k, torch.tensor(psi.astype(np.complex64), device="cuda"),
                                      precision=ikr.MIXED).cpu().numpy()
        assert rel(out32, ref) < 2e-6, k


@pytest.mark.parametrize("name", ["slab_full_grid", "kb_cell_full_grid"])
def test_chi0_on_the_large_grids(name):
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = reduced(name), oracle_gs(name), ctx_of(name)
    info = ctx.groundstate_info(ctx.nbands, s.n_grid)
    assert list(info["nocc"]) == [kb.nocc for kb in gs.kblocks]
    dV = perturbation(s)
    out, _ = ctx.apply_chi0(dev(dV), tol=np.full(ctx.groundstate_nsys, 1e-13))
    assert rel(out.cpu().numpy(), response.chi0(gs, dV)) < 1e-10


@pytest.mark.parametrize("name", ["slab_full_grid", "slab_study_grid"])
def test_slab_kerker_mixed_solve_reaches_tau_against_the_oracle(name):
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = reduced(name), oracle_gs(name), ctx_of(name)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    alpha, tau = 0.8, 1e-8
    x, rep = ctx.solve_response(dev(b), tau=tau, strategy="grt_exact", precision="mixed", kerker_alpha=alpha)
    assert rep[0]["status"] == 0 and rep[0]["e_applies_fp32"] >= 0
    r = b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))
    assert np.linalg.norm(response.kerker(r, s.lattice, s.dims, alpha)) <= tau
