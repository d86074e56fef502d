"""Schur-complement Sternheimer solves on the GPU (ikr_set_schur).

The Schur form changes the operator CG iterates on, not the solution: chi0
with it enabled must equal the oracle's chi0 (exact pseudo-inverse solves) to
the same 1e-10 as the plain CG, the mixed-precision Dyson solve must still
reach tau, and on cfg1 (gap 0.011 Ha, two computed bands above it) it must
take fewer Hamiltonian applications than the plain projected CG."""
import numpy as np
import pytest

import gpu_common
from gpu_common import dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu


def _context(name, dense=True, **kw):
    """dense: the ground state of the dense diagonalisation (test helper); else
    the library's eigensolver."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import groundstate
    if dense:
        return gpu_common.dense_context_for(system(name), **kw)
    return groundstate.context_for(system(name), **kw)


@pytest.mark.parametrize("name", ["tiny_insulator", "tiny_ortho_k", "tiny_metal", "tiny_kb"])
def test_schur_chi0_matches_oracle(name):
    from oracle import response
    from workloads import perturbation
    s, gs = system(name), oracle_state(name)
    ctx = _context(name, schur=True)
    dV = perturbation(s)
    d_gpu, _ = ctx.apply_chi0(dev(dV), tol=None)
    assert rel(d_gpu.cpu().numpy(), response.chi0(gs, dV)) < 1e-10
    ctx.destroy()


def test_schur_chi0_with_gpu_eigenpairs():
    from oracle import response
    from workloads import perturbation
    s, gs = system("tiny_kb"), oracle_state("tiny_kb")
    ctx = _context("tiny_kb", dense=False, eig_tol=1e-11, schur=True)
    dV = perturbation(s)
    d_gpu, _ = ctx.apply_chi0(dev(dV), tol=None)
    assert rel(d_gpu.cpu().numpy(), response.chi0(gs, dV)) < 1e-9
    ctx.destroy()


@pytest.mark.parametrize("name", ["tiny_metal", "tiny_kb"])
def test_schur_mixed_solve_reaches_tau(name):
    from oracle import response
    from workloads import perturbation
    s, gs = system(name), oracle_state(name)
    ctx = _context(name, schur=True)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))) <= 1e-8
    ctx.destroy()


def test_schur_needs_fewer_hamiltonian_applications_on_cfg1():
    from workloads import perturbation
    s = system("cfg1")
    ctx = _context("cfg1", dense=False)
    nsys = ctx.groundstate_nsys
    b, _ = ctx.apply_chi0(dev(perturbation(s)), tol=np.full(nsys, 1e-12))
    b = (b / torch.linalg.norm(b)).contiguous()
    x0, rep0 = ctx.solve_response(b, tau=1e-8, strategy="bal")
    ctx.set_schur(True)
    x1, rep1 = ctx.solve_response(b, tau=1e-8, strategy="bal")
    assert rep0[0]["status"] == 0 and rep1[0]["status"] == 0
    assert rep1[0]["n_ham"] < rep0[0]["n_ham"], (rep0[0]["n_ham"], rep1[0]["n_ham"])
    assert float(torch.linalg.norm(x1 - x0)) < 1e-6
    ctx.destroy()


def test_schur_before_the_ground_state_is_rejected():
    from paper_2505_02319_gb300 import ikr
    s = system("tiny_insulator")
    ctx = ikr.Context.setup_groundstate(s.lattice, s.dims, s.Ecut, s.kpoints, s.kweights, s.V, s.temperature,
                                        s.n_electrons)
    with pytest.raises(ikr.IkrError) as e:
        ctx.set_schur(True)
    assert e.value.status == ikr.IKR_ERR_STATE
    ctx.destroy()
