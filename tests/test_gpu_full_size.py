"""Parity at the full size of the benchmark workload (cfg2: 48^3 grid, 2x2x2 k,
Ecut = 15 Ha, 251 Sternheimer systems), in the launch configuration bench.py
times.  The oracle's dense ground state of all eight k-points takes about a
minute of CPU time; it is computed once per module."""
import numpy as np
import pytest

from gpu_common import context, dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu

NAME = "cfg2"


def test_hamiltonian_full_size():
    from oracle import groundstate
    s, ctx = system(NAME), context(NAME)
    rng = np.random.default_rng(7)
    for k in (0, 7):
        miller, flat, kin, H = groundstate.hamiltonian(s.lattice, s.dims, s.Ecut, s.kpoints[k], s.V)
        np.testing.assert_array_equal(ctx.basis_millers(k), miller)
        psi = rng.normal(size=(4, len(kin))) + 1j * rng.normal(size=(4, len(kin)))
        out = ctx.apply_hamiltonian(k, torch.tensor(psi, device="cuda")).cpu().numpy()
        assert rel(out, (H @ psi.T).T) < 1e-12
        from paper_2505_02319_gb300 import ikr
        out32 = ctx.apply_hamiltonian(k, torch.tensor(psi.astype(np.complex64), device="cuda"),
                                      precision=ikr.MIXED).cpu().numpy()
        assert rel(out32, (H @ psi.astype(np.complex64).astype(np.complex128).T).T) < 2e-6


def test_chi0_full_size():
    """drho = chi0 dV0 of the workload against the oracle's exact chi0 (all
    Ng = 110,592 grid values), FP64 path with tight Sternheimer tolerances."""
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = system(NAME), oracle_state(NAME), context(NAME)
    info = ctx.groundstate_info(ctx.nbands, s.n_grid)
    np.testing.assert_array_equal(info["nocc"], [kb.nocc for kb in gs.kblocks])
    assert rel(info["rho"].cpu().numpy(), gs.rho) < 1e-11
    dV = perturbation(s)
    out, rep = ctx.apply_chi0(dev(dV), tol=np.full(int(info["nocc"].sum()), 1e-12))
    assert rel(out.cpu().numpy(), response.chi0(gs, dV)) < 1e-10


def test_dielectric_full_size_mixed_residual():
    """The benchmark's solve (mixed precision, bal, tau = 1e-8) reaches a true
    residual ||b - E x|| <= 1e-8, E applied by the oracle."""
    from oracle import response
    from workloads import perturbation
    s, gs, ctx = system(NAME), oracle_state(NAME), context(NAME)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="bal", precision="mixed")
    res = np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims)))
    assert res <= 1e-8
