"""Supercells on the GPU (Remark rmk:scaling; Bloch folding).

The GPU path on a supercell of two replicas at the Gamma point is compared
with the oracle on the small cell with its two k-points, tiled: the two sides
share neither the cell nor the k-points, so the comparison checks the GPU's
Gamma-point path against the oracle's k-point path.  A three-replica
insulator then runs the mixed-precision solve with the guaranteed rule."""
import numpy as np
import pytest

import gpu_common
from gpu_common import dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu


def _supercell_context(name, ell, **kw):
    import __graft_entry__
    __graft_entry__.build()
    from workloads import supercell
    S = supercell(system(name), ell, **kw)
    return S, gpu_common.dense_context_for(S)


@pytest.mark.parametrize("name", ["tiny_ortho_k", "tiny_metal"])
def test_gpu_supercell_chi0_is_the_tiled_small_cell_response(name):
    from oracle import response
    from workloads import perturbation
    P, gp = system(name), oracle_state(name)            # k-grid (2, 1, 1)
    S, ctx = _supercell_context(name, 2)                # Gamma only
    dV = perturbation(P)
    d_gpu, _ = ctx.apply_chi0(dev(np.tile(dV, (2, 1, 1))), tol=None)
    d_ref = np.tile(response.chi0(gp, dV), (2, 1, 1))
    assert rel(d_gpu.cpu().numpy(), d_ref) < 1e-10
    ctx.destroy()


def test_gpu_supercell_mixed_solve_reaches_tau():
    from oracle import groundstate as ogs, response
    from workloads import perturbation
    S, ctx = _supercell_context("tiny_insulator", 3, kgrid=(1, 1, 1))
    gs = ogs.solve(S)
    b = response.chi0(gs, perturbation(S, center=S.lattice @ np.array([0.1, 0.6, 0.45])))
    b /= np.linalg.norm(b)
    x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(S.dims))) <= 1e-8
    ctx.destroy()
