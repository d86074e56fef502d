"""The GPU ground-state eigensolver (ikr_compute_eigenpairs: Chebyshev-filtered
subspace iteration on the library's H_k): eigenvalues against the oracle's
dense diagonalisation, chi0 with its eigenpairs against the oracle at the
FP64 parity tolerance, and the cfg2 spectrum against the dense GPU path."""
import numpy as np
import pytest

import gpu_common
from gpu_common import dev, oracle_state, rel, system

pytestmark = pytest.mark.gpu


def _ctx(name, **kw):
    from paper_2505_02319_gb300 import groundstate
    return groundstate.context_for(system(name), **kw)


@pytest.mark.parametrize("name", ["tiny_insulator", "tiny_ortho_k", "tiny_metal", "cfg1"])
def test_eigenvalues_and_chi0_match_oracle(name):
    from oracle import response
    from workloads import perturbation
    s, gs = system(name), oracle_state(name)
    ctx = _ctx(name, eig_tol=1e-11)
    info = ctx.groundstate_info(ctx.nbands, s.n_grid)
    for k, kb in enumerate(gs.kblocks):
        assert np.max(np.abs(ctx.eigenvalues[k] - kb.eps[:ctx.nbands])) < 1e-10
    assert rel(info["rho"].cpu().numpy(), gs.rho) < 1e-10
    dV = perturbation(s)
    nsys = ctx.groundstate_nsys
    out = ctx.apply_chi0(dev(dV), tol=np.full(nsys, 1e-13))[0].cpu().numpy()
    assert rel(out, response.chi0(gs, dV)) < 1e-10


def test_cfg2_spectrum_matches_dense():
    from paper_2505_02319_gb300 import groundstate
    s = system("cfg2")
    ctx = _ctx("cfg2")
    ev_chfsi, res = ctx.eigenvalues, ctx.eig_residuals
    assert max(res) <= 1e-10
    ev_dense, _ = gpu_common.dense_eigenpairs(ctx, s.nbands)
    assert np.max(np.abs(ev_chfsi - ev_dense)) < 1e-9
