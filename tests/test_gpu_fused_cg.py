"""The fused FP32 CG update (one thread-block cluster per k-point: alpha, x, r,
the stopping test, z = Q M^-1 r and p in one launch) against the sequence of
kernels it replaces, selected with IKR_CG_FUSED=0 when a context plans: both
solve the Dyson equation to the true residual tau with the guaranteed
tolerances (grt_exact, Theorem inexact_gmres_dyson; bal drops the gap terms
and carries no such guarantee), their solutions agree to the FP32 level, and
the fused path really replaces the scalar launches."""
import os

import numpy as np
import pytest

import gpu_common
from gpu_common import dev, oracle_state, system

pytestmark = pytest.mark.gpu


def _run(name, b, fused):
    from paper_2505_02319_gb300 import groundstate
    os.environ["IKR_CG_FUSED"] = "1" if fused else "0"
    try:
        ctx = gpu_common.dense_context_for(system(name))
        ctx.profile_start()
        x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
        prof = ctx.profile_read()
    finally:
        del os.environ["IKR_CG_FUSED"]
    return x.cpu().numpy(), rep, prof


@pytest.mark.parametrize("name", ["tiny_ortho_k", "cfg1"])
def test_fused_cg_matches_unfused(name):
    from oracle import response
    from workloads import perturbation
    s, gs = system(name), oracle_state(name)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    xf, repf, pf = _run(name, b, True)
    xu, repu, pu = _run(name, b, False)
    for x in (xf, xu):
        assert np.linalg.norm(b - response.dielectric(gs, x.reshape(s.dims))) <= 1e-8
    assert np.linalg.norm(xf - xu) <= 1e-6 * np.linalg.norm(xu)
    # the fused update takes the place of three scalar stages per CG iteration
    assert pf["scalar"]["launches"] < pu["scalar"]["launches"] / 2
