"""The autotuner (ikr_autotune): it times the interchangeable kernel variants
(FP32 plane kernel x projection path in a few CG iterations; the cluster size
of the fused CG update; the padded and the swizzled double-float plane pass)
on the context's own systems and keeps the fastest.  Checks: every candidate was timed, the choice is the fastest
one, and a mixed-precision solve after tuning still matches the oracle's E to
tau (the variants agree to rounding)."""
import numpy as np
import pytest

import gpu_common
from gpu_common import dev, oracle_state, system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny_ortho_k", "cfg2"])
def test_autotune_picks_the_fastest_variant(name):
    ctx = gpu_common.dense_context_for(system(name))
    r = ctx.autotune()
    cg = {(tc, rc): v for tc, key in ((False, "cg_iter_ms_cuda_cores"), (True, "cg_iter_ms_tensor_cores"))
          for rc, v in zip((0, 4, 5), (r[key]["plane_full"], r[key]["plane_compact4"], r[key]["plane_compact5"]))}
    assert all(v > 0 for v in cg.values())
    assert cg[(r["tensor_cores"], r["plane_rc"])] == min(cg.values())
    cl = {int(k): v for k, v in r["cg_iter_ms_cluster"].items() if v > 0}
    if r["tensor_cores"] or not cl:   # no fused update (tensor cores, or no cluster size fits)
        assert r["cg_fused_cluster"] == 0
    else:
        assert cl and r["cg_fused_cluster"] in cl
        assert cl[r["cg_fused_cluster"]] == min(cl.values())
    if name == "cfg2":
        d = r["df64_apply_ms"]
        assert d["padded"] > 0 and d["swizzled"] > 0
        assert r["plane_sw"] == (d["swizzled"] <= d["padded"])
    ctx.destroy()


def test_solve_after_autotune_meets_tau():
    from oracle import response
    from workloads import perturbation
    s, gs = system("tiny_metal"), oracle_state("tiny_metal")
    ctx = gpu_common.dense_context_for(s)
    ctx.autotune()
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    x, rep = ctx.solve_response(dev(b), tau=1e-8, strategy="grt_exact", precision="mixed")
    assert rep[0]["status"] == 0
    assert np.linalg.norm(b - response.dielectric(gs, x.cpu().numpy().reshape(s.dims))) <= 1e-8
    ctx.destroy()
