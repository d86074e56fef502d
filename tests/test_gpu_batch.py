"""Several right-hand sides in lockstep (ikr_solve_response with nrhs > 1).

Each right-hand side keeps its own GMRES state; the E applications of a round
share one CG over all their Sternheimer systems.  Checks: in FP64 the batched
solutions equal the ones solved one after another (IKR_BATCH=0) up to
rounding; every solution meets its own tau against the oracle's E (mixed
precision, Kerker, adjoint); the cfg1 batch of 32 perturbations (16 bumps, 16
atom displacements) beats solving them one after another."""
import os
import time

import numpy as np
import pytest

from gpu_common import context, dev, oracle_state, system, torch

pytestmark = pytest.mark.gpu


def _rhs(name, n):
    from oracle import response
    from workloads import response_batch
    gs = oracle_state(name)
    dvs = response_batch(system(name), n_bumps=n - n // 2, n_displacements=n // 2)
    b = np.array([response.chi0(gs, dv).ravel() for dv in dvs])
    return b / np.linalg.norm(b, axis=1, keepdims=True)


def _sequential(fn):
    os.environ["IKR_BATCH"] = "0"
    try:
        return fn()
    finally:
        del os.environ["IKR_BATCH"]


@pytest.mark.parametrize("name", ["tiny_insulator", "tiny_metal", "tiny_kb"])
def test_batch_equals_sequential_fp64(name):
    ctx = context(name)
    b = torch.tensor(_rhs(name, 4), device="cuda")
    xb, rb = ctx.solve_response(b, tau=1e-10, strategy="bal")
    xs, rseq = _sequential(lambda: ctx.solve_response(b, tau=1e-10, strategy="bal"))
    for r in range(4):
        assert rb[r]["status"] == 0 and rseq[r]["status"] == 0
        d = float(torch.linalg.norm(xb[r] - xs[r]) / torch.linalg.norm(xs[r]))
        assert d < 1e-12, (r, d)
        assert rb[r]["outer_iters"] == rseq[r]["outer_iters"]


@pytest.mark.parametrize("name", ["tiny_metal", "tiny_ortho_k"])
def test_batch_mixed_each_meets_tau(name):
    from oracle import response
    s, gs, ctx = system(name), oracle_state(name), context(name)
    b = _rhs(name, 5)
    x, rep = ctx.solve_response(torch.tensor(b, device="cuda"), tau=1e-8, strategy="grt_exact", precision="mixed")
    for r in range(5):
        assert rep[r]["status"] == 0
        res = np.linalg.norm(b[r] - response.dielectric(gs, x[r].cpu().numpy().reshape(s.dims)).ravel())
        assert res <= 1e-8, (r, res)


def test_batch_kerker_meets_tau():
    from oracle import response
    s, gs, ctx = system("tiny_metal"), oracle_state("tiny_metal"), context("tiny_metal")
    b = _rhs("tiny_metal", 3)
    alpha = 0.8
    x, rep = ctx.solve_response(torch.tensor(b, device="cuda"), tau=1e-9, strategy="bal", kerker_alpha=alpha)
    for r in range(3):
        assert rep[r]["status"] == 0
        Ex = response.dielectric(gs, x[r].cpu().numpy().reshape(s.dims))
        tr = response.kerker(b[r].reshape(s.dims) - Ex, s.lattice, s.dims, alpha)
        assert np.linalg.norm(tr) <= 1e-9


def test_batch_adjoint_each_meets_tau():
    from oracle import response
    s, gs, ctx = system("tiny_metal"), oracle_state("tiny_metal"), context("tiny_metal")
    g = _rhs("tiny_metal", 3)
    lam, rep = ctx.solve_response_adjoint(torch.tensor(g, device="cuda"), tau=1e-9, strategy="bal")
    for r in range(3):
        assert rep[r]["status"] == 0
        res = np.linalg.norm(g[r] - response.dielectric_adjoint(gs, lam[r].cpu().numpy().reshape(s.dims)).ravel())
        assert res <= 1e-9


def test_batch_of_32_perturbations_on_cfg1_is_faster():
    from workloads import response_batch
    s = system("cfg1")
    ctx = context("cfg1")
    nsys = ctx.groundstate_nsys
    dvs = response_batch(s)
    b = torch.stack([ctx.apply_chi0(dev(dv), tol=np.full(nsys, 1e-12))[0] for dv in dvs])
    b = (b / torch.linalg.norm(b, dim=1, keepdim=True)).contiguous()
    ctx.solve_response(b[:2], tau=1e-8, strategy="bal", precision="mixed")   # warm-up
    torch.cuda.synchronize()
    t0 = time.time()
    xb, rb = ctx.solve_response(b, tau=1e-8, strategy="bal", precision="mixed")
    torch.cuda.synchronize()
    t_batch = time.time() - t0
    t0 = time.time()
    xs, rs = _sequential(lambda: ctx.solve_response(b, tau=1e-8, strategy="bal", precision="mixed"))
    torch.cuda.synchronize()
    t_seq = time.time() - t0
    assert all(r["status"] == 0 for r in rb)
    # both meet tau, so they agree to about 2 tau times ||E^-1||
    assert float(torch.max(torch.linalg.norm(xb - xs, dim=1))) < 1e-6
    assert t_batch < 0.8 * t_seq, (t_batch, t_seq)
