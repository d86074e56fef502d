"""The differentiated batch on the 10-bohr Gamma-point cell (cfg1's system):
32 seeded perturbations (16 Gaussian bumps, 16 atom-displacement derivatives
dV/dR of the Gaussian potentials), solved together in lockstep.

1. The mixed-precision lockstep solve with the guaranteed rule (Theorem
   inexact_gmres_dyson): every right-hand side's true residual against the
   oracle's E is at most tau = 1e-8.
2. The gradient of L = sum_r ||W drho_r||^2 (W a seeded random diagonal)
   through the batched autograd function (mixed precision; backward = one
   lockstep adjoint solve E^T lambda = g and chi0 lambda per row, nothing kept
   from the forward pass): along a random direction in all 32 perturbations it
   equals the central finite difference (h = 1e-4; L is quadratic in dV, so the
   difference is exact up to solver error, here FP64 lockstep solves at 1e-11)
   to 1e-6 relative, and two of its rows equal the oracle's adjoint gradient
   chi0 E^-T (2 W^2 drho_r) to 1e-6."""
import numpy as np
import pytest

from gpu_common import context, dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu


def _batch():
    from workloads import response_batch
    s = system("cfg1")
    dvs = response_batch(s)
    assert dvs.shape[0] == 32
    return s, torch.tensor(dvs.reshape(32, -1), dtype=torch.float64, device="cuda")


def test_lockstep_batch_of_32_meets_tau_against_the_oracle():
    from oracle import response
    s, dV = _batch()
    gs, ctx = oracle_state("cfg1"), context("cfg1")
    nsys = ctx.groundstate_nsys
    b = torch.stack([ctx.apply_chi0(row.contiguous(), tol=np.full(nsys, 1e-12))[0] for row in dV])
    b = (b / torch.linalg.norm(b, dim=1, keepdim=True)).contiguous()
    x, rep = ctx.solve_response(b, tau=1e-8, strategy="grt_exact", precision="mixed")
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    for r in range(32):
        assert rep[r]["status"] == 0, r
        res = np.linalg.norm(bh[r] - response.dielectric(gs, xh[r].reshape(s.dims)).ravel())
        assert res <= 1e-8, (r, res)


def test_batched_gradient_matches_finite_difference_and_oracle():
    from oracle import gmres, response
    from paper_2505_02319_gb300.autograd import dyson_response
    from workloads import loss_weights
    s, dV = _batch()
    gs, ctx = oracle_state("cfg1"), context("cfg1")
    W = dev(loss_weights(s))
    D = torch.tensor(np.random.default_rng(21).normal(size=dV.shape), device="cuda")
    D *= float(torch.linalg.norm(dV)) / float(torch.linalg.norm(D))

    def loss(v, precision):
        return float(torch.sum((W * dyson_response(v, ctx, tau_rel=1e-11, precision=precision)) ** 2))

    x = dV.clone().requires_grad_(True)
    drho = dyson_response(x, ctx, tau_rel=1e-11, precision="mixed")
    assert drho.shape == dV.shape
    L = torch.sum((W * drho) ** 2)
    L.backward()
    grad = x.grad.detach()
    h = 1e-4
    fd = (loss(dV + h * D, "fp64") - loss(dV - h * D, "fp64")) / (2 * h)
    ad = float((grad * D).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)
    for r in (0, 16):                     # a bump and a displacement
        dv = dV[r].cpu().numpy().reshape(s.dims)
        b = response.chi0(gs, dv)
        xo, _ = gmres.gmres(lambda v: response.dielectric(gs, v), b, tol=1e-13 * np.linalg.norm(b), m=30)
        go = 2 * loss_weights(s) ** 2 * xo
        lam, _ = gmres.gmres(lambda v: response.dielectric_adjoint(gs, v), go, tol=1e-13 * np.linalg.norm(go), m=30)
        assert rel(grad[r].cpu().numpy(), response.chi0(gs, lam)) < 1e-6, r
