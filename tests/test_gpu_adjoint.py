"""The adjoint (backward) solve and the differentiable response.

E^T = 1 - K chi0 (Sec. 2.2); the gradient of L(drho), drho = E^-1 chi0 dV, is
chi0 E^-T dL/d drho.  Checked against the oracle and against central finite
differences of a quadratic loss (exact up to solver error)."""
import numpy as np
import pytest

from gpu_common import context, dev, oracle_state, rel, system, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny_metal", "cfg1"])
def test_adjoint_apply_parity(name):
    from oracle import response
    s, gs, ctx = system(name), oracle_state(name), context(name)
    v = np.random.default_rng(8).normal(size=s.dims)
    out, _ = ctx.apply_dielectric_adjoint(dev(v), tol=None)
    assert rel(out.cpu().numpy(), response.dielectric_adjoint(gs, v)) < 1e-10
    # <u, E v> = <E^T u, v> with the GPU operators
    u = np.random.default_rng(9).normal(size=s.dims)
    Ev, _ = ctx.apply_dielectric(dev(v), tol=None)
    Etu, _ = ctx.apply_dielectric_adjoint(dev(u), tol=None)
    lhs = float((dev(u) * Ev).sum())
    rhs = float((Etu * dev(v)).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)   # both operators carry ~1e-10 relative CG error


@pytest.mark.parametrize("name", ["tiny_metal", "cfg1"])
def test_adjoint_solve_parity(name):
    from oracle import gmres, response
    s, gs, ctx = system(name), oracle_state(name), context(name)
    g = np.random.default_rng(10).normal(size=s.dims)
    g /= np.linalg.norm(g)
    lam, rep = ctx.solve_response_adjoint(dev(g), tau=1e-12, strategy="bal")
    ref, _ = gmres.gmres(lambda v: response.dielectric_adjoint(gs, v), g, tol=1e-13, m=30)
    assert rel(lam.cpu().numpy(), ref) < 1e-10
    assert rep[0]["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_of_quadratic_loss(precision):
    """L(dV) = ||W drho(dV)||^2 on the cfg1 system: the autograd gradient along a
    random direction equals the central finite difference (h = 1e-4, L quadratic)
    to 1e-6, and the oracle's adjoint gradient chi0 E^-T (2 W^2 drho)."""
    from oracle import gmres, response
    from paper_2505_02319_gb300.autograd import dyson_response
    from workloads import loss_weights, perturbation
    name = "cfg1"
    s, gs, ctx = system(name), oracle_state(name), context(name)
    W = dev(loss_weights(s))
    dV0 = dev(perturbation(s))
    d = dev(np.random.default_rng(11).normal(size=s.dims))
    d *= float(torch.linalg.norm(dV0)) / float(torch.linalg.norm(d))

    def loss(v):
        return float(torch.sum((W * dyson_response(v, ctx, tau_rel=1e-11, precision=precision)) ** 2))

    x = dV0.clone().requires_grad_(True)
    drho = dyson_response(x, ctx, tau_rel=1e-11, precision=precision)
    L = torch.sum((W * drho) ** 2)
    L.backward()
    grad = x.grad.detach()
    h = 1e-4
    fd = (loss(dV0 + h * d) - loss(dV0 - h * d)) / (2 * h)
    ad = float((grad * d).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd)
    # oracle adjoint gradient
    b = response.chi0(gs, perturbation(s))
    xo, _ = gmres.gmres(lambda v: response.dielectric(gs, v), b, tol=1e-13 * np.linalg.norm(b), m=30)
    go = 2 * loss_weights(s) ** 2 * xo
    lam, _ = gmres.gmres(lambda v: response.dielectric_adjoint(gs, v), go, tol=1e-13 * np.linalg.norm(go), m=30)
    gref = response.chi0(gs, lam)
    assert rel(grad.cpu().numpy(), gref) < (1e-9 if precision == "fp64" else 1e-6)
