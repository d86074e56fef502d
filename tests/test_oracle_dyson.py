"""Pins for the dielectric adjoint E and the GMRES solvers (eqs.
dyson_discretised, op_discretised; Algorithm 1; Lemmas
inexact_residual_norm, gmres_y_k_bound; Theorem inexact_gmres_dyson).  CPU only."""
import numpy as np
import pytest

from oracle import gmres, groundstate, response
from workloads import make_system, perturbation


@pytest.fixture(scope="module")
def ins():
    s = make_system("tiny_insulator")
    return s, groundstate.solve(s)


@pytest.fixture(scope="module")
def metal():
    s = make_system("tiny_metal")
    return s, groundstate.solve(s)


@pytest.fixture(scope="module")
def metal_E(metal):
    """The dense E of the tiny metal (one column per grid point)."""
    s, gs = metal
    return response.dense_operator(lambda v: response.dielectric(gs, v), s.dims)


def test_rescaling_is_an_identity(ins):
    """eq. op_discretised: v - ||Kv|| chi0(Kv/||Kv||) = v - chi0 K v (linearity)."""
    s, gs = ins
    v = np.random.default_rng(0).normal(size=s.dims)
    np.testing.assert_allclose(response.dielectric(gs, v),
                               v - response.chi0(gs, response.apply_K(v, gs)), atol=1e-13)


def test_adjoint_is_the_dielectric_operator(ins):
    """E = 1 - chi0 K has transpose 1 - K chi0 (chi0 and K symmetric, Sec. 2.2)."""
    s, gs = ins
    rng = np.random.default_rng(1)
    u, v = rng.normal(size=s.dims), rng.normal(size=s.dims)
    lhs = (u * response.dielectric(gs, v)).sum()
    rhs = ((u - response.apply_K(response.chi0(gs, u), gs)) * v).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_function_is_the_transpose(metal, metal_E):
    """dielectric_adjoint is the transpose of the dense E (metal, k-points)."""
    s, gs = metal
    E = metal_E
    rng = np.random.default_rng(4)
    v = rng.normal(size=s.dims)
    np.testing.assert_allclose(response.dielectric_adjoint(gs, v).ravel(), E.T @ v.ravel(), atol=1e-12)


@pytest.mark.parametrize("which", ["ins", "metal"])
def test_gmres_matches_dense_solve(which, ins, metal, metal_E):
    s, gs = ins if which == "ins" else metal
    E = response.dense_operator(lambda v: response.dielectric(gs, v), s.dims) if which == "ins" else metal_E
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    x_dense = np.linalg.solve(E, b.ravel()).reshape(s.dims)
    x, hist = gmres.gmres(lambda v: response.dielectric(gs, v), b, tol=1e-13, m=20)
    np.testing.assert_allclose(x, x_dense, atol=1e-11)
    assert np.linalg.norm(b - response.dielectric(gs, x)) < 1e-12


@pytest.fixture(scope="module")
def rhs(ins):
    s, gs = ins
    b = response.chi0(gs, perturbation(s))
    return b / np.linalg.norm(b)


def _true_residual(gs, b, x):
    return float(np.linalg.norm(b - response.dielectric(gs, x)))


def test_guaranteed_strategy_reaches_tau(ins, rhs):
    """Theorem inexact_gmres_dyson: with tau^CG <= C_{i,n} s/(3m) tau/||r~_{i-1}||
    (exact prefactor, gaps kept) the true residual is <= tau."""
    s, gs = ins
    for tau in (1e-6, 1e-9):
        res = gmres.inexact_gmres(gs, rhs, tau, 10, "grt_exact")
        assert res.converged
        assert _true_residual(gs, rhs, res.x) <= tau


def test_residual_lemmas_hold(ins, rhs):
    """Lemma inexact_residual_norm and Lemma gmres_y_k_bound on the last cycle,
    with a deliberately loose static strategy so that the errors matter."""
    s, gs = ins
    for strategy in ("D10", "agr", "bal"):
        res = gmres.inexact_gmres(gs, rhs, 1e-8, 8, strategy, track_errors=True)
        y, H, r = res.cycle_y, res.cycle_H, res.cycle_res
        true = _true_residual(gs, rhs, res.x)
        bound = res.cycle_err0 + r[-1] + sum(e * abs(yi) for e, yi in zip(res.cycle_errs, y))
        assert true <= bound * (1 + 1e-8) + 1e-15
        sigma = np.linalg.svd(H, compute_uv=False)[-1]
        for i in range(len(y)):
            assert abs(y[i]) <= r[i] / sigma * (1 + 1e-10)


def test_adaptive_tolerances_grow_as_gmres_converges(ins, rhs):
    """tau^CG_i ~ 1/||r~_{i-1}|| (Remark rmk:superlinear_convergence): the CG
    tolerance rises and the inner work per step falls."""
    s, gs = ins
    kxc = response.exchange_kernel(gs.rho)
    tols = [gmres.cg_tolerances(gs, "bal", 1e-9, i, 10, 1.0, r, 1.0, 1.0)[0]
            for i, r in [(1, 1.0), (2, 1e-3), (3, 1e-6)]]
    assert tols[0] < tols[1] < tols[2]
    res = gmres.inexact_gmres(gs, rhs, 1e-9, 20, "bal")
    assert res.converged
    assert _true_residual(gs, rhs, res.x) < 1e-8
    del kxc


def test_bal_prefactor_formula(ins, metal):
    """Table strategies: bal = sqrt|Omega|/sqrt(Nocc) * sqrt|Omega| / (2 f_n sqrt(Ng Nocc));
    k-form (Table strategies_k with Nocc_k N_mp -> Nocc): |Omega|/(2 f w_k Nocc sqrt(Ng))."""
    s, gs = ins
    nocc = gs.kblocks[0].nocc
    pf = gmres.prefactors(gs, "bal", 1.0)
    ref = np.sqrt(gs.volume) / np.sqrt(nocc) * np.sqrt(gs.volume) / (
        2 * 2.0 * np.sqrt(gs.n_grid * nocc))
    np.testing.assert_allclose(pf, ref, rtol=1e-14)
    s, gs = metal
    pf = gmres.prefactors(gs, "bal", 1.0)
    ntot = sum(kb.nocc for kb in gs.kblocks)
    i = 0
    for kb in gs.kblocks:
        for n in range(kb.nocc):
            assert abs(pf[i] - gs.volume / (2 * kb.f[n] * kb.weight * ntot * np.sqrt(gs.n_grid))) \
                <= 1e-12 * pf[i]
            i += 1


def test_cg_stays_in_range_of_Q(ins):
    """Remark rmk:sternheimer_solution: CG iterates lie in range(Q); >= 1 iteration."""
    s, gs = ins
    kb = gs.kblocks[0]
    Phi = kb.vecs[:, :kb.nocc]
    rng = np.random.default_rng(3)
    b = rng.normal(size=len(kb.eps)) + 1j * rng.normal(size=len(kb.eps))
    b -= Phi @ (Phi.conj().T @ b)
    x, it, rn = gmres.sternheimer_cg(kb.H, kb.eps[0], Phi, b, 1e-12, kb.kinetic, 1.0)
    assert np.abs(Phi.conj().T @ x).max() < 1e-12
    A = kb.H - kb.eps[0] * np.eye(len(kb.eps))
    Q = np.eye(len(kb.eps)) - Phi @ Phi.conj().T
    assert np.linalg.norm(b - Q @ A @ Q @ x) < 1e-11
    _, it1, _ = gmres.sternheimer_cg(kb.H, kb.eps[0], Phi, b, 1e3, kb.kinetic, 1.0)
    assert it1 == 1


@pytest.mark.parametrize("which", ["ins", "metal"])
def test_adaptive_strategies_are_more_efficient_than_fixed_ones(which, ins, metal):
    """The paper's efficiency claim (Sec. 4, Tables summary_*): with the
    efficiency eta = -log10(||r_end|| / ||r_0||) / N_ham of Sec. 4.1.3, the
    adaptive rules (agr, bal, grt and the exact prefactor) have eta_rel =
    eta / eta_D10 > 1 and need fewer Hamiltonian applications than the fixed
    rule D10, which needs fewer than D100; bal and grt_exact still reach tau."""
    s, gs = ins if which == "ins" else metal
    b = response.chi0(gs, perturbation(s))
    tau, m = 1e-9, 10
    r0 = float(np.linalg.norm(b))
    eta, nham = {}, {}
    for strategy in ("D10", "D100", "agr", "bal", "grt", "grt_exact"):
        res = gmres.inexact_gmres(gs, b, tau, m, strategy)
        assert res.converged
        r_end = _true_residual(gs, b, res.x)
        if strategy in ("bal", "grt_exact"):
            assert r_end <= tau
        eta[strategy] = -np.log10(r_end / r0) / res.nham
        nham[strategy] = res.nham
    assert nham["D10"] < nham["D100"]
    for strategy in ("agr", "bal", "grt", "grt_exact"):
        assert nham[strategy] < nham["D10"], (strategy, nham)
        assert eta[strategy] / eta["D10"] > 1.0, (strategy, eta)


@pytest.mark.parametrize("which", ["ins", "metal"])
def test_kerker_preconditioned_algorithm(which, ins, metal):
    """Algorithm 1 on T E x = T b (eq. precond_dyson, Kerker T of eq. kerker):
    with the exact prefactor the preconditioned residual ||T (b - E x)|| is
    <= tau (reading A10: the guarantee holds for T r, ||T|| = 1), and x solves
    E x = b to ||T^-1|| tau, ||T^-1|| = 1 / min_{G != 0} |G|^2 / (|G|^2 + alpha^2)."""
    from oracle import basis
    s, gs = ins if which == "ins" else metal
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    tau, alpha = 1e-9, 0.8
    res = gmres.inexact_gmres(gs, b, tau, 10, "grt_exact", kerker_alpha=alpha)
    assert res.converged
    r = b - response.dielectric(gs, res.x)
    assert np.linalg.norm(response.kerker(r, s.lattice, s.dims, alpha)) <= tau
    g2 = np.sort(np.unique(np.round(np.sum(basis.grid_G(s.lattice, s.dims) ** 2, axis=-1).ravel(), 12)))
    g2min = g2[g2 > 0][0]
    assert np.linalg.norm(r) <= tau * (g2min + alpha ** 2) / g2min


@pytest.mark.parametrize("which", ["ins", "metal"])
def test_schur_complement_solves_inside_algorithm_1(which, ins, metal):
    """The Schur-complement Sternheimer solves (Sec. 3.4.2) change the operator
    CG iterates on, not the solutions: Algorithm 1 with them and the exact
    prefactor still reaches tau, its solution agrees with the plain one to the
    accuracy both reach, and no more Hamiltonian applications are needed."""
    s, gs = ins if which == "ins" else metal
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    tau = 1e-9
    plain = gmres.inexact_gmres(gs, b, tau, 10, "grt_exact")
    nb = max(kb.nocc for kb in gs.kblocks) + 4
    sch = gmres.inexact_gmres(gs, b, tau, 10, "grt_exact", schur_nbands=nb)
    assert sch.converged and _true_residual(gs, b, sch.x) <= tau
    assert np.linalg.norm(sch.x - plain.x) < 100 * tau
    assert sch.nham <= plain.nham


def test_adjoint_gradient_equals_finite_difference(metal, metal_E):
    """The gradient of L(dV) = ||W drho||^2, drho = E^-1 chi0 dV, is
    chi0 E^-T (2 W^2 drho) (the adjoint solve of Sec. 2.2 with E^T = 1 - K chi0).
    L is quadratic in dV, so the central difference is exact up to rounding;
    dense solves on the tiny grid."""
    from workloads import loss_weights
    s, gs = metal
    E = metal_E
    W2 = loss_weights(s).ravel() ** 2
    dV = perturbation(s)
    d = np.random.default_rng(12).normal(size=s.dims)
    d *= np.linalg.norm(dV) / np.linalg.norm(d)

    def drho(v):
        return np.linalg.solve(E, response.chi0(gs, v).ravel())

    def loss(v):
        return float(np.sum(W2 * drho(v) ** 2))

    lam = np.linalg.solve(E.T, 2.0 * W2 * drho(dV))
    grad = response.chi0(gs, lam.reshape(s.dims)).ravel()
    h = 1e-3
    fd = (loss(dV + h * d) - loss(dV - h * d)) / (2 * h)
    assert abs(float(grad @ d.ravel()) - fd) <= 1e-9 * abs(fd)


@pytest.mark.parametrize("which", ["ins", "metal"])
def test_adjoint_algorithm_1_reaches_tau_with_the_kernel_bound(which, ins, metal):
    """Algorithm 1 on E^T lambda = g (the adjoint solve of the differentiated
    response) with the exact prefactor, ||K v_i|| replaced by the bound
    ||K|| <= max 4 pi/|G|^2 + max |K^xc|: the true residual ||g - E^T lambda||
    is <= tau, and lambda is the dense solution to that accuracy."""
    s, gs = ins if which == "ins" else metal
    g = response.chi0(gs, perturbation(s))
    g /= np.linalg.norm(g)
    tau = 1e-9
    res = gmres.inexact_gmres(gs, g, tau, 10, "grt_exact", adjoint=True)
    assert res.converged
    assert np.linalg.norm(g - response.dielectric_adjoint(gs, res.x)) <= tau
    # the bound dominates ||K v|| / ||v||, also for the smoothest vectors K^H amplifies most
    kxc = response.exchange_kernel(gs.rho)
    bound = gmres.kernel_norm_bound(gs, kxc)
    rng = np.random.default_rng(5)
    for v in list(rng.normal(size=(4,) + s.dims)) + [g]:
        assert np.linalg.norm(response.apply_K(v, gs, kxc)) <= bound * np.linalg.norm(v)
