"""Pins for the oracle's chi0 (eqs. chi0, delta_f, fprime, delta_phi_P,
sternheimer_equation; k-form eq. kchi0).  CPU only."""
import numpy as np
import pytest

from oracle import dft, groundstate, response
from workloads import make_system, perturbation

NAMES = ["tiny_insulator", "tiny_ortho_k", "tiny_metal"]


@pytest.fixture(scope="module")
def states():
    return {n: (make_system(n), groundstate.solve(make_system(n))) for n in NAMES}


def _rand(dims, seed):
    return np.random.default_rng(seed).normal(size=dims)


@pytest.mark.parametrize("name", NAMES)
def test_chi0_self_adjoint_and_negative(states, name):
    s, gs = states[name]
    a, b = _rand(s.dims, 1), _rand(s.dims, 2)
    ca, cb = response.chi0(gs, a), response.chi0(gs, b)
    assert abs((a * cb).sum() - (ca * b).sum()) < 1e-13 * np.abs(a * cb).sum()
    for seed in range(3, 8):
        v = _rand(s.dims, seed)
        assert (v * response.chi0(gs, v)).sum() <= 0.0


@pytest.mark.parametrize("name", NAMES)
def test_charge_conservation(states, name):
    """sum_r drho(r) = 0: insulators by orthogonality, metals through deps_F."""
    s, gs = states[name]
    d = response.chi0(gs, perturbation(s))
    assert abs(d.sum()) < 1e-13 * np.abs(d).sum()


def _density(s, V):
    return groundstate.solve(s, V=V).rho


@pytest.mark.parametrize("name", NAMES)
def test_chi0_equals_finite_difference_of_density(states, name):
    """chi0 dV = d rho[V + h dV]/dh at h = 0 (Sec. 2.2: chi0 is the derivative of
    the potential-to-density map), with re-diagonalisation and a re-solved Fermi
    level; Richardson extrapolation of central differences."""
    s, gs = states[name]
    dV = perturbation(s)

    def central(h):
        return (_density(s, s.V + h * dV) - _density(s, s.V - h * dV)) / (2 * h)

    h = 2e-3
    fd = (4 * central(h / 2) - central(h)) / 3
    d = response.chi0(gs, dV)
    assert np.linalg.norm(d - fd) / np.linalg.norm(d) < 1e-9


def test_printed_dphiP_coefficient_fails_the_finite_difference(states, monkeypatch):
    """Reading A1: with the coefficient as printed in eq. delta_phi_P
    (f_n^2/(f_n^2+f_m^2) (f_n-f_m)/(eps_n-eps_m)) next to the factor f_n of
    eq. chi0, chi0 of a metal misses the finite difference; the reading
    f_n/(f_n^2+f_m^2) (f_n-f_m)/(eps_n-eps_m) passes (previous test)."""
    s, gs = states["tiny_metal"]
    dV = perturbation(s)
    h = 2e-3
    fd = (_density(s, s.V + h * dV) - _density(s, s.V - h * dV)) / (2 * h)
    monkeypatch.setattr(response, "dphiP_coefficient",
                        lambda fn, fm, d: fn * fn / (fn * fn + fm * fm) * d)
    d = response.chi0(gs, dV)
    assert np.linalg.norm(d - fd) / np.linalg.norm(fd) > 1e-2


def _sum_over_states(gs, dV):
    """drho = sum_k w_k sum_{n,m} D_nm conj(psi_n) psi_m <phi_m, dV phi_n>
    - deps_F sum_k w_k sum_n f'_n |psi_n|^2 over ALL eigenpairs of the discrete H_k
    (Adler-Wiser form), D_nm = (f_n - f_m)/(eps_n - eps_m) with f truncated to the
    occupied set and the f' limit for degenerate pairs."""
    out = np.zeros(gs.dims)
    num = den = 0.0
    for kb in gs.kblocks:
        nb = len(kb.eps)
        f = np.where(np.arange(nb) < kb.nocc, kb.f, 0.0)
        fp = np.where(np.arange(nb) < kb.nocc, kb.fprime, 0.0)
        psi = dft.F_inv(kb.vecs.T, kb.flat, gs.dims, gs.volume).reshape(nb, -1)
        Vmn = (gs.volume / gs.n_grid) * (psi.conj() * dV.ravel()) @ psi.T   # [m, n]
        e = kb.eps
        de = e[:, None] - e[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            D = (f[:, None] - f[None, :]) / de
        deg = np.abs(de) < response.DEGENERATE
        D[deg] = (0.5 * (fp[:, None] + fp[None, :]))[deg]
        # drho(r) = sum_{n,m} D_nm conj(psi_n(r)) psi_m(r) V_mn
        acc = np.einsum("nm,nr,mr,mn->r", D, psi.conj(), psi, Vmn, optimize=True)
        out += kb.weight * acc.real.reshape(gs.dims)
        num += kb.weight * np.dot(fp, np.diag(Vmn).real)
        den += kb.weight * fp.sum()
        kb._rho_fp = (np.abs(psi) ** 2 * fp[:, None]).sum(0)
    deF = num / den if den else 0.0
    for kb in gs.kblocks:
        out -= deF * kb.weight * kb._rho_fp.reshape(gs.dims)
    return out


@pytest.mark.parametrize("name", NAMES)
def test_sternheimer_route_equals_sum_over_states(states, name):
    s, gs = states[name]
    for seed in (0, 1):
        dV = _rand(s.dims, 20 + seed)
        d = response.chi0(gs, dV)
        np.testing.assert_allclose(d, _sum_over_states(gs, dV), atol=1e-12 * np.abs(d).max())


def test_free_electron_lindhard():
    """V = 0 with smearing: chi0 cos(q.r) = L(q)/|Omega| cos(q.r), L(q) the
    discrete Lindhard sum sum_k w_k sum_{G, G+q in sphere} D(eps_kG, eps_k,G+q)."""
    s = make_system("tiny_metal")
    s.V = np.zeros(s.dims)
    gs = groundstate.solve(s)
    fr = np.stack(np.meshgrid(*[np.arange(n) / n for n in s.dims], indexing="ij"), -1)
    from oracle import basis
    B = basis.reciprocal_lattice(s.lattice)
    for j in [(1, 0, 0), (1, 1, 0), (0, 2, 1)]:
        q = np.array(j)
        dV = np.cos(2 * np.pi * (fr @ q.astype(float)))
        L = 0.0
        for kb in gs.kblocks:
            # plane-wave eigenstates: energy and truncated occupation per G
            order = np.argsort(kb.kinetic, kind="stable")
            occ = np.zeros(len(kb.kinetic), bool)
            occ[order[:kb.nocc]] = True
            idx = {tuple(m): i for i, m in enumerate(kb.miller)}
            fG = np.where(occ, groundstate.fermi_dirac((kb.kinetic - gs.eF) / s.temperature), 0.0)
            fpG = np.where(occ, groundstate.fermi_dirac_derivative((kb.kinetic - gs.eF)
                                                                   / s.temperature) / s.temperature, 0.0)
            for i, m in enumerate(kb.miller):
                jj = idx.get(tuple(m + q))
                if jj is None:
                    continue
                ea, eb = kb.kinetic[i], kb.kinetic[jj]
                if abs(ea - eb) < response.DEGENERATE:
                    D = 0.5 * (fpG[i] + fpG[jj])
                else:
                    D = (fG[i] - fG[jj]) / (ea - eb)
                L += kb.weight * D
        d = response.chi0(gs, dV)
        np.testing.assert_allclose(d, L / gs.volume * dV, atol=1e-12)


@pytest.mark.parametrize("name", NAMES)
def test_sternheimer_solutions(states, name):
    """dphi^Q_n solves Q(H - eps_n)Q x = -Q F(dV F^-1 phi_n) and lies in range(Q)
    (proof of Lemma cgtol_E, Remark rmk:sternheimer_solution)."""
    s, gs = states[name]
    dV = perturbation(s)
    _, info = response.chi0(gs, dV, return_parts=True)
    for kb, (psi, deps, dphi) in zip(gs.kblocks, info["parts"]):
        Phi = kb.vecs[:, :kb.nocc]
        Q = np.eye(len(kb.eps)) - Phi @ Phi.conj().T
        y = dft.F(dV[None] * psi, kb.flat, s.dims, gs.volume)
        for n in range(kb.nocc):
            xq = Q @ dphi[n]
            A = Q @ (kb.H - kb.eps[n] * np.eye(len(kb.eps))) @ Q
            np.testing.assert_allclose(A @ xq, -Q @ y[n], atol=1e-12)
            if s.temperature == 0.0:
                assert np.abs(Phi.conj().T @ dphi[n]).max() < 1e-13
