"""Pins of the guaranteed CG-tolerance prefactor C_{i,nk} (Theorem
inexact_gmres_dyson in its k-point form, App. F) and of the grt rule derived
from it (Table strategies_k).  CPU only.

Lemma cgtol_E (k-form, App. F) bounds the error of an inexact E application
by a chain of inequalities that ends in

    B = 2 w^-1 ||K v|| sum_k w_k sqrt(N_occ,k) ||F_k^-1 Phi_k||_{2,inf} max_n f_nk ||z_nk||,

w = sqrt|Omega| / sqrt(Ng), z_nk the error of the Sternheimer solution, and
||z_nk|| <= tau^CG_nk / (eps_{N_occ,k + 1,k} - eps_nk) by the proof's bound on
A_n^+.  C_{i,nk} is the tolerance prefactor for which B equals delta when every
CG residual sits at tau^CG = C delta.  The tests build exactly that worst case:
each inexact solution differs from A_n^+ b_n by an error along the eigenvector
of the smallest gap, so that the residual norm equals the tolerance and
||z|| = tolerance / gap.  They then evaluate the true error ||(E - E~) v||
from the oracle's exact and inexact E, and the last line B from pieces computed
here (row norms by numpy's FFT, gaps from the eigenvalues), and check
  error <= delta (the guarantee), B == delta (the prefactor is the one of the
  proof), error >= delta / 1000 (the guarantee is not absurdly strict).
Dropping w_k, an extra N_mp or the real part in place of the full orbitals in
C each move B away from delta; ``test_planted_prefactor_mistakes_are_caught``
plants those mistakes in the oracle's prefactors and checks that they are.

grt (Table strategies_k) is C with three named approximations (Sec. 3.4: the
orbitals' real part, the gaps dropped, and sqrt(N_occ,k) N_mp replaced by
sqrt(N_occ), App. F).  Undoing them turns the grt prefactor back into C
exactly; the real-part row norm itself is pinned by its properties (equal to
the full norm where the orbitals have a real representation, gauge invariant,
strictly smaller at a zone-boundary k-point).
"""
import numpy as np
import pytest

from oracle import gmres, groundstate, response
from workloads import make_system

DELTA = 1e-4


@pytest.fixture(scope="module", params=["tiny_ortho_k", "tiny_metal"])
def kcase(request):
    s = make_system(request.param)
    return s, groundstate.solve(s)


@pytest.fixture(scope="module")
def gamma_case():
    s = make_system("tiny_insulator")
    return s, groundstate.solve(s)


def _row_norm_fft(gs, kb):
    """||F_k^-1 Phi_k||_{2,inf} with the synthesis done by numpy's inverse FFT
    (F^-1 c = |Omega|^-1/2 sum_G c_G e^{iG.r}; ifftn carries a factor 1/Ng)."""
    ng = gs.n_grid
    pad = np.zeros((kb.nocc, ng), dtype=np.complex128)
    pad[:, kb.flat] = kb.vecs[:, :kb.nocc].T
    u = np.fft.ifftn(pad.reshape((kb.nocc,) + tuple(gs.dims)), axes=(1, 2, 3)) * ng / np.sqrt(gs.volume)
    return float(np.sqrt((np.abs(u) ** 2).sum(axis=0)).max())


class _WorstCaseSolver:
    """Stands in for the CG of the oracle: returns A_n^+ b - z with
    z = (tol / gap) e, e the first unoccupied eigenvector, so that
    ||b - A_n x|| = tol and ||z|| = tol / gap (equality in the proof's bound)."""

    def __init__(self):
        self.cache = {}
        self.z_norms = []

    def __call__(self, H, eps_n, Phi, b, tol, kinetic, kappa, maxiter=500):
        key = id(H)
        if key not in self.cache:
            self.cache[key] = np.linalg.eigh(H)
        w, U = self.cache[key]
        no = Phi.shape[1]
        perp = U[:, no:]
        exact = perp @ ((perp.conj().T @ b) / (w[no:] - eps_n))
        gap = w[no] - eps_n
        z = (tol / gap) * U[:, no]
        self.z_norms.append(float(np.linalg.norm(z)))
        return exact - z, 1, float(tol)


def _lemma_check(gs, v, prefactor_fn, monkeypatch):
    """(true error ||(E - E~) v||, last line B of Lemma cgtol_E) for CG
    residuals at tolerance prefactor_fn(||K v||) * DELTA."""
    solver = _WorstCaseSolver()
    monkeypatch.setattr(gmres, "sternheimer_cg", solver)
    exact = response.dielectric(gs, v)
    Kv = response.apply_K(v, gs)
    kvn = float(np.linalg.norm(Kv))
    inexact, _ = gmres.dielectric_inexact(gs, v, lambda nrm: prefactor_fn(nrm) * DELTA)
    monkeypatch.undo()
    err = float(np.linalg.norm(exact - inexact))
    w_inv = np.sqrt(gs.n_grid) / np.sqrt(gs.volume)
    B, s = 0.0, 0
    for kb in gs.kblocks:
        zs = np.array(solver.z_norms[s:s + kb.nocc])
        s += kb.nocc
        B += kb.weight * np.sqrt(kb.nocc) * _row_norm_fft(gs, kb) * float((kb.f[:kb.nocc] * zs).max())
    assert s == len(solver.z_norms)
    return err, 2.0 * w_inv * kvn * B


def _random_v(s, seed=3):
    return np.random.default_rng(seed).normal(size=s.dims)


def test_row_norm_routes_agree(kcase):
    """The oracle's row norm (naive separable DFT) equals numpy's FFT route."""
    s, gs = kcase
    for kb in gs.kblocks:
        a = gmres.orbital_row_norm(gs, kb, False)
        assert abs(a - _row_norm_fft(gs, kb)) <= 1e-12 * a


def test_guaranteed_prefactor_makes_the_lemma_bound_exact(kcase, monkeypatch):
    """Worst-case Sternheimer errors at tau^CG = C_{i,nk} delta: the true error
    of E~ v is at most delta, the lemma's last line equals delta, and the error
    is not below delta/1000."""
    s, gs = kcase
    err, B = _lemma_check(gs, _random_v(s), lambda nrm: gmres.prefactors(gs, "grt_exact", nrm), monkeypatch)
    assert err <= DELTA
    assert abs(B - DELTA) <= 1e-10 * DELTA
    assert err >= DELTA / 1000.0


def _planted(gs, kind):
    """The oracle's prefactors with one plausible mistake planted."""
    nmp = len(gs.kblocks)

    def fn(strategy, nrm):
        p = gmres.prefactors(gs, strategy, nrm).copy()
        q = 0
        for kb in gs.kblocks:
            rc = gmres.orbital_row_norm(gs, kb, False)
            rr = gmres.orbital_row_norm(gs, kb, True)
            for _ in range(kb.nocc):
                if kind == "drop_wk":
                    p[q] *= kb.weight
                elif kind == "extra_nmp":
                    p[q] /= nmp
                elif kind == "swap_norm":          # the other row norm than the rule's own
                    p[q] *= (rc / rr) if strategy == "grt_exact" else (rr / rc)
                q += 1
        return p
    return fn


def _grt_undone(gs, p_grt):
    """The grt prefactors with its three approximations undone: times the gap,
    times ||Re F^-1 Phi_k|| / ||F^-1 Phi_k||, times sqrt(N_occ) / (N_mp sqrt(N_occ,k))."""
    nocc = sum(kb.nocc for kb in gs.kblocks)
    nmp = len(gs.kblocks)
    out = p_grt.copy()
    q = 0
    for kb in gs.kblocks:
        ratio = gmres.orbital_row_norm(gs, kb, True) / gmres.orbital_row_norm(gs, kb, False)
        for n in range(kb.nocc):
            out[q] *= (kb.eps[kb.nocc] - kb.eps[n]) * ratio * np.sqrt(nocc) / (nmp * np.sqrt(kb.nocc))
            q += 1
    return out


def test_grt_is_the_guaranteed_prefactor_with_its_approximations(kcase):
    """Undoing grt's approximations gives C_{i,nk} to rounding."""
    s, gs = kcase
    for nrm in (0.7, 3.0):
        exact = gmres.prefactors(gs, "grt_exact", nrm)
        np.testing.assert_allclose(_grt_undone(gs, gmres.prefactors(gs, "grt", nrm)), exact, rtol=1e-12)


def test_planted_prefactor_mistakes_are_caught(kcase, monkeypatch):
    """Each planted mistake in the grt_exact prefactor moves the lemma's last
    line off delta by more than 1e-3 relative; in the grt prefactor it breaks
    the undo identity by as much."""
    s, gs = kcase
    v = _random_v(s)
    for kind in ("drop_wk", "extra_nmp", "swap_norm"):
        fn = _planted(gs, kind)
        _, B = _lemma_check(gs, v, lambda nrm: fn("grt_exact", nrm), monkeypatch)
        assert abs(B - DELTA) > 1e-3 * DELTA, kind
        exact = gmres.prefactors(gs, "grt_exact", 1.3)
        undone = _grt_undone(gs, fn("grt", 1.3))
        assert np.abs(undone / exact - 1.0).max() > 1e-3, kind


def test_real_part_loses_nothing_where_the_orbitals_are_real(gamma_case):
    """At Gamma with a real potential each orbital is real up to a phase: in the
    most-real gauge the real-part row norm equals the full one (Sec. "Dropping
    the imaginary part of the orbitals")."""
    s, gs = gamma_case
    kb = gs.kblocks[0]
    a, b = gmres.orbital_row_norm(gs, kb, False), gmres.orbital_row_norm(gs, kb, True)
    assert abs(a - b) <= 1e-10 * a


def test_real_part_row_norm_is_gauge_invariant(kcase, gamma_case):
    """Random phases on the eigenvectors change neither row norm."""
    rng = np.random.default_rng(11)
    for s, gs in (kcase, gamma_case):
        for kb in gs.kblocks:
            ref = (gmres.orbital_row_norm(gs, kb, False), gmres.orbital_row_norm(gs, kb, True))
            saved = kb.vecs
            kb.vecs = saved * np.exp(2j * np.pi * rng.random(saved.shape[1]))[None, :]
            try:
                got = (gmres.orbital_row_norm(gs, kb, False), gmres.orbital_row_norm(gs, kb, True))
            finally:
                kb.vecs = saved
            np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_real_part_is_smaller_at_the_zone_boundary(kcase):
    """At k = b1/2 the lattice-periodic parts u_nk = e^{-ik.r} psi_nk are not real
    in any gauge: the real-part row norm is strictly below the full one, and the
    full one lies in the bounds of Proposition FinvPhi_bound."""
    s, gs = kcase
    kb = [b for b in gs.kblocks if np.linalg.norm(b.kfrac) > 0][0]
    a, b = gmres.orbital_row_norm(gs, kb, False), gmres.orbital_row_norm(gs, kb, True)
    assert b < a * (1.0 - 1e-3)
    assert b > 0.5 * a
    for kb in gs.kblocks:
        r = gmres.orbital_row_norm(gs, kb, False)
        assert np.sqrt(kb.nocc / gs.volume) <= r * (1 + 1e-12)
        assert r <= np.sqrt(gs.n_grid / gs.volume) * (1 + 1e-12)
