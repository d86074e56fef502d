"""Supercells: Bloch folding identities and the size scaling of the CG
tolerance prefactors (Remark rmk:scaling), checked on the oracle.

Pins that come from outside the oracle's own formulas:

* Folding (Bloch's theorem).  A supercell of ell replicas along a_1, sampled at
  the k-points of its own grid (l1, l2, l3), is the same crystal as the small
  cell on the grid (ell l1, l2, l3): the occupied eigenvalues are the union of
  the small cell's, the Fermi level and the density agree (the density tiled),
  and a perturbation with the small cell's period has the tiled response.  The
  two sides share no k-point: a wrong Bloch phase, k-shift, k-weight,
  Fermi-level or projector Bloch sum breaks the identity.
* Remark rmk:scaling: |Omega|, N_occ and N_g grow linearly with ell, the gap,
  ||K v|| and ||F^{-1} Phi||_{2,inf} stay roughly constant, so the prefactors
  of the bal and grt strategies and the exact C_{i,n} fall like 1/sqrt(ell).
  A dropped or misplaced |Omega|, N_g or N_occ factor changes that power by
  +-1/2, i.e. by a factor 1.41 at ell = 2 and 2 at ell = 4.
"""
import numpy as np
import pytest

from oracle import groundstate as ogs, response as oresp, gmres as og
from workloads import make_system, supercell, with_kgrid, perturbation, gaussian_sum_on_grid


def _occupied(gs):
    return np.sort(np.concatenate([kb.eps[:kb.nocc] for kb in gs.kblocks]))


def test_supercell_geometry_matches_a_direct_construction():
    P = make_system("tiny_ortho_k")
    S = supercell(P, 3, kgrid=(1, 1, 1))
    assert S.dims == (3 * P.dims[0], P.dims[1], P.dims[2])
    assert np.allclose(S.lattice[:, 0], 3 * P.lattice[:, 0])
    assert np.allclose(S.lattice[:, 1:], P.lattice[:, 1:])
    assert (S.n_electrons, S.nbands) == (3 * P.n_electrons, 3 * P.nbands)
    assert len(S.positions) == 3 * len(P.positions)
    # the tiled potential is the Gaussian sum of the replicated atoms evaluated
    # on the supercell grid directly
    direct = gaussian_sum_on_grid(S.lattice, S.dims, S.positions, -P.depth, P.width)
    assert np.abs(direct - S.V).max() < 1e-12 * np.abs(direct).max()
    assert S.kgrid == (1, 1, 1) and np.allclose(S.kpoints, 0.0)
    # default: the k-point density is kept
    assert supercell(P, 2).kgrid == (1, 1, 1)
    with pytest.raises(ValueError):
        supercell(P, 3)


@pytest.mark.parametrize("name", ["tiny_ortho_k", "tiny_metal", "tiny_kb"])
def test_two_replicas_fold_onto_the_two_point_k_grid(name):
    P = make_system(name)                    # k-grid (2, 1, 1)
    S = supercell(P, 2)                      # Gamma only
    assert P.kgrid == (2, 1, 1) and S.kgrid == (1, 1, 1)
    gp, gsS = ogs.solve(P), ogs.solve(S)
    occP, occS = _occupied(gp), _occupied(gsS)
    assert len(occP) == len(occS)
    assert np.abs(occP - occS).max() < 1e-11
    assert abs(gp.eF - gsS.eF) < 1e-11
    rho_t = np.tile(gp.rho, (2, 1, 1))
    assert np.abs(rho_t - gsS.rho).max() < 1e-12 * np.abs(rho_t).max()
    dV = perturbation(P)
    c_p = oresp.chi0(gp, dV)
    c_s = oresp.chi0(gsS, np.tile(dV, (2, 1, 1)))
    assert np.linalg.norm(np.tile(c_p, (2, 1, 1)) - c_s) < 1e-11 * np.linalg.norm(c_s)
    # the dielectric operator E = 1 - chi0 K on a tiled vector
    e_p = oresp.dielectric(gp, c_p)
    e_s = oresp.dielectric(gsS, np.tile(c_p, (2, 1, 1)))
    assert np.linalg.norm(np.tile(e_p, (2, 1, 1)) - e_s) < 1e-11 * np.linalg.norm(e_s)


def test_three_replicas_fold_onto_a_three_point_k_grid():
    P = make_system("tiny_insulator")        # Gamma only
    P3 = with_kgrid(P, (3, 1, 1))            # k = 0, +-1/3 along b_1
    S = supercell(P, 3, kgrid=(1, 1, 1))
    g3, gsS = ogs.solve(P3), ogs.solve(S)
    assert np.abs(_occupied(g3) - _occupied(gsS)).max() < 1e-11
    rho_t = np.tile(g3.rho, (3, 1, 1))
    assert np.abs(rho_t - gsS.rho).max() < 1e-12 * np.abs(rho_t).max()
    dV = perturbation(P)
    c3 = oresp.chi0(g3, dV)
    cs = oresp.chi0(gsS, np.tile(dV, (3, 1, 1)))
    assert np.linalg.norm(np.tile(c3, (3, 1, 1)) - cs) < 1e-11 * np.linalg.norm(cs)
    # and the Gamma-only small cell is a different crystal sampling: its density differs
    assert np.abs(np.tile(ogs.solve(P).rho, (3, 1, 1)) - gsS.rho).max() > 1e-6


@pytest.mark.parametrize("name", ["tiny_insulator", "tiny_ortho_k"])
def test_prefactors_scale_like_inverse_sqrt_of_the_supercell_size(name):
    P = make_system(name)
    gp = ogs.solve(P)
    v = oresp.chi0(gp, perturbation(P))
    base = {}
    for ell in (1, 2, 4):
        gs = ogs.solve(supercell(P, ell, kgrid=(1, 1, 1)))
        vt = np.tile(v, (ell, 1, 1))
        vt /= np.linalg.norm(vt)
        kv = float(np.linalg.norm(oresp.apply_K(vt, gs)))
        assert np.all(og.prefactors(gs, "agr", kv) == 1.0)          # agr ignores the size
        for st in ("bal", "grt", "grt_exact"):
            c = float(og.prefactors(gs, st, kv).min()) * np.sqrt(ell)
            base.setdefault(st, c)
            ratio = c / base[st]
            if st == "bal":
                # |Omega| / (N_occ sqrt(N_g)) with all three linear in ell: exactly 1/sqrt(ell)
                assert abs(ratio - 1.0) < 1e-12, (st, ell, ratio)
            else:
                # gap, ||K v|| and the orbital row norm are only asymptotically constant
                assert 0.8 < ratio < 1.25, (st, ell, ratio)


def test_guaranteed_rules_keep_tau_while_agr_drifts_as_the_cell_grows():
    """Remark rmk:scaling on the oracle's Algorithm 1: replicas of a fine-grid
    insulator at the Gamma point with the same localised bump dV0 in each, b =
    chi0 dV0, tau = 1e-9, m = 10.  grt_exact (the guarantee of Theorem
    inexact_gmres_dyson) and bal end below tau at every size; agr, whose
    prefactor does not shrink with ell, ends further from tau for larger ell;
    and a fixed rule carries no guarantee: D10n (tau / (10 ||b||), ||b|| = 0.12
    here) ends above tau at ell = 4 (the paper's subsection on why a naive static
    tolerance selection can fail: the true residual stalls above tau)."""
    P = make_system("tiny_insulator_fine")
    center = P.lattice @ np.array([0.3, 0.6, 0.45])
    tau, m = 1e-9, 10
    ratio = {}
    for ell in (1, 4):
        S = supercell(P, ell, kgrid=(1, 1, 1))
        gs = ogs.solve(S)
        b = oresp.chi0(gs, perturbation(S, center=center))
        kxc = oresp.exchange_kernel(gs.rho)
        for st in ("agr", "bal", "grt_exact") + (("D10n",) if ell == 4 else ()):
            r = og.inexact_gmres(gs, b, tau, m, st, kxc=kxc)
            assert r.converged
            ratio[st, ell] = float(np.linalg.norm(b - oresp.dielectric(gs, r.x, kxc))) / tau
    for ell in (1, 4):
        assert ratio["grt_exact", ell] < 1.0 and ratio["bal", ell] < 1.0, ratio
    assert ratio["agr", 4] > 1.5 * ratio["agr", 1], ratio
    assert ratio["agr", 4] > 3.0 * ratio["grt_exact", 4], ratio
    assert ratio["D10n", 4] > 1.0 > ratio["grt_exact", 4], ratio
