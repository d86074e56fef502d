"""Algorithm 1 step by step at the benchmark size (cfg2: 48^3 grid, 2 x 2 x 2
k-points, 251 Sternheimer systems per E application, bal, tau = 1e-8, m = 20).

The FP64 GPU solve against the oracle's emulation of the same algorithm
(tests/golden/cfg2_bal_fp64.txt, written by make_cfg2_bal.py from oracle/
only): the same number of GMRES steps and restarts, the same residual
estimates ||r~_i|| step by step, the same number of Hamiltonian applications
(the CG iteration counts of every Sternheimer solve of every E application,
summed), and a true residual below tau.  Agreement of the iteration counts
shows that the GPU's projected CG, its preconditioner and the tolerance rule
follow the oracle's, not only that the answers agree."""
import os

import numpy as np
import pytest

import gpu_common
from gpu_common import context, dev, system, torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg2_bal_fp64.txt")


def _golden(path=GOLDEN):
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals] if key == "history" else float(vals[0])
    return out


def test_fp64_solve_follows_the_oracle_step_by_step():
    from workloads import perturbation
    g = _golden()
    s = system("cfg2")
    ctx = context("cfg2")
    nsys = ctx.groundstate_nsys
    b, _ = ctx.apply_chi0(dev(perturbation(s)), tol=np.full(nsys, 1e-12))
    b = (b / torch.linalg.norm(b)).contiguous()
    x, rep = ctx.solve_response(b, tau=1e-8, m=20, strategy="bal")
    r = rep[0]
    assert r["status"] == 0
    assert r["outer_iters"] == int(g["steps"]) and r["restarts"] == int(g["restarts"])
    assert abs(r["n_ham"] - g["n_ham"]) <= 0.005 * g["n_ham"], (r["n_ham"], g["n_ham"])
    hist = np.array(r["history"][:len(g["history"])])
    ref = np.array(g["history"])
    assert len(hist) == len(ref)
    # the estimates agree to the CG truncation of the E applications (tau-level, relative to ||r~||)
    assert np.all(np.abs(hist - ref) <= 1e-3 * ref + 1e-9), np.max(np.abs(hist - ref) / ref)
    Ex, _ = ctx.apply_dielectric(x, tol=np.full(nsys, 1e-12))
    assert float(torch.linalg.norm(b - Ex)) <= 1e-8


@pytest.mark.parametrize("schur", [False, True])
def test_cfg1_fp64_solve_follows_the_oracle(schur):
    """The 10-bohr cell (cfg1), bal, with the plain projected CG and with the
    Schur-complement form over its two computed bands above N_occ: for exact
    eigenvectors both sides iterate on R (H - eps) R with the same right-hand
    side and preconditioner, so the traces agree."""
    from paper_2505_02319_gb300 import groundstate
    from workloads import perturbation
    name = "cfg1_bal_schur_fp64.txt" if schur else "cfg1_bal_fp64.txt"
    g = _golden(os.path.join(os.path.dirname(GOLDEN), name))
    s = system("cfg1")
    ctx = gpu_common.dense_context_for(s, schur=schur)
    nsys = ctx.groundstate_nsys
    b, _ = ctx.apply_chi0(dev(perturbation(s)), tol=np.full(nsys, 1e-12))
    b = (b / torch.linalg.norm(b)).contiguous()
    x, rep = ctx.solve_response(b, tau=1e-8, m=20, strategy="bal")
    r = rep[0]
    assert r["outer_iters"] == int(g["steps"]) and r["restarts"] == int(g["restarts"])
    assert abs(r["n_ham"] - g["n_ham"]) <= 0.005 * g["n_ham"], (r["n_ham"], g["n_ham"])
    hist, ref = np.array(r["history"]), np.array(g["history"])
    assert len(hist) == len(ref)
    assert np.all(np.abs(hist - ref) <= 1e-3 * ref + 1e-9), np.max(np.abs(hist - ref) / ref)
    Ex, _ = ctx.apply_dielectric(x, tol=np.full(nsys, 1e-12))
    tr = float(torch.linalg.norm(b - Ex))
    assert abs(tr - g["true_residual"]) <= 0.05 * g["true_residual"] + 1e-10
    ctx.destroy()


def test_metallic_slab_kerker_solve_follows_the_oracle():
    """The metallic slab at a reduced cut-off (cfg3's atoms, Ecut 2.5 Ha,
    12 x 12 x 64, 2 x 2 x 1 k, N_occ,k 68-76), bal with the Kerker
    preconditioner: the dphi^P and Fermi-level terms of the metal and the left
    preconditioner T, trace against the oracle's."""
    from oracle import response
    from paper_2505_02319_gb300 import groundstate
    from workloads import make_system, perturbation, with_cutoff, with_kgrid
    g = _golden(os.path.join(os.path.dirname(GOLDEN), "slab_bal_kerker_fp64.txt"))
    s = with_cutoff(with_kgrid(make_system("cfg3"), (2, 2, 1)), 2.5, (12, 12, 64))
    ctx = gpu_common.dense_context_for(s)
    nsys = ctx.groundstate_nsys
    b, _ = ctx.apply_chi0(dev(perturbation(s)), tol=np.full(nsys, 1e-12))
    b = (b / torch.linalg.norm(b)).contiguous()
    alpha = 0.8
    x, rep = ctx.solve_response(b, tau=1e-8, m=20, strategy="bal", kerker_alpha=alpha)
    r = rep[0]
    assert r["outer_iters"] == int(g["steps"]) and r["restarts"] == int(g["restarts"])
    assert abs(r["n_ham"] - g["n_ham"]) <= 0.005 * g["n_ham"], (r["n_ham"], g["n_ham"])
    hist, ref = np.array(r["history"]), np.array(g["history"])
    assert len(hist) == len(ref)
    assert np.all(np.abs(hist - ref) <= 1e-3 * ref + 1e-9), np.max(np.abs(hist - ref) / ref)
    Ex, _ = ctx.apply_dielectric(x, tol=np.full(nsys, 1e-12))
    res = (b - Ex).cpu().numpy().reshape(s.dims)
    tr = float(np.linalg.norm(response.kerker(res, s.lattice, s.dims, alpha)))
    assert tr <= 1e-8 and abs(tr - g["true_residual"]) <= 0.05 * g["true_residual"] + 1e-10
    ctx.destroy()


def test_cfg2_schur_fp64_solve_follows_the_oracle():
    """The bench problem with the Schur-complement solves over its 36 computed
    bands: the trace of the oracle's Schur CG (11 % fewer Hamiltonian
    applications than the plain CG)."""
    from paper_2505_02319_gb300 import groundstate
    from workloads import perturbation
    g = _golden(os.path.join(os.path.dirname(GOLDEN), "cfg2_bal_schur_fp64.txt"))
    s = system("cfg2")
    ctx = gpu_common.dense_context_for(s, schur=True)
    nsys = ctx.groundstate_nsys
    b, _ = ctx.apply_chi0(dev(perturbation(s)), tol=np.full(nsys, 1e-12))
    b = (b / torch.linalg.norm(b)).contiguous()
    x, rep = ctx.solve_response(b, tau=1e-8, m=20, strategy="bal")
    r = rep[0]
    assert r["outer_iters"] == int(g["steps"]) and r["restarts"] == int(g["restarts"])
    assert abs(r["n_ham"] - g["n_ham"]) <= 0.005 * g["n_ham"], (r["n_ham"], g["n_ham"])
    hist, ref = np.array(r["history"]), np.array(g["history"])
    assert len(hist) == len(ref)
    assert np.all(np.abs(hist - ref) <= 1e-3 * ref + 1e-9), np.max(np.abs(hist - ref) / ref)
    ctx.destroy()
