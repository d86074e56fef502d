"""Writes slab_bal_kerker_fp64.txt: the oracle's Algorithm 1 on the metallic
slab (cfg3's atoms) at a reduced cut-off (Ecut 2.5 Ha, 12 x 12 x 64 grid,
2 x 2 x 1 k-points, N_occ,k = 68-76), b = chi0 dV0 / ||chi0 dV0||, bal, left
Kerker preconditioner alpha = 0.8 (eq. precond_dyson), tau = 1e-8, m = 20:
GMRES steps, restarts, N_ham, the true preconditioned residual ||T r|| and
the residual estimates of every step.  Calls only oracle/ and workloads/:
python tests/golden/make_slab_trace.py"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import groundstate, gmres, response  # noqa: E402
from workloads import make_system, perturbation, with_cutoff, with_kgrid  # noqa: E402


def main():
    s = with_cutoff(with_kgrid(make_system("cfg3"), (2, 2, 1)), 2.5, (12, 12, 64))
    gs = groundstate.solve(s)
    kxc = response.exchange_kernel(gs.rho)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    alpha = 0.8
    r = gmres.inexact_gmres(gs, b, 1e-8, 20, "bal", kxc=kxc, kerker_alpha=alpha)
    res = b - response.dielectric(gs, r.x, kxc)
    true = float(np.linalg.norm(response.kerker(res, s.lattice, s.dims, alpha)))
    with open(os.path.join(HERE, "slab_bal_kerker_fp64.txt"), "w") as f:
        f.write("# Algorithm 1 (oracle emulation, FP64), cfg3 slab at Ecut 2.5 Ha, 12x12x64, 2x2x1 k, bal, "
                "Kerker 0.8, tau = 1e-8, m = 20; written by tests/golden/make_slab_trace.py\n")
        f.write(f"steps {r.steps}\nrestarts {r.restarts}\nn_ham {r.nham}\ntrue_residual {true:.6e}\n")
        f.write("history " + " ".join(f"{v:.9e}" for v in r.estimated) + "\n")


if __name__ == "__main__":
    main()
