"""Writes cfg2_bal_fp64.txt: the oracle's Algorithm 1 on the diamond-like cell
(cfg2: 48^3 grid, 2x2x2 k-points, 251 Sternheimer systems per E application),
b = chi0 dV0 / ||chi0 dV0|| for the workload's Gaussian bump, bal tolerances,
tau = 1e-8, m = 20: the GMRES step count, restarts, N_ham (CG iterations with
the kinetic preconditioner of the projected CG), the true residual and the
residual estimates ||r~_i|| of every step.  Calls only oracle/ and workloads/
(several minutes of CPU):  python tests/golden/make_cfg2_bal.py"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import groundstate, gmres, response  # noqa: E402
from workloads import make_system, perturbation  # noqa: E402


def main():
    s = make_system("cfg2")
    gs = groundstate.solve(s)
    kxc = response.exchange_kernel(gs.rho)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    r = gmres.inexact_gmres(gs, b, 1e-8, 20, "bal", kxc=kxc)
    true = float(np.linalg.norm(b - response.dielectric(gs, r.x, kxc)))
    with open(os.path.join(HERE, "cfg2_bal_fp64.txt"), "w") as f:
        f.write("# Algorithm 1 (oracle emulation, FP64), cfg2, bal, tau = 1e-8, m = 20; "
                "written by tests/golden/make_cfg2_bal.py\n")
        f.write(f"steps {r.steps}\nrestarts {r.restarts}\nn_ham {r.nham}\ntrue_residual {true:.6e}\n")
        f.write("history " + " ".join(f"{v:.9e}" for v in r.estimated) + "\n")


if __name__ == "__main__":
    main()
