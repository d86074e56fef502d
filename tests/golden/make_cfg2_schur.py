"""Writes cfg2_bal_schur_fp64.txt: as make_cfg2_bal.py (cfg2, bal, tau = 1e-8,
m = 20), with the Schur-complement Sternheimer solves over the workload's
computed bands above N_occ,k (bands up to 36; Sec. 3.4.2).  Calls only
oracle/ and workloads/ (several minutes of CPU):
python tests/golden/make_cfg2_schur.py"""
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
    r = gmres.inexact_gmres(gs, b, 1e-8, 20, "bal", kxc=kxc, schur_nbands=s.nbands)
    true = float(np.linalg.norm(b - response.dielectric(gs, r.x, kxc)))
    with open(os.path.join(HERE, "cfg2_bal_schur_fp64.txt"), "w") as f:
        f.write(f"# Algorithm 1 (oracle emulation, FP64), cfg2, bal, tau = 1e-8, m = 20, Schur-complement CG "
                f"over the bands above N_occ,k up to {s.nbands}; written by tests/golden/make_cfg2_schur.py\n")
        f.write(f"steps {r.steps}\nrestarts {r.restarts}\nn_ham {r.nham}\ntrue_residual {true:.6e}\n")
        f.write("history " + " ".join(f"{v:.9e}" for v in r.estimated) + "\n")


if __name__ == "__main__":
    main()
