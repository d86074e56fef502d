"""Writes cfg1_bal_fp64.txt and cfg1_bal_schur_fp64.txt: the oracle's
Algorithm 1 on the 10-bohr Gamma-point cell (cfg1: 32^3 grid, 4 occupied bands,
6 computed), b = chi0 dV0 / ||chi0 dV0||, bal, tau = 1e-8, m = 20, with the
plain projected CG and with the Schur-complement form over bands 5 and 6
(Sec. 3.4.2): GMRES steps, restarts, N_ham, true residual and the residual
estimates of every step.  Calls only oracle/ and workloads/:
python tests/golden/make_cfg1_traces.py"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import groundstate, gmres, response  # noqa: E402
from workloads import make_system, perturbation  # noqa: E402


def _write(name, title, r, true):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {title}; written by tests/golden/make_cfg1_traces.py\n")
        f.write(f"steps {r.steps}\nrestarts {r.restarts}\nn_ham {r.nham}\ntrue_residual {true:.6e}\n")
        f.write("history " + " ".join(f"{v:.9e}" for v in r.estimated) + "\n")


def main():
    s = make_system("cfg1")
    gs = groundstate.solve(s)
    kxc = response.exchange_kernel(gs.rho)
    b = response.chi0(gs, perturbation(s))
    b /= np.linalg.norm(b)
    for schur, name in ((0, "cfg1_bal_fp64.txt"), (s.nbands, "cfg1_bal_schur_fp64.txt")):
        r = gmres.inexact_gmres(gs, b, 1e-8, 20, "bal", kxc=kxc, schur_nbands=schur)
        true = float(np.linalg.norm(b - response.dielectric(gs, r.x, kxc)))
        title = "Algorithm 1 (oracle emulation, FP64), cfg1, bal, tau = 1e-8, m = 20"
        if schur:
            title += f", Schur-complement CG over bands {max(k.nocc for k in gs.kblocks) + 1}..{schur}"
        _write(name, title, r, true)


if __name__ == "__main__":
    main()
