"""The synthetic inputs: the displacement perturbation is the derivative of the
pseudo-atom potential with respect to the atom position (central difference)."""
import numpy as np

from workloads import make_system, perturbation, gaussian_sum_on_grid


def test_displacement_is_potential_derivative():
    s = make_system("tiny_insulator")
    h = 1e-5
    for atom, axis in [(0, 0), (1, 2)]:
        dV = perturbation(s, "displacement", atom=atom, axis=axis)
        pos_p = s.positions.copy()
        pos_m = s.positions.copy()
        pos_p[atom, axis] += h
        pos_m[atom, axis] -= h
        Vp = gaussian_sum_on_grid(s.lattice, s.dims, pos_p, -s.depth, s.width)
        Vm = gaussian_sum_on_grid(s.lattice, s.dims, pos_m, -s.depth, s.width)
        np.testing.assert_allclose(dV, (Vp - Vm) / (2 * h), atol=1e-7)
