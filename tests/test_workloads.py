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


def test_with_cutoff_keeps_the_atoms_and_resamples_the_potential():
    import numpy as np
    from workloads import gaussian_sum_on_grid, make_system, with_cutoff
    s = make_system("tiny_ortho_k")
    r = with_cutoff(s, 6.0, (20, 24, 32))
    assert r.dims == (20, 24, 32) and r.Ecut == 6.0
    assert np.array_equal(r.positions, s.positions) and np.array_equal(r.kpoints, s.kpoints)
    assert (r.n_electrons, r.nbands, r.temperature) == (s.n_electrons, s.nbands, s.temperature)
    direct = gaussian_sum_on_grid(s.lattice, (20, 24, 32), s.positions, -s.depth, s.width)
    assert np.array_equal(r.V, direct)
    # the coarse grid's points are a subset of the fine one's: the potential agrees there
    assert np.allclose(r.V[::2, ::2, ::2], s.V, atol=1e-12)


def test_separable_gaussian_sum_equals_the_image_sum():
    """For an orthorhombic cell the product of the three axis image sums is the
    sum over the image box (same terms, another order)."""
    import math
    from workloads.systems import _gaussian_sum_images
    for name, dims in (("tiny_ortho_k", (10, 12, 16)), ("cfg2", (24, 24, 24))):
        s = make_system(name)
        reach = 9.0 * s.width
        nimg = [int(math.ceil(reach / np.linalg.norm(s.lattice[:, i]))) + 1 for i in range(3)]
        fast = gaussian_sum_on_grid(s.lattice, dims, s.positions, -s.depth, s.width)
        slow = _gaussian_sum_images(s.lattice, dims, s.positions, -s.depth, s.width, nimg)
        np.testing.assert_allclose(fast, slow, rtol=1e-13, atol=1e-14 * np.abs(slow).max())
