"""Seeded synthetic systems shaped like the paper's workloads.

The paper's experiments (Sec. 4: an aluminium supercell, a Heusler alloy and
silicon, all with GTH pseudopotentials and PBE) cannot be reproduced without
DFTK and its pseudopotential files.  These systems stand in for them: a
local external potential made of attractive Gaussian pseudo-atoms,
``V(r) = -D * sum_a sum_R exp(-|r - R_a - R|^2 / (2 sigma^2))``, sampled on
the real-space grid X of Sec. 2.3.1, a Gamma-centred Monkhorst-Pack k-grid
(Sec. 4.1.1) and a Gaussian-bump perturbation dV0.

Conventions (shared with the C ABI, see include/ikr.h):
  * ``lattice`` is 3x3 with the cell vectors a_1, a_2, a_3 as COLUMNS (bohr).
  * Real-space arrays have shape (N1, N2, N3) in C order; point (i1,i2,i3) is
    r = i1/N1 a_1 + i2/N2 a_2 + i3/N3 a_3.
  * k-points are fractional coordinates in the reciprocal basis b_1, b_2, b_3.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np


@dataclasses.dataclass
class System:
    name: str
    lattice: np.ndarray          # (3,3) columns are cell vectors [bohr]
    dims: tuple                  # FFT grid (N1, N2, N3)
    Ecut: float                  # kinetic-energy cut-off [Ha]
    kpoints: np.ndarray          # (Nk, 3) fractional reciprocal coordinates
    kweights: np.ndarray         # (Nk,) weights summing to 1
    V: np.ndarray                # (N1,N2,N3) external potential on the grid [Ha]
    n_electrons: int             # total electron count N
    temperature: float           # smearing T [Ha]; 0 => insulator, f = 2 for N/2 bands
    nbands: int                  # eigenpairs requested per k-point
    positions: np.ndarray        # (Natom, 3) Cartesian atom positions [bohr]
    depth: float
    width: float
    seed: int
    # Kleinman-Bylander nonlocal projectors (or None): a Gaussian s and p channel
    # on every centre, kb_sigma[l] their widths [bohr] and kb_D[l] their coupling
    # energies [Ha] (the projector functions themselves are defined where they
    # are used: the oracle and the GPU setup)
    kb_centers: np.ndarray = None   # (Nkb, 3) Cartesian [bohr]
    kb_sigma: tuple = None          # (sigma_s, sigma_p)
    kb_D: tuple = None              # (D_s, D_p)
    kgrid: tuple = (1, 1, 1)        # Monkhorst-Pack counts (l1, l2, l3) behind kpoints

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    @property
    def n_grid(self) -> int:
        return int(np.prod(self.dims))


def monkhorst_pack(grid):
    """Gamma-centred, unshifted MP grid k = sum_i (j_i / l_i) b_i with equal
    weights 1/(l1 l2 l3) (Sec. 4.1.1; no symmetry reduction), folded to
    fractional coordinates in [-1/2, 1/2)."""
    ks = []
    for j in itertools.product(*[range(l) for l in grid]):
        k = np.array([jj / l for jj, l in zip(j, grid)], dtype=np.float64)
        k = k - np.floor(k + 0.5)
        ks.append(k)
    ks = np.array(ks)
    w = np.full(len(ks), 1.0 / len(ks))
    return ks, w


def _grid_points(lattice, dims):
    fr = [np.arange(n) / n for n in dims]
    f1, f2, f3 = np.meshgrid(*fr, indexing="ij")
    frac = np.stack([f1, f2, f3], axis=-1)          # (N1,N2,N3,3)
    return frac @ lattice.T                          # Cartesian


def gaussian_sum_on_grid(lattice, dims, centers, amplitude, width):
    """sum_c sum_R amplitude * exp(-|r - c - R|^2 / (2 width^2)) on the grid,
    with enough periodic images R for the tail to fall below 1e-16.

    For an orthorhombic cell the images R = sum_a n_a a_a form a product set
    and the Gaussian is a product over the Cartesian axes, so the image sum is
    the product of three one-dimensional image sums (the same terms, summed in
    another order); other cells take the direct sum over images."""
    reach = 9.0 * width
    nimg = [int(math.ceil(reach / np.linalg.norm(lattice[:, i]))) + 1 for i in range(3)]
    lattice = np.asarray(lattice, dtype=np.float64)
    if np.array_equal(lattice, np.diag(np.diag(lattice))):
        out = np.zeros(dims, dtype=np.float64)
        L = np.diag(lattice)
        x = [np.arange(n) / n * L[a] for a, n in enumerate(dims)]
        for c in np.atleast_2d(centers):
            g = []
            for a in range(3):
                n = np.arange(-nimg[a], nimg[a] + 1, dtype=np.float64)
                d = x[a][:, None] - (c[a] + n[None, :] * L[a])
                g.append(np.exp(-d * d / (2.0 * width * width)).sum(axis=1))
            out += amplitude * (g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :])
        return out
    return _gaussian_sum_images(lattice, dims, centers, amplitude, width, nimg)


def _gaussian_sum_images(lattice, dims, centers, amplitude, width, nimg):
    """The direct sum over the periodic images (any cell)."""
    r = _grid_points(lattice, dims)
    out = np.zeros(dims, dtype=np.float64)
    for c in np.atleast_2d(centers):
        for n in itertools.product(*[range(-m, m + 1) for m in nimg]):
            shift = lattice @ np.array(n, dtype=np.float64)
            d = r - (c + shift)
            d2 = np.einsum("...i,...i->...", d, d)
            out += amplitude * np.exp(-d2 / (2.0 * width * width))
    return out


def _random_positions(rng, lattice, natoms, min_sep):
    pos = []
    inv = np.linalg.inv(lattice)
    while len(pos) < natoms:
        p = lattice @ rng.random(3)
        ok = True
        for q in pos:
            d = inv @ (p - q)
            d -= np.round(d)
            if np.linalg.norm(lattice @ d) < min_sep:
                ok = False
                break
        if ok:
            pos.append(p)
    return np.array(pos)


def make_system(name: str) -> System:
    """Build one of the named synthetic systems (see CONFIGS / TEST_SYSTEMS)."""
    spec = dict(_SPECS[name])
    seed = spec["seed"]
    rng = np.random.default_rng(seed)
    lattice = np.diag(spec["cell"]).astype(np.float64)
    if spec["layout"] == "random":
        positions = _random_positions(rng, lattice, spec["natoms"], spec["min_sep"])
    elif spec["layout"] == "diamond":
        a = spec["cell"][0]
        fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
        basis = np.concatenate([fcc, fcc + 0.25]) * a
        positions = basis + rng.normal(0.0, spec["jitter"], size=basis.shape)
    elif spec["layout"] == "slab":
        Lx, Ly, _ = spec["cell"]
        pts = []
        for z in spec["layers"]:
            for i, j in itertools.product(range(2), range(2)):
                pts.append([(i + 0.25) * Lx / 2, (j + 0.25) * Ly / 2, z])
        positions = np.array(pts) + rng.normal(0.0, spec["jitter"], size=(len(pts), 3))
    elif spec["layout"] == "cubic_lattice":
        n = spec["per_side"]
        a = spec["cell"][0] / n
        pts = [[(i + .5) * a, (j + .5) * a, (k + .5) * a]
               for i, j, k in itertools.product(range(n), repeat=3)]
        positions = np.array(pts) + rng.normal(0.0, spec["jitter"], size=(n ** 3, 3))
    else:
        raise ValueError(spec["layout"])
    dims = tuple(spec["dims"])
    V = gaussian_sum_on_grid(lattice, dims, positions, -spec["depth"], spec["width"])
    kpts, kw = monkhorst_pack(spec.get("kgrid", (1, 1, 1)))
    kb = spec.get("kb")
    return System(name=name, lattice=lattice, dims=dims, Ecut=float(spec["Ecut"]),
                  kpoints=kpts, kweights=kw, V=V, n_electrons=int(spec["n_electrons"]),
                  temperature=float(spec.get("T", 0.0)), nbands=int(spec["nbands"]),
                  positions=positions, depth=float(spec["depth"]),
                  width=float(spec["width"]), seed=seed,
                  kb_centers=positions.copy() if kb else None,
                  kb_sigma=tuple(kb["sigma"]) if kb else None,
                  kb_D=tuple(kb["D"]) if kb else None,
                  kgrid=tuple(spec.get("kgrid", (1, 1, 1))))


def with_kgrid(system: System, kgrid) -> System:
    """The same cell and potential on another Gamma-centred MP k-grid."""
    kpts, kw = monkhorst_pack(kgrid)
    name = f"{system.name}_k{'x'.join(str(int(l)) for l in kgrid)}"
    return dataclasses.replace(system, name=name, kpoints=kpts, kweights=kw,
                               kgrid=tuple(int(l) for l in kgrid))


def with_cutoff(system: System, Ecut: float, dims) -> System:
    """The same atoms, k-points and counts at another cut-off and FFT grid (the
    potential evaluated on the new grid), for reduced-size versions of a workload."""
    dims = tuple(int(n) for n in dims)
    V = gaussian_sum_on_grid(system.lattice, dims, system.positions, -system.depth, system.width)
    return dataclasses.replace(system, name=f"{system.name}_E{Ecut:g}", Ecut=float(Ecut), dims=dims, V=V)


def supercell(system: System, ell: int, axis: int = 0, kgrid=None) -> System:
    """The supercell of `ell` replicas of `system` along cell vector `axis`
    (the construction of Remark rmk:scaling): a_axis -> ell a_axis, N_axis ->
    ell N_axis, the external potential tiled (it is periodic in the small
    cell, so tiling is exact), atoms and projector centres replicated at
    R + j a_axis, and the electron and band counts multiplied by ell.

    k-grid: by default the k-point density is kept, i.e. l_axis -> l_axis/ell,
    which needs ell to divide l_axis; otherwise pass `kgrid`.  A supercell on
    grid (l1, l2, l3) describes the same crystal as the small cell on the grid
    with l_axis replaced by ell * l_axis (band folding, Bloch's theorem).
    """
    ell = int(ell)
    if ell < 1 or axis not in (0, 1, 2):
        raise ValueError("ell must be >= 1 and axis one of 0, 1, 2")
    if kgrid is None:
        kg = list(system.kgrid)
        if kg[axis] % ell:
            raise ValueError(f"k-grid {system.kgrid} cannot be folded by {ell} along axis {axis}; pass kgrid")
        kg[axis] //= ell
        kgrid = tuple(kg)
    lattice = system.lattice.copy()
    a = system.lattice[:, axis].copy()
    lattice[:, axis] = ell * a
    dims = list(system.dims)
    dims[axis] *= ell
    reps = [1, 1, 1]
    reps[axis] = ell
    V = np.tile(system.V, reps)

    def replicate(p):
        return None if p is None else np.concatenate([p + j * a for j in range(ell)])

    kpts, kw = monkhorst_pack(kgrid)
    return dataclasses.replace(
        system, name=f"{system.name}_x{ell}", lattice=lattice, dims=tuple(dims), V=V,
        kpoints=kpts, kweights=kw, kgrid=tuple(int(l) for l in kgrid),
        n_electrons=ell * system.n_electrons, nbands=ell * system.nbands,
        positions=replicate(system.positions), kb_centers=replicate(system.kb_centers))


def perturbation(system: System, kind: str = "bump", seed: int = 0,
                 amplitude: float = 0.1, width: float = 1.0, atom: int = 0, axis: int = 0,
                 center=None) -> np.ndarray:
    """A seeded local perturbation dV0 on the grid.

    kind="bump": a periodic Gaussian bump of the given amplitude [Ha] and width
    [bohr] at a random centre (or at the Cartesian point `center`).  kind="displacement": the change of the external
    potential per unit displacement of pseudo-atom `atom` along Cartesian
    `axis`, i.e. d/dR_axis of -D exp(-|r - R|^2 / (2 sigma^2)) summed over images,
    = -D exp(...) (r - R)_axis / sigma^2 (the perturbation of Sec. 4.1.2, where
    atoms are displaced)."""
    rng = np.random.default_rng(10_000 + seed)
    if kind == "bump":
        c = system.lattice @ rng.random(3) if center is None else np.asarray(center, dtype=np.float64)
        return gaussian_sum_on_grid(system.lattice, system.dims, c[None, :], amplitude, width)
    if kind == "displacement":
        lattice, dims = system.lattice, system.dims
        R = system.positions[atom]
        sig = system.width
        r = _grid_points(lattice, dims)
        out = np.zeros(dims)
        reach = 9.0 * sig
        nimg = [int(math.ceil(reach / np.linalg.norm(lattice[:, i]))) + 1 for i in range(3)]
        for n in itertools.product(*[range(-m, m + 1) for m in nimg]):
            d = r - (R + lattice @ np.array(n, dtype=np.float64))
            d2 = np.einsum("...i,...i->...", d, d)
            out += -system.depth * np.exp(-d2 / (2 * sig * sig)) * d[..., axis] / (sig * sig)
        return out
    raise ValueError(kind)


def response_batch(system: System, n_bumps: int = 16, n_displacements: int = 16) -> np.ndarray:
    """The differentiated batch of right-hand sides: seeded Gaussian bumps and
    atom-displacement derivatives of the pseudo-atom potentials, shape (n, N1, N2, N3)."""
    out = [perturbation(system, "bump", seed=i) for i in range(n_bumps)]
    natoms = len(system.positions)
    for j in range(n_displacements):
        out.append(perturbation(system, "displacement", atom=j % natoms, axis=(j // natoms) % 3))
    return np.array(out)


def loss_weights(system: System, seed: int = 5) -> np.ndarray:
    """W = diag(U(0.5, 1.5)) on the grid, for the loss ||W drho||^2."""
    return np.random.default_rng(20_000 + seed).uniform(0.5, 1.5, size=system.dims)


# name -> recipe.  "cfg*" follow the five workload descriptions; "tiny*" are
# the small cases the oracle solves densely in seconds.
_SPECS = {
    # Plain Gamma-point insulator: L=10, Ecut=10, 2 Gaussians (3 Ha, 1 bohr), 4 bands.
    "cfg1": dict(seed=1, cell=(10.0, 10.0, 10.0), dims=(32, 32, 32), Ecut=10.0,
                 layout="random", natoms=2, min_sep=3.0, depth=3.0, width=1.0,
                 n_electrons=8, nbands=6),
    # Diamond-like cell: a=10.26, 8 Gaussians (4 Ha, 0.8 bohr), 2x2x2 k, 32 electrons.
    # With these wells band 16 sits inside a near-degenerate group (gap ~2e-4 Ha),
    # so the system is treated as a metal with Fermi-Dirac smearing T = 0.01 Ha.
    "cfg2": dict(seed=2, cell=(10.26, 10.26, 10.26), dims=(48, 48, 48), Ecut=15.0,
                 layout="diamond", jitter=0.02, depth=4.0, width=0.8,
                 n_electrons=32, nbands=36, T=0.01, kgrid=(2, 2, 2)),
    # Metallic slab: 10x10x60, 12 Gaussians in 3 layers, 4x4x1 k, FD T=0.01.  With
    # the occupation threshold 1e-10, bands up to T ln(2e10) ~ 0.24 Ha above the
    # Fermi level count as occupied: N_occ,k = 60-72 here, so 80 bands (the
    # solver needs one band with f below the threshold at every k).
    "cfg3": dict(seed=3, cell=(10.0, 10.0, 60.0), dims=(40, 40, 216), Ecut=20.0,
                 layout="slab", layers=(25.0, 30.0, 35.0), jitter=0.02, depth=3.0,
                 width=1.0, n_electrons=48, nbands=80, T=0.01, kgrid=(4, 4, 1)),
    # Large Gamma-point cell: 20.5 bohr, 64 Gaussians with 4 Kleinman-Bylander
    # projectors each (s + p), 128 bands, 96^3 grid.
    "cfg4": dict(seed=4, cell=(20.5, 20.5, 20.5), dims=(96, 96, 96), Ecut=20.0,
                 layout="cubic_lattice", per_side=4, jitter=0.05, depth=3.0,
                 width=1.0, n_electrons=256, nbands=136, kb=dict(sigma=(0.8, 0.8), D=(1.0, 0.5))),
    # Tiny cases for dense checks.
    "tiny_insulator": dict(seed=11, cell=(6.0, 6.0, 6.0), dims=(12, 12, 12), Ecut=3.0,
                           layout="random", natoms=2, min_sep=2.5, depth=3.0, width=1.0,
                           n_electrons=4, nbands=4),
    # tiny_insulator's atoms on a finer grid (64 points per bohr^3 instead of 8),
    # for the supercell-size study of Remark rmk:scaling
    "tiny_insulator_fine": dict(seed=11, cell=(6.0, 6.0, 6.0), dims=(24, 24, 24), Ecut=10.0,
                                layout="random", natoms=2, min_sep=2.5, depth=3.0, width=1.0,
                                n_electrons=4, nbands=4),
    "tiny_ortho_k": dict(seed=12, cell=(5.0, 6.0, 7.0), dims=(10, 12, 16), Ecut=3.0,
                         layout="random", natoms=2, min_sep=2.5, depth=3.0, width=1.0,
                         n_electrons=4, nbands=4, kgrid=(2, 1, 1)),
    "tiny_kb": dict(seed=14, cell=(6.0, 6.5, 7.0), dims=(12, 12, 12), Ecut=3.0,
                    layout="random", natoms=2, min_sep=2.5, depth=3.0, width=1.0,
                    n_electrons=4, nbands=6, kgrid=(2, 1, 1), kb=dict(sigma=(0.8, 0.9), D=(1.0, 0.5))),
    "tiny_metal": dict(seed=13, cell=(6.0, 6.0, 6.0), dims=(12, 12, 12), Ecut=3.0,
                       layout="random", natoms=2, min_sep=2.5, depth=2.0, width=1.0,
                       n_electrons=6, nbands=24, T=0.05, kgrid=(2, 1, 1)),
}

CONFIGS = ("cfg1", "cfg2", "cfg3", "cfg4")
TEST_SYSTEMS = ("tiny_insulator", "tiny_ortho_k", "tiny_metal", "tiny_kb")
