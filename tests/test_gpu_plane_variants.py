"""The compact FP32 plane pass (k_plane_rc: only the active x positions of every
row in shared memory) against the full-plane kernel (k_plane_r) it replaces in
the CG's H_k applications, on a small grid and at the benchmark's 48^3 grid,
for both register bounds (5 and 4 blocks per SM).  Both run the same transforms
on the same values, so their results agree to FP32 rounding (they are expected
to be identical)."""
import numpy as np
import pytest

from gpu_common import system, torch

pytestmark = pytest.mark.gpu


def _bare_context(s):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import ikr
    return ikr.Context.setup_groundstate(s.lattice, s.dims, s.Ecut, s.kpoints, s.kweights, s.V,
                                         s.temperature, s.n_electrons)


@pytest.mark.parametrize("variant", ["5", "4"])
@pytest.mark.parametrize("name", ["tiny_ortho_k", "cfg2"])
def test_compact_fp32_plane_matches_full_plane(name, variant, monkeypatch):
    from paper_2505_02319_gb300 import ikr
    s = system(name)
    monkeypatch.setenv("IKR_PLANE_RC", "0")
    full = _bare_context(s)
    monkeypatch.setenv("IKR_PLANE_RC", variant)
    compact = _bare_context(s)
    rng = np.random.default_rng(17)
    for k in range(full.nkpt):
        nb = full.basis_size(k)
        psi = torch.tensor((rng.normal(size=(9, nb)) + 1j * rng.normal(size=(9, nb))).astype(np.complex64),
                           device="cuda")
        a = full.apply_hamiltonian(k, psi, precision=ikr.MIXED)
        b = compact.apply_hamiltonian(k, psi, precision=ikr.MIXED)
        scale = float(torch.abs(a).max())
        assert float(torch.abs(a - b).max()) <= 1e-6 * scale, k
    full.destroy()
    compact.destroy()


@pytest.mark.parametrize("name", ["tiny_ortho_k", "cfg2"])
def test_double_float_hamiltonian_matches_oracle(name):
    """H_k with the plane pass in double-float (IKR_DF64; on the 48 x 48 planes of
    cfg2 the swizzled kernel) against the oracle's dense H_k: FP64 accuracy up
    to the double-float roundings of the butterflies (~1e-13 per pass)."""
    from gpu_common import context, oracle_state
    from paper_2505_02319_gb300 import ikr
    gs, ctx = oracle_state(name), context(name)
    rng = np.random.default_rng(19)
    for k, kb in enumerate(gs.kblocks[:3]):
        nb = len(kb.eps)
        psi = rng.normal(size=(4, nb)) + 1j * rng.normal(size=(4, nb))
        out = ctx.apply_hamiltonian(k, torch.tensor(psi, device="cuda"), precision=ikr.DF64).cpu().numpy()
        ref = psi @ kb.H.T
        assert np.linalg.norm(out - ref) < 1e-11 * np.linalg.norm(ref), k


def test_swizzled_double_float_plane_matches_padded_one(monkeypatch):
    """cfg2: the swizzled double-float plane pass (8-lane y-lines) against
    k_plane_t<dfloat> (4-lane y-lines, padded rows): both FP64-accurate, so
    they agree to the double-float rounding level."""
    from paper_2505_02319_gb300 import ikr
    s = system("cfg2")
    monkeypatch.setenv("IKR_PLANE_SW", "0")
    padded = _bare_context(s)
    monkeypatch.setenv("IKR_PLANE_SW", "1")
    swz = _bare_context(s)
    rng = np.random.default_rng(23)
    for k in (0, 5):
        nb = padded.basis_size(k)
        psi = torch.tensor(rng.normal(size=(6, nb)) + 1j * rng.normal(size=(6, nb)), device="cuda")
        a = padded.apply_hamiltonian(k, psi, precision=ikr.DF64)
        b = swz.apply_hamiltonian(k, psi, precision=ikr.DF64)
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) < 1e-12, k
    padded.destroy()
    swz.destroy()
