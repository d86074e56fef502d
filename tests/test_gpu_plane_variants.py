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
