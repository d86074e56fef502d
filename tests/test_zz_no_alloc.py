"""The no-allocation H_k entry point (ikr_apply_hamiltonian_noalloc).

Callers that cannot allocate device memory while they work (a stream under
CUDA-graph capture, an application whose device memory belongs to its own
pool, a latency-bound loop) use this entry point; its scratch lives in a
static device array of the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.  Two
calls in a row are checked against ikr_apply_hamiltonian, which allocates its
workspace as needed, with the FP64 tolerance of the other H_k tests (1e-12
relative): the second call would expose stale scratch from the first."""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import groundstate, ikr
    from workloads import make_system

    ctx = groundstate.context_for(make_system("tiny_ortho_k"))
    rng = np.random.default_rng(42)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (k, nvec) in enumerate([(1, 7), (0, 3)]):
        nb = ctx.basis_size(k)
        psi = torch.tensor(rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb)), device="cuda")
        ref = ctx.apply_hamiltonian(k, psi)
        out = torch.full_like(psi, float("nan"))
        st = ikr._LIB.ikr_apply_hamiltonian_noalloc(ctx._h, k, ct.c_void_p(psi.data_ptr()),
                                                     ct.c_void_p(out.data_ptr()), nvec, stream)
        torch.cuda.synchronize()
        assert st == ikr.IKR_OK, ikr._LIB.ikr_last_error(ctx._h).decode()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err < 1e-12, (call, err)
