"""The no-allocation H_k entry point (ikr_apply_hamiltonian_noalloc).

Callers that cannot allocate device memory while they work (a stream under
CUDA-graph capture, an application whose device memory belongs to its own
pool, a latency-bound loop) use this entry point; its scratch lives in a
static 32 MiB device array of the library.  This file is collected last so
that a run stopping at the first failure has already run every other test.
Results are checked against ikr_apply_hamiltonian, which allocates its
workspace as needed, with the FP64 tolerance of the other H_k tests (1e-12
relative), on two calls in a row (the second would expose stale scratch from
the first); with more vectors than one chunk of the scratch holds; on a wide
96 x 96 plane without projectors; and a grid whose single vector does not fit
is rejected with IKR_ERR_ARG before any work."""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCRATCH = 32 << 20


def _setup():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_02319_gb300 import ikr
    return torch, ikr


def _noalloc(torch, ikr, ctx, k, psi):
    out = torch.full_like(psi, float("nan"))
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ikr._LIB.ikr_apply_hamiltonian_noalloc(ctx._h, k, ct.c_void_p(psi.data_ptr()),
                                                 ct.c_void_p(out.data_ptr()), psi.shape[0], stream)
    torch.cuda.synchronize()
    return st, out


def _per_vector_bytes(ctx):
    g = ctx.fft_geometry()
    return 2 * 16 * g["dims"][2] * ((g["ncols"] + 15) // 16 * 16)


def _compare_twice(torch, ikr, ctx, calls, seed):
    rng = np.random.default_rng(seed)
    for call, (k, nvec) in enumerate(calls):
        nb = ctx.basis_size(k)
        psi = torch.tensor(rng.normal(size=(nvec, nb)) + 1j * rng.normal(size=(nvec, nb)), device="cuda")
        ref = ctx.apply_hamiltonian(k, psi)
        st, out = _noalloc(torch, ikr, ctx, k, psi)
        assert st == ikr.IKR_OK, ikr._LIB.ikr_last_error(ctx._h).decode()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err < 1e-12, (call, err)


def test_noalloc_matches_allocating_entry_point_twice():
    torch, ikr = _setup()
    from paper_2505_02319_gb300 import groundstate
    from workloads import make_system
    ctx = groundstate.context_for(make_system("tiny_ortho_k"))
    _compare_twice(torch, ikr, ctx, [(1, 7), (0, 3)], 42)
    ctx.destroy()


def test_noalloc_with_several_chunks():
    """More vectors than the scratch holds at once: the chunk loop runs two
    and three times, each chunk checked against the allocating call."""
    torch, ikr = _setup()
    from paper_2505_02319_gb300 import groundstate
    from workloads import make_system
    ctx = groundstate.context_for(make_system("tiny_ortho_k"))
    cap = SCRATCH // _per_vector_bytes(ctx)
    chunk = 1 << (int(cap).bit_length() - 1)          # the power of two the entry point takes
    assert 256 <= chunk <= 4096, chunk
    _compare_twice(torch, ikr, ctx, [(1, chunk + chunk // 2 + 3), (0, 2 * chunk + 5)], 43)
    ctx.destroy()


def test_noalloc_on_a_wide_plane_without_projectors():
    """A 96 x 96 x 8 grid (no projectors): the compiled 96 x 96 plane kernel
    that ikr_apply_hamiltonian runs; the runtime-size kernel would need more
    shared memory than a block may use."""
    torch, ikr = _setup()
    from workloads.systems import gaussian_sum_on_grid
    lattice = np.diag([20.5, 20.5, 4.0])
    dims = (96, 96, 8)
    centres = np.array([[3.0, 4.0, 1.0], [12.0, 9.5, 2.5]])
    V = gaussian_sum_on_grid(lattice, dims, centres, -3.0, 1.0)
    ctx = ikr.Context.setup_groundstate(lattice, dims, 2.0, np.zeros((1, 3)), np.ones(1), V, 0.0, 2)
    assert 16 * (96 + 96 + 2 * 96 * 97) > 227 * 1024
    _compare_twice(torch, ikr, ctx, [(0, 5), (0, 2)], 44)
    ctx.destroy()


def test_noalloc_rejects_a_vector_beyond_the_scratch():
    """A 40 x 40 x 100 bohr cell at 20 Ha on a 96 x 96 x 216 grid: one vector
    needs more than 32 MiB of scratch, so the call returns IKR_ERR_ARG and
    leaves the output untouched."""
    torch, ikr = _setup()
    lattice = np.diag([40.0, 40.0, 100.0])
    dims = (96, 96, 216)
    V = np.full(int(np.prod(dims)), -0.5)
    ctx = ikr.Context.setup_groundstate(lattice, dims, 20.0, np.zeros((1, 3)), np.ones(1), V, 0.0, 2)
    assert _per_vector_bytes(ctx) > SCRATCH
    nb = ctx.basis_size(0)
    psi = torch.ones((1, nb), dtype=torch.complex128, device="cuda")
    st, out = _noalloc(torch, ikr, ctx, 0, psi)
    assert st == ikr.IKR_ERR_ARG
    assert "32 MiB" in ikr._LIB.ikr_last_error(ctx._h).decode()
    assert bool(torch.isnan(out).all())
    ctx.destroy()
