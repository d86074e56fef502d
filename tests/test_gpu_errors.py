"""Failure detection, exercised on the host side (no GPU fault, hang or trap):
the library turns missing gaps, non-finite inputs, iteration caps, timeouts
and invalid arguments into status codes and stays usable afterwards."""
import ctypes as ct

import numpy as np
import pytest

import gpu_common
from gpu_common import context, dev, system, torch

pytestmark = pytest.mark.gpu


def _ikr():
    from paper_2505_02319_gb300 import ikr
    return ikr


def test_no_gap_is_reported():
    """An insulator whose band N/2+1 is not above band N/2 (proof of Lemma cgtol_E)."""
    ikr = _ikr()
    from paper_2505_02319_gb300 import groundstate
    s = system("tiny_insulator")
    ctx = ikr.Context.setup_groundstate(s.lattice, s.dims, s.Ecut, s.kpoints, s.kweights, s.V,
                                        s.temperature, s.n_electrons)
    ev, vecs = gpu_common.dense_eigenpairs(ctx, 4)
    ev = ev.copy()
    ev[0, 2] = ev[0, 1]            # degenerate HOMO/LUMO
    with pytest.raises(ikr.IkrError) as e:
        ctx.set_eigenpairs(ev, vecs)
    assert e.value.status == ikr.IKR_ERR_NOGAP
    ctx.set_eigenpairs(*gpu_common.dense_eigenpairs(ctx, 4))   # still usable


def test_nonfinite_rhs_is_numeric_error():
    ikr = _ikr()
    s, ctx = system("tiny_insulator"), context("tiny_insulator")
    b = np.zeros(s.n_grid)
    b[3] = np.nan
    with pytest.raises(ikr.IkrError) as e:
        ctx.solve_response(dev(b), tau=1e-8)
    assert e.value.status == ikr.IKR_ERR_NUMERIC
    # the context is still usable
    x, rep = ctx.solve_response(dev(np.ones(s.n_grid) / np.sqrt(s.n_grid)), tau=1e-8)
    assert rep[0]["status"] == ikr.IKR_OK


def test_cg_iteration_cap_is_reported():
    ikr = _ikr()
    s, ctx = system("cfg1"), context("cfg1")
    nsys = ctx.groundstate_nsys
    v = dev(np.random.default_rng(0).normal(size=s.n_grid))
    rep = ikr.Report()
    out = torch.empty_like(v)
    st = ikr._LIB.ikr_apply_chi0(ctx._h, ct.c_void_p(v.data_ptr()), ct.c_void_p(out.data_ptr()),
                                 np.full(nsys, 1e-30).ctypes.data_as(ct.POINTER(ct.c_double)), ikr.FP64,
                                 ct.byref(rep), ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == ikr.IKR_ERR_NOCONV and rep.cg_noconv == nsys


def test_restart_cap_and_timeout():
    ikr = _ikr()
    s, ctx = system("cfg1"), context("cfg1")
    b = dev(np.random.default_rng(1).normal(size=s.n_grid))
    b /= torch.linalg.norm(b)
    x, rep = ctx.solve_response(b, tau=1e-14, m=2, max_restarts=1, strategy="bal")
    assert rep[0]["status"] == ikr.IKR_ERR_NOCONV and rep[0]["restarts"] >= 1
    x, rep = ctx.solve_response(b, tau=1e-12, timeout_s=1e-6)
    assert rep[0]["status"] == ikr.IKR_ERR_TIMEOUT


def test_invalid_arguments():
    ikr = _ikr()
    s, ctx = system("tiny_insulator"), context("tiny_insulator")
    psi = torch.zeros((2, ctx.basis_size(0)), dtype=torch.complex128, device="cuda")
    with pytest.raises(ikr.IkrError) as e:
        ctx.apply_hamiltonian(5, psi)                      # k out of range
    assert e.value.status == ikr.IKR_ERR_ARG
    with pytest.raises(ikr.IkrError) as e:
        ctx.solve_sternheimer([0, 0], [0, 7], torch.zeros((2, ctx.basis_size(0)), dtype=torch.complex128,
                                                           device="cuda"), [1e-8, 1e-8])   # band not occupied
    assert e.value.status == ikr.IKR_ERR_ARG
    with pytest.raises(ikr.IkrError):
        ikr.Context.setup_groundstate(s.lattice, (14, 12, 12), s.Ecut, s.kpoints, s.kweights,
                                      np.zeros(14 * 144), 0.0, 4)          # factor 7 in the grid
