"""Thin ctypes binding of libikr.so (include/ikr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are torch tensors (their data pointers are passed),
the CUDA stream is torch's current stream.  The library must be built
(``paper_2505_02319_gb300.build.build()``); importing this module without it
raises ImportError - there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libikr.so")

IKR_OK, IKR_ERR_ARG, IKR_ERR_CUDA, IKR_ERR_OOM, IKR_ERR_NOGAP, IKR_ERR_NOCONV, \
    IKR_ERR_NUMERIC, IKR_ERR_TIMEOUT, IKR_ERR_STATE = range(9)
FP64, MIXED, DF64 = 0, 1, 2
STRATEGIES = {"agr": 0, "bal": 1, "grt": 2, "D10": 3, "D100": 4, "D10n": 5, "grt_exact": 6, "fixed": 7}


class IkrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class System(ct.Structure):
    _fields_ = [("lattice", ct.c_double * 9), ("dims", ct.c_int * 3), ("Ecut", ct.c_double),
                ("nkpt", ct.c_int), ("kpoints", ct.POINTER(ct.c_double)),
                ("kweights", ct.POINTER(ct.c_double)), ("V", ct.POINTER(ct.c_double)),
                ("temperature", ct.c_double), ("n_electrons", ct.c_int)]


class Eigenpairs(ct.Structure):
    _fields_ = [("nbands", ct.c_int), ("eigenvalues", ct.POINTER(ct.c_double)),
                ("eigenvectors", ct.POINTER(ct.c_void_p))]


class Report(ct.Structure):
    _fields_ = [("status", ct.c_int), ("outer_iters", ct.c_int), ("restarts", ct.c_int),
                ("e_applies", ct.c_int), ("e_applies_fp32", ct.c_int), ("n_ham", ct.c_longlong),
                ("n_ham_fp64", ct.c_longlong), ("cg_max_iters", ct.c_int), ("cg_noconv", ct.c_int),
                ("est_residual", ct.c_double), ("sigma", ct.c_double), ("b_norm", ct.c_double),
                ("kv_norm", ct.c_double), ("min_cg_tol", ct.c_double), ("max_cg_tol", ct.c_double),
                ("ms", ct.c_double), ("history", ct.POINTER(ct.c_double)), ("history_cap", ct.c_int),
                ("history_len", ct.c_int), ("first_min_cg_tol", ct.c_double), ("first_kv_norm", ct.c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "history"}
        if self.history_len and self.history:
            d["history"] = [self.history[i] for i in range(self.history_len)]
        return d


class SolveOpts(ct.Structure):
    _fields_ = [("tau", ct.c_double), ("m", ct.c_int), ("strategy", ct.c_int), ("precision", ct.c_int),
                ("max_restarts", ct.c_int), ("cg_maxit", ct.c_int), ("kerker_alpha", ct.c_double),
                ("fixed_cg_tol", ct.c_double), ("s0", ct.c_double), ("use_x0", ct.c_int),
                ("timeout_s", ct.c_double)]


class KernelStat(ct.Structure):
    _fields_ = [("name", ct.c_char_p), ("launches", ct.c_longlong), ("timed_calls", ct.c_longlong),
                ("ms", ct.c_double), ("units_fp32", ct.c_longlong), ("units_fp64", ct.c_longlong),
                ("ms_fp32", ct.c_double), ("ms_fp64", ct.c_double), ("timed_calls_fp32", ct.c_longlong),
                ("timed_calls_fp64", ct.c_longlong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2505_02319_gb300.build.build()")
    lib = ct.CDLL(LIB_PATH)
    P, I, D, S = ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p
    sig = {
        "ikr_default_opts": (None, [ct.POINTER(SolveOpts)]),
        "ikr_setup_groundstate": (I, [ct.POINTER(System), ct.POINTER(Eigenpairs), S, ct.POINTER(P)]),
        "ikr_set_eigenpairs": (I, [P, ct.POINTER(Eigenpairs), S]),
        "ikr_compute_eigenpairs": (I, [P, I, D, I, I, ct.POINTER(D), ct.POINTER(I), ct.POINTER(D), S]),
        "ikr_set_nonlocal": (I, [P, I, ct.POINTER(D), ct.POINTER(D), ct.POINTER(D), S]),
        "ikr_set_schur": (I, [P, I]),
        "ikr_set_tensor_cores": (I, [P, I]),
        "ikr_projection_coefficients": (I, [P, I, I, P, I, ct.POINTER(D), S]),
        "ikr_project_out": (I, [P, I, I, P, I, S]),
        "ikr_hermitian_eigh": (I, [I, ct.POINTER(D), ct.POINTER(D), ct.POINTER(D)]),
        "ikr_num_kpoints": (I, [P]),
        "ikr_basis_size": (I, [P, I, ct.POINTER(I)]),
        "ikr_basis_millers": (I, [P, I, ct.POINTER(I)]),
        "ikr_groundstate_info": (I, [P, ct.POINTER(D), ct.POINTER(I), ct.POINTER(D), P, S]),
        "ikr_apply_hamiltonian": (I, [P, I, P, P, I, I, S]),
        "ikr_apply_hamiltonian_noalloc": (I, [P, I, P, P, I, S]),
        "ikr_solve_sternheimer": (I, [P, I, ct.POINTER(I), ct.POINTER(I), P, P, I, ct.POINTER(D), I, I,
                                      ct.POINTER(I), ct.POINTER(D), S]),
        "ikr_apply_chi0": (I, [P, P, P, ct.POINTER(D), I, ct.POINTER(Report), S]),
        "ikr_apply_dielectric": (I, [P, P, P, ct.POINTER(D), I, ct.POINTER(Report), S]),
        "ikr_solve_response": (I, [P, I, P, P, ct.POINTER(SolveOpts), ct.POINTER(Report), S]),
        "ikr_apply_dielectric_adjoint": (I, [P, P, P, ct.POINTER(D), I, ct.POINTER(Report), S]),
        "ikr_solve_response_adjoint": (I, [P, I, P, P, ct.POINTER(SolveOpts), ct.POINTER(Report), S]),
        "ikr_destroy": (None, [P]),
        "ikr_last_error": (ct.c_char_p, [P]),
        "ikr_status_string": (ct.c_char_p, [I]),
        "ikr_version": (ct.c_char_p, []),
        "ikr_profile_start": (I, [P, ct.c_uint]),
        "ikr_profile_read": (I, [P, ct.POINTER(KernelStat), I]),
        "ikr_fft_geometry": (I, [P, ct.POINTER(I)]),
        "ikr_device_peaks": (I, [ct.POINTER(ct.c_double), P]),
        "ikr_autotune": (I, [P, ct.POINTER(ct.c_double), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = _load()


def _status_name(s):
    return _LIB.ikr_status_string(int(s)).decode()


def version():
    return _LIB.ikr_version().decode()


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ct.c_void_p(t.data_ptr())


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ct.POINTER(ct.c_double))


def default_opts(**kw):
    o = SolveOpts()
    _LIB.ikr_default_opts(ct.byref(o))
    for k, v in kw.items():
        if k == "strategy" and isinstance(v, str):
            v = STRATEGIES[v]
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        setattr(o, k, v)
    return o


def device_peaks():
    """Measured arithmetic throughput of the current device (ikr_device_peaks):
    SMs, FP32 and FP64 FMA TFLOP/s, FP32 and double-float radix-4 butterfly
    TFLOP/s, and the device's reported SM clock (MHz)."""
    out = (ct.c_double * 6)()
    st = _LIB.ikr_device_peaks(out, _stream())
    if st != IKR_OK:
        raise IkrError(st, "device_peaks failed")
    keys = ("sms", "fp32_fma_tflops", "fp64_fma_tflops", "fp32_butterfly_tflops", "df64_butterfly_tflops",
            "sm_clock_mhz")
    return {k: (int(v) if k == "sms" else float(v)) for k, v in zip(keys, out)}


class Context:
    """One system: plane-wave bases, potential and (optionally) ground state."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    # -- creation ----------------------------------------------------------
    @classmethod
    def setup_groundstate(cls, lattice, dims, Ecut, kpoints, kweights, V, temperature, n_electrons,
                          eigenvalues=None, eigenvectors=None):
        """Create a context (ikr_setup_groundstate).  ``lattice`` has the cell
        vectors as columns; V is the potential on the grid in C order."""
        sysd = System()
        lat = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
        for i in range(3):
            for j in range(3):
                sysd.lattice[3 * i + j] = lat[i, j]
        for i in range(3):
            sysd.dims[i] = int(dims[i])
        sysd.Ecut = float(Ecut)
        kp, sysd.kpoints = _dbl(np.asarray(kpoints).reshape(-1, 3))
        kw, sysd.kweights = _dbl(kweights)
        sysd.nkpt = int(kp.shape[0])
        Vh, sysd.V = _dbl(np.asarray(V).ravel())
        sysd.temperature = float(temperature)
        sysd.n_electrons = int(n_electrons)
        keep = [kp, kw, Vh]
        eig, ekeep = _eigenpairs(eigenvalues, eigenvectors)
        h = ct.c_void_p()
        st = _LIB.ikr_setup_groundstate(ct.byref(sysd), ct.byref(eig) if eig else None, _stream(),
                                        ct.byref(h))
        if st != IKR_OK:
            raise IkrError(st, "setup_groundstate failed")
        return cls(h, keep + ekeep)

    def set_eigenpairs(self, eigenvalues, eigenvectors):
        eig, keep = _eigenpairs(eigenvalues, eigenvectors)
        self._check(_LIB.ikr_set_eigenpairs(self._h, ct.byref(eig), _stream()))

    def set_nonlocal(self, centres, sigma, D):
        """Kleinman-Bylander projectors (Gaussian s and p) on the given centres."""
        cen, cp = _dbl(np.asarray(centres, dtype=np.float64).reshape(-1, 3))
        sg, sp = _dbl(sigma)
        dd, dp = _dbl(D)
        self._check(_LIB.ikr_set_nonlocal(self._h, len(cen), cp, sp, dp, _stream()))

    def set_schur(self, enable=True):
        """Schur-complement Sternheimer solves over the extra computed bands
        (ikr_set_schur): same chi0, better conditioned CG."""
        self._check(_LIB.ikr_set_schur(self._h, 1 if enable else 0))

    def autotune(self):
        """Time the interchangeable kernel variants on this context's systems and
        keep the fastest (ikr_autotune); returns the timings and the choice."""
        out = (ct.c_double * 16)()
        self._check(_LIB.ikr_autotune(self._h, out, _stream()))
        v = list(out)
        return {"cg_iter_ms_cuda_cores": {"plane_full": v[0], "plane_compact4": v[1], "plane_compact5": v[2]},
                "cg_iter_ms_tensor_cores": {"plane_full": v[3], "plane_compact4": v[4], "plane_compact5": v[5]},
                "plane_rc": int(v[6]), "tensor_cores": bool(v[7]),
                "df64_apply_ms": {"padded": v[8], "swizzled": v[9]}, "plane_sw": bool(v[10]),
                "cg_fused_cluster": int(v[11]),
                "cg_iter_ms_cluster": {"16": v[12], "12": v[13], "10": v[14], "8": v[15]}}

    def set_tensor_cores(self, enable=True, swizzle=True):
        """FP32 projection products on the tensor cores (ikr_set_tensor_cores):
        swizzle=False selects the canonical operand layout."""
        self._check(_LIB.ikr_set_tensor_cores(self._h, (1 if swizzle else 2) if enable else 0))

    def projection_coefficients(self, k, y, method=0):
        """<phi_m, y_s> for the occupied orbitals of k-point k, FP32 arithmetic:
        y a (nvec, Nb_k) complex64 CUDA tensor; method 0 CUDA cores, 1 tensor
        cores (swizzled operand tiles), 2 tensor cores (canonical layout).  Returns a (nvec, N_occ,k) complex128 numpy array."""
        yy = y.reshape(-1, y.shape[-1]).contiguous()
        nvec = yy.shape[0]
        nocc = int(self.groundstate_info(self.nbands, self.ngrid)["nocc"][k])
        out = np.zeros((nvec, nocc), dtype=np.complex128)
        self._check(_LIB.ikr_projection_coefficients(self._h, int(k), nvec, _dptr(yy), int(method),
                                                      out.ctypes.data_as(ct.POINTER(ct.c_double)), _stream()))
        return out

    def project_out(self, k, y, method=0):
        """Q_k y = y - Phi_k (Phi_k^H y) for a (nvec, Nb_k) complex64 CUDA tensor
        (in place; returned); method as projection_coefficients."""
        self._check(_LIB.ikr_project_out(self._h, int(k), int(y.reshape(-1, y.shape[-1]).shape[0]), _dptr(y),
                                         int(method), _stream()))
        return y

    def compute_eigenpairs(self, nbands, tol=1e-10, maxit=200, degree=12):
        """Lowest ``nbands`` eigenpairs of every H_k on the GPU (Chebyshev-filtered
        subspace iteration on the library's H_k), set as the ground state.
        Returns (eigenvalues (nk, nbands), cycles per k-point, largest residual
        per k-point)."""
        nk = self.nkpt
        ev = np.zeros((nk, int(nbands)))
        iters = (ct.c_int * nk)()
        res = (ct.c_double * nk)()
        st = _LIB.ikr_compute_eigenpairs(self._h, int(nbands), float(tol), int(maxit), int(degree),
                                         ev.ctypes.data_as(ct.POINTER(ct.c_double)), iters, res, _stream())
        self.eigenvalues, self.eig_iters, self.eig_residuals = ev, list(iters), list(res)
        self._check(st)
        return ev, list(iters), list(res)

    def _check(self, st, allow=()):
        if st != IKR_OK and st not in allow:
            raise IkrError(st, _LIB.ikr_last_error(self._h).decode())
        return st

    def destroy(self):
        if self._h:
            _LIB.ikr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # -- accounting ----------------------------------------------------------
    KERNEL_CLASSES = ("z_inverse", "plane", "z_forward", "proj_coef", "proj_apply", "cg_vector",
                      "density", "grid_fft", "grid_ops", "scalar")

    def profile_start(self, timed=()):
        mask = 0
        for name in timed:
            mask |= 1 << self.KERNEL_CLASSES.index(name)
        self._check(_LIB.ikr_profile_start(self._h, mask))

    def profile_read(self):
        arr = (KernelStat * 16)()
        n = _LIB.ikr_profile_read(self._h, arr, 16)
        return {arr[i].name.decode(): dict(launches=arr[i].launches, timed_calls=arr[i].timed_calls,
                                           ms=arr[i].ms, units_fp32=arr[i].units_fp32,
                                           units_fp64=arr[i].units_fp64,
                                           units=arr[i].units_fp32 + arr[i].units_fp64,
                                           ms_fp32=arr[i].ms_fp32, ms_fp64=arr[i].ms_fp64,
                                           calls_fp32=arr[i].timed_calls_fp32,
                                           calls_fp64=arr[i].timed_calls_fp64) for i in range(n)}

    def fft_geometry(self):
        g = (ct.c_int * 5)()
        self._check(_LIB.ikr_fft_geometry(self._h, g))
        return dict(dims=(g[0], g[1], g[2]), ncols=g[3], nxa=g[4])

    # -- queries -------------------------------------------------------------
    @property
    def nkpt(self):
        return _LIB.ikr_num_kpoints(self._h)

    def basis_size(self, k):
        n = ct.c_int()
        self._check(_LIB.ikr_basis_size(self._h, k, ct.byref(n)))
        return n.value

    def basis_millers(self, k):
        nb = self.basis_size(k)
        out = np.zeros((nb, 3), dtype=np.int32)
        self._check(_LIB.ikr_basis_millers(self._h, k, out.ctypes.data_as(ct.POINTER(ct.c_int))))
        return out

    def groundstate_info(self, nbands, ngrid):
        f = np.zeros((self.nkpt, nbands))
        nocc = np.zeros(self.nkpt, dtype=np.int32)
        eF = ct.c_double()
        rho = torch.empty(ngrid, dtype=torch.float64, device="cuda")
        self._check(_LIB.ikr_groundstate_info(self._h, f.ctypes.data_as(ct.POINTER(ct.c_double)),
                                              nocc.ctypes.data_as(ct.POINTER(ct.c_int)), ct.byref(eF),
                                              _dptr(rho), _stream()))
        return dict(f=f, nocc=nocc, eF=eF.value, rho=rho)

    # -- the hot path ----------------------------------------------------------
    def apply_hamiltonian(self, k, psi, precision=FP64):
        """H_k psi for psi of shape (nvec, Nb_k), complex128 (FP64) or complex64 (MIXED)."""
        out = torch.empty_like(psi)
        self._check(_LIB.ikr_apply_hamiltonian(self._h, k, _dptr(psi), _dptr(out), psi.shape[0],
                                               precision, _stream()))
        return out

    def solve_sternheimer(self, k_of, band_of, rhs, tol, maxit=400, precision=FP64):
        """Solve Q(H_k - eps_n)Q x = Q rhs for systems (k_of[s], band_of[s]); rhs (nsys, ld)."""
        k_of = np.ascontiguousarray(k_of, dtype=np.int32)
        band_of = np.ascontiguousarray(band_of, dtype=np.int32)
        tol, tolp = _dbl(tol)
        x = torch.zeros_like(rhs)
        it = np.zeros(len(k_of), dtype=np.int32)
        res = np.zeros(len(k_of))
        st = _LIB.ikr_solve_sternheimer(self._h, len(k_of), k_of.ctypes.data_as(ct.POINTER(ct.c_int)),
                                        band_of.ctypes.data_as(ct.POINTER(ct.c_int)), _dptr(rhs), _dptr(x),
                                        rhs.shape[1], tolp, maxit, precision,
                                        it.ctypes.data_as(ct.POINTER(ct.c_int)),
                                        res.ctypes.data_as(ct.POINTER(ct.c_double)), _stream())
        self._check(st, allow=(IKR_ERR_NOCONV,))
        return x, it, res, st

    def apply_chi0(self, dV, tol=None, precision=FP64):
        out = torch.empty_like(dV)
        rep = Report()
        tp = None
        if tol is not None:
            tarr, tp = _dbl(tol)
        st = _LIB.ikr_apply_chi0(self._h, _dptr(dV), _dptr(out), tp, precision, ct.byref(rep), _stream())
        self._check(st, allow=(IKR_ERR_NOCONV,))
        return out, rep.as_dict()

    def apply_dielectric(self, v, tol=None, precision=FP64):
        out = torch.empty_like(v)
        rep = Report()
        tp = None
        if tol is not None:
            tarr, tp = _dbl(tol)
        st = _LIB.ikr_apply_dielectric(self._h, _dptr(v), _dptr(out), tp, precision, ct.byref(rep), _stream())
        self._check(st, allow=(IKR_ERR_NOCONV,))
        return out, rep.as_dict()

    def apply_dielectric_adjoint(self, v, tol=None, precision=FP64):
        out = torch.empty_like(v)
        rep = Report()
        tp = None
        if tol is not None:
            tarr, tp = _dbl(tol)
        st = _LIB.ikr_apply_dielectric_adjoint(self._h, _dptr(v), _dptr(out), tp, precision, ct.byref(rep),
                                               _stream())
        self._check(st, allow=(IKR_ERR_NOCONV,))
        return out, rep.as_dict()

    def solve_response_adjoint(self, g, x0=None, opts=None, history=64, **kw):
        """Solve E^T lambda = g (the adjoint solve).  Arguments as solve_response."""
        return self._solve(_LIB.ikr_solve_response_adjoint, g, x0, opts, history, kw)

    def solve_response(self, b, x0=None, opts=None, history=64, **kw):
        """Solve E x = b (Algorithm 1).  b: (Ng,) or (nrhs, Ng) float64 CUDA tensor."""
        return self._solve(_LIB.ikr_solve_response, b, x0, opts, history, kw)

    def _solve(self, fn, b, x0, opts, history, kw):
        o = opts if opts is not None else default_opts(**kw)
        bb = b.reshape(-1, b.shape[-1]) if b.dim() > 1 else b.reshape(1, -1)
        nrhs = bb.shape[0]
        if x0 is not None:
            x = x0.reshape(nrhs, -1).clone().contiguous()
            o.use_x0 = 1
        else:
            x = torch.zeros_like(bb)
        reps = (Report * nrhs)()
        hists = [np.zeros(history) for _ in range(nrhs)]
        for r in range(nrhs):
            reps[r].history = hists[r].ctypes.data_as(ct.POINTER(ct.c_double))
            reps[r].history_cap = history
        st = fn(self._h, nrhs, _dptr(bb.contiguous()), _dptr(x), ct.byref(o), reps, _stream())
        self._check(st, allow=(IKR_ERR_NOCONV, IKR_ERR_TIMEOUT))
        out = x.reshape(b.shape)
        return out, [reps[r].as_dict() for r in range(nrhs)]


def _eigenpairs(eigenvalues, eigenvectors):
    if eigenvalues is None:
        return None, []
    ev = np.ascontiguousarray(eigenvalues, dtype=np.float64)
    nk, nb = ev.shape
    vecs = [v.contiguous() for v in eigenvectors]
    ptrs = (ct.c_void_p * nk)(*[v.data_ptr() for v in vecs])
    e = Eigenpairs()
    e.nbands = nb
    e.eigenvalues = ev.ctypes.data_as(ct.POINTER(ct.c_double))
    e.eigenvectors = ct.cast(ptrs, ct.POINTER(ct.c_void_p))
    return e, [ev, vecs, ptrs]


# module-level functions with the names of the C ABI
setup_groundstate = Context.setup_groundstate


def apply_hamiltonian(ctx, k, psi, precision=FP64):
    return ctx.apply_hamiltonian(k, psi, precision)


def solve_sternheimer(ctx, *a, **kw):
    return ctx.solve_sternheimer(*a, **kw)


def apply_chi0(ctx, dV, tol=None, precision=FP64):
    return ctx.apply_chi0(dV, tol, precision)


def apply_dielectric(ctx, v, tol=None, precision=FP64):
    return ctx.apply_dielectric(v, tol, precision)


def solve_response(ctx, b, **kw):
    return ctx.solve_response(b, **kw)


def apply_dielectric_adjoint(ctx, v, tol=None, precision=FP64):
    return ctx.apply_dielectric_adjoint(v, tol, precision)


def solve_response_adjoint(ctx, g, **kw):
    return ctx.solve_response_adjoint(g, **kw)


def hermitian_eigh(a):
    """Eigenvalues (ascending) and eigenvectors (columns) of a Hermitian matrix
    by the library's host Jacobi solver (the Rayleigh-Ritz step of the GPU
    eigensolver); no GPU needed."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    n = a.shape[0]
    w = np.empty(n)
    v = np.empty((n, n), dtype=np.complex128)
    st = _LIB.ikr_hermitian_eigh(n, a.ctypes.data_as(ct.POINTER(ct.c_double)), w.ctypes.data_as(ct.POINTER(ct.c_double)),
                                 v.ctypes.data_as(ct.POINTER(ct.c_double)))
    if st != IKR_OK:
        raise IkrError(st, "ikr_hermitian_eigh failed")
    return w, v
