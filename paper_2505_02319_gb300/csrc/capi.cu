// extern "C" entry points (include/ikr.h).  Each wraps the C++ implementation,
// turns exceptions into status codes and records the message in the context.
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <cmath>
#include <new>

#include "solver.hpp"

using namespace ikr;

namespace {

template <typename F> ikr_status guarded(ikr_ctx* c, F&& f) {
  try {
    f();
    if (c) c->err.clear();
    return IKR_OK;
  } catch (const Error& e) {
    if (c) c->err = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return IKR_ERR_OOM;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return IKR_ERR_ARG;
  }
}

void fill_report(ikr_report* r, const RunStats& rs, double ms) {
  if (!r) return;
  r->status = IKR_OK;
  r->outer_iters = 0;
  r->restarts = 0;
  r->e_applies = rs.e_applies;
  r->e_applies_fp32 = rs.e_applies_fp32;
  r->n_ham = rs.n_ham;
  r->n_ham_fp64 = rs.n_ham_fp64;
  r->cg_max_iters = rs.cg_max_iters;
  r->cg_noconv = rs.cg_noconv;
  r->est_residual = 0.0;
  r->sigma = 0.0;
  r->b_norm = 0.0;
  r->kv_norm = rs.kv_norm;
  r->ms = ms;
  r->history_len = 0;
}

std::vector<double> tol_vector(ikr_ctx* c, const double* tol) {
  const int n = c->occ.n;
  std::vector<double> t(n, 1e-12);
  if (tol) t.assign(tol, tol + n);
  for (double v : t) IKR_REQUIRE(v > 0.0 && std::isfinite(v), IKR_ERR_ARG, "tolerances must be positive");
  return t;
}

double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

ikr_status solve_any(ikr_ctx* c, int nrhs, const double* b, double* x, const ikr_solve_opts* opts,
                            ikr_report* report, cudaStream_t stream, bool adjoint) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  ikr_status worst = IKR_OK;
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(nrhs >= 0 && (nrhs == 0 || (b && x)), IKR_ERR_ARG, "invalid right-hand sides");
    ikr_solve_opts o;
    if (opts) o = *opts; else ikr_default_opts(&o);
    IKR_REQUIRE(o.strategy >= IKR_AGR && o.strategy <= IKR_FIXED, IKR_ERR_ARG, "unknown strategy");
    IKR_REQUIRE(o.precision == IKR_FP64 || o.precision == IKR_MIXED, IKR_ERR_ARG, "unknown precision");
    IKR_REQUIRE(o.cg_maxit >= 1, IKR_ERR_ARG, "cg_maxit must be >= 1");
    const char* env = std::getenv("IKR_BATCH");
    if (nrhs > 1 && !(env && env[0] == '0')) {
      try {
        gmres_solve_batch(c, nrhs, b, x, o, report, adjoint);
      } catch (const Error& e) {
        if (e.status != IKR_ERR_NOCONV && e.status != IKR_ERR_TIMEOUT) throw;
        c->err = e.what();
        worst = e.status;
      }
      return;
    }
    for (int r = 0; r < nrhs; ++r) {
      ikr_report* rep = report ? report + r : nullptr;
      try {
        gmres_solve(c, b + (size_t)r * c->Ng, x + (size_t)r * c->Ng, o, rep, adjoint);
      } catch (const Error& e) {
        if (e.status != IKR_ERR_NOCONV && e.status != IKR_ERR_TIMEOUT) throw;
        c->err = e.what();
        if (worst == IKR_OK) worst = e.status;
      }
    }
  });
  if (s != IKR_OK) return s;
  return worst;
}

}  // namespace

extern "C" {

void ikr_default_opts(ikr_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau = 1e-8;
  o->m = 20;
  o->strategy = IKR_BAL;
  o->precision = IKR_FP64;
  o->max_restarts = 20;
  o->cg_maxit = 400;
  o->kerker_alpha = 0.0;
  o->fixed_cg_tol = 1e-10;
  o->s0 = 1.0;
  o->use_x0 = 0;
  o->timeout_s = 0.0;
}

ikr_status ikr_setup_groundstate(const ikr_system* sys, const ikr_eigenpairs* eig, cudaStream_t stream,
                                 ikr_ctx** out) {
  if (!out) return IKR_ERR_ARG;
  *out = nullptr;
  ikr_ctx* c = new (std::nothrow) ikr_ctx();
  if (!c) return IKR_ERR_OOM;
  c->stream = stream;
  ikr_status s = guarded(c, [&] {
    setup_system(c, sys);
    ensure_pinned(c, 64);
    if (eig) set_eigenpairs(c, eig);
  });
  if (s != IKR_OK) {
    delete c;
    return s;
  }
  *out = c;
  return IKR_OK;
}

ikr_status ikr_set_eigenpairs(ikr_ctx* c, const ikr_eigenpairs* eig, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  return guarded(c, [&] { set_eigenpairs(c, eig); });
}

ikr_status ikr_set_nonlocal(ikr_ctx* c, int ncentres, const double* centres, const double* sigma, const double* D,
                            cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  return guarded(c, [&] {
    IKR_REQUIRE(!c->have_gs, IKR_ERR_STATE, "set the nonlocal part before the eigenpairs");
    set_nonlocal(c, ncentres, centres, sigma, D);
  });
}

ikr_status ikr_set_schur(ikr_ctx* c, int enable) {
  if (!c) return IKR_ERR_ARG;
  return guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(c->xmax >= 1, IKR_ERR_ARG, "no extra computed bands above N_occ,k");
    c->schur = enable != 0;
  });
}

ikr_status ikr_set_tensor_cores(ikr_ctx* c, int mode) {
  if (!c) return IKR_ERR_ARG;
  return guarded(c, [&] {
    IKR_REQUIRE(mode >= 0 && mode <= 2, IKR_ERR_ARG, "mode must be 0, 1 or 2");
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    c->tc_proj = mode != 0;
    if (mode != 0) c->tc_swizzle = mode == 1;
  });
}

ikr_status ikr_projection_coefficients(ikr_ctx* c, int k, int nvec, const void* y, int method, double* coef,
                                       cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  const bool old = c->tc_proj, old_swz = c->tc_swizzle;
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(k >= 0 && k < (int)c->k.size() && nvec >= 1 && y && coef, IKR_ERR_ARG, "invalid arguments");
    IKR_REQUIRE(method >= 0 && method <= 2, IKR_ERR_ARG, "method must be 0, 1 or 2");
    const KPoint& K = c->k[k];
    std::vector<int> kof(nvec, k), band(nvec, 0);
    SysList L;
    make_syslist(c, L, nvec, kof.data(), band.data());
    ensure_workspace(c, nvec);
    Workspace& w = c->ws;
    const int ld = c->ld;
    IKR_CUDA(cudaMemsetAsync(w.Z32.p, 0, sizeof(float2) * (size_t)nvec * ld, stream));
    IKR_CUDA(cudaMemcpy2DAsync(w.Z32.p, sizeof(float2) * ld, y, sizeof(float2) * K.nb, sizeof(float2) * K.nb, nvec,
                               cudaMemcpyDeviceToDevice, stream));
    c->tc_proj = method != 0;
    c->tc_swizzle = method != 2;
    double2* cf = reinterpret_cast<double2*>(w.coef.p);
    proj_coef<float>(c, L, w.Z32.p, ld, nullptr, cf);
    if (c->tc_proj) tc_check(c);
    std::vector<double2> h((size_t)nvec * std::max(c->noccmax, 1));
    IKR_CUDA(cudaMemcpyAsync(h.data(), cf, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, stream));
    IKR_CUDA(cudaStreamSynchronize(stream));
    for (int q = 0; q < nvec; ++q)
      for (int m = 0; m < K.nocc; ++m) {
        coef[2 * ((size_t)q * K.nocc + m)] = h[(size_t)q * c->noccmax + m].x;
        coef[2 * ((size_t)q * K.nocc + m) + 1] = h[(size_t)q * c->noccmax + m].y;
      }
  });
  c->tc_proj = old;
  c->tc_swizzle = old_swz;
  return s;
}

ikr_status ikr_project_out(ikr_ctx* c, int k, int nvec, void* y, int method, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  const bool old = c->tc_proj, old_swz = c->tc_swizzle;
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(k >= 0 && k < (int)c->k.size() && nvec >= 1 && y, IKR_ERR_ARG, "invalid arguments");
    IKR_REQUIRE(method >= 0 && method <= 2, IKR_ERR_ARG, "method must be 0, 1 or 2");
    const KPoint& K = c->k[k];
    std::vector<int> kof(nvec, k), band(nvec, 0);
    SysList L;
    make_syslist(c, L, nvec, kof.data(), band.data());
    ensure_workspace(c, nvec);
    Workspace& w = c->ws;
    const int ld = c->ld;
    IKR_CUDA(cudaMemsetAsync(w.Z32.p, 0, sizeof(float2) * (size_t)nvec * ld, stream));
    IKR_CUDA(cudaMemcpy2DAsync(w.Z32.p, sizeof(float2) * ld, y, sizeof(float2) * K.nb, sizeof(float2) * K.nb, nvec,
                               cudaMemcpyDeviceToDevice, stream));
    c->tc_proj = method != 0;
    c->tc_swizzle = method != 2;
    double2* cf = reinterpret_cast<double2*>(w.coef.p);
    proj_coef<float>(c, L, w.Z32.p, ld, nullptr, cf);
    proj_apply<float>(c, L, cf, w.Z32.p, 1.0f, -1.0f, w.Z32.p, ld, nullptr, nullptr, nullptr);
    if (c->tc_proj) tc_check(c);
    IKR_CUDA(cudaMemcpy2DAsync(y, sizeof(float2) * K.nb, w.Z32.p, sizeof(float2) * ld, sizeof(float2) * K.nb, nvec,
                               cudaMemcpyDeviceToDevice, stream));
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
  c->tc_proj = old;
  c->tc_swizzle = old_swz;
  return s;
}

ikr_status ikr_compute_eigenpairs(ikr_ctx* c, int nbands, double tol, int maxit, int degree, double* eigenvalues,
                                  int* iters, double* max_residual, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  bool conv = true;
  ikr_status s = guarded(c, [&] {
    std::vector<DBuf<double2>> vecs;
    std::vector<double> eps;
    const std::vector<EigenStats> st = compute_eigenpairs(c, nbands, tol, maxit, degree, vecs, eps);
    std::vector<const double*> ptrs(vecs.size());
    for (size_t k = 0; k < vecs.size(); ++k) {
      ptrs[k] = reinterpret_cast<const double*>(vecs[k].p);
      if (iters) iters[k] = st[k].iters;
      if (max_residual) max_residual[k] = st[k].max_residual;
      conv = conv && st[k].max_residual <= tol;
    }
    if (eigenvalues) std::copy(eps.begin(), eps.end(), eigenvalues);
    ikr_eigenpairs e;
    e.nbands = nbands;
    e.eigenvalues = eps.data();
    e.eigenvectors = ptrs.data();
    set_eigenpairs(c, &e);
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
  if (s == IKR_OK && !conv) {
    c->err = "eigensolver stopped at maxit above tol";
    return IKR_ERR_NOCONV;
  }
  return s;
}

ikr_status ikr_autotune(ikr_ctx* c, double* out, cudaStream_t stream) {
  if (!c || !out) return IKR_ERR_ARG;
  c->stream = stream;
  return guarded(c, [&] { ikr::autotune(c, out); });
}

ikr_status ikr_device_peaks(double* out, cudaStream_t stream) {
  if (!out) return IKR_ERR_ARG;
  try {
    ikr::device_peaks(out, stream);
  } catch (const ikr::Error& e) {
    return e.status;
  } catch (...) {
    return IKR_ERR_CUDA;
  }
  return IKR_OK;
}

ikr_status ikr_hermitian_eigh(int n, const double* a, double* w, double* v) {
  if (n < 1 || !a || !w || !v) return IKR_ERR_ARG;
  try {
    std::vector<std::complex<double>> A((size_t)n * n), V;
    for (size_t i = 0; i < (size_t)n * n; ++i) A[i] = {a[2 * i], a[2 * i + 1]};
    std::vector<double> ww;
    herm_jacobi(n, A, ww, V);
    for (int i = 0; i < n; ++i) w[i] = ww[i];
    for (size_t i = 0; i < (size_t)n * n; ++i) {
      v[2 * i] = V[i].real();
      v[2 * i + 1] = V[i].imag();
    }
  } catch (...) {
    return IKR_ERR_ARG;
  }
  return IKR_OK;
}

int ikr_num_kpoints(const ikr_ctx* c) { return c ? (int)c->k.size() : 0; }

ikr_status ikr_basis_size(const ikr_ctx* c, int k, int* nb) {
  if (!c || !nb || k < 0 || k >= (int)c->k.size()) return IKR_ERR_ARG;
  *nb = c->k[k].nb;
  return IKR_OK;
}

ikr_status ikr_basis_millers(const ikr_ctx* c, int k, int* millers) {
  if (!c || !millers || k < 0 || k >= (int)c->k.size()) return IKR_ERR_ARG;
  std::memcpy(millers, c->k[k].miller.data(), sizeof(int) * c->k[k].miller.size());
  return IKR_OK;
}

ikr_status ikr_groundstate_info(const ikr_ctx* cc, double* f, int* nocc, double* eF, double* rho_device,
                                cudaStream_t stream) {
  ikr_ctx* c = const_cast<ikr_ctx*>(cc);
  if (!c) return IKR_ERR_ARG;
  return guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    for (size_t k = 0; k < c->k.size(); ++k) {
      const KPoint& K = c->k[k];
      if (f) std::memcpy(f + k * K.nbands, K.f.data(), sizeof(double) * K.nbands);
      if (nocc) nocc[k] = K.nocc;
    }
    if (eF) *eF = c->eF;
    if (rho_device) {
      IKR_CUDA(cudaMemcpyAsync(rho_device, c->d_rho.p, sizeof(double) * c->Ng, cudaMemcpyDeviceToDevice, stream));
      IKR_CUDA(cudaStreamSynchronize(stream));
    }
  });
}

ikr_status ikr_apply_hamiltonian(ikr_ctx* c, int k, const void* psi, void* hpsi, int nvec, int precision,
                                 cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  return guarded(c, [&] {
    IKR_REQUIRE(k >= 0 && k < (int)c->k.size(), IKR_ERR_ARG, "k out of range");
    IKR_REQUIRE(nvec >= 0, IKR_ERR_ARG, "nvec must be >= 0");
    if (nvec == 0) return;
    IKR_REQUIRE(psi && hpsi && psi != hpsi, IKR_ERR_ARG, "psi and hpsi must be distinct device pointers");
    const int nb = c->k[k].nb;
    if (precision == IKR_MIXED) {
      hamiltonian<float>(c, k, static_cast<const float2*>(psi), static_cast<float2*>(hpsi), nb, nvec);
    } else {
      // IKR_DF64: the plane pass in double-float, as in the mixed path's FP64-accurate sections
      const bool old = c->emulate_fp64;
      c->emulate_fp64 = precision == IKR_DF64;
      try {
        hamiltonian<double>(c, k, static_cast<const double2*>(psi), static_cast<double2*>(hpsi), nb, nvec);
      } catch (...) {
        c->emulate_fp64 = old;
        throw;
      }
      c->emulate_fp64 = old;
    }
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
}

ikr_status ikr_apply_hamiltonian_noalloc(ikr_ctx* c, int k, const void* psi, void* hpsi, int nvec,
                                         cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  return guarded(c, [&] {
    IKR_REQUIRE(k >= 0 && k < (int)c->k.size(), IKR_ERR_ARG, "k out of range");
    IKR_REQUIRE(nvec >= 0, IKR_ERR_ARG, "nvec must be >= 0");
    if (nvec == 0) return;
    IKR_REQUIRE(psi && hpsi && psi != hpsi, IKR_ERR_ARG, "psi and hpsi must be distinct device pointers");
    IKR_REQUIRE(c->nproj == 0, IKR_ERR_ARG, "the no-allocation H_k has no nonlocal part");
    hamiltonian_noalloc(c, k, static_cast<const double2*>(psi), static_cast<double2*>(hpsi), nvec);
  });
}

ikr_status ikr_solve_sternheimer(ikr_ctx* c, int nsys, const int* k_of, const int* band_of, const void* rhs,
                                 void* x, int ld, const double* tol, int maxit, int precision, int* iters_out,
                                 double* resid_out, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  ikr_status result = IKR_OK;
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(nsys >= 0 && maxit >= 1, IKR_ERR_ARG, "invalid nsys or maxit");
    if (nsys == 0) return;
    IKR_REQUIRE(k_of && band_of && rhs && x && tol, IKR_ERR_ARG, "NULL argument");
    SysList L;
    make_syslist(c, L, nsys, k_of, band_of);
    int nbmax = 0;
    for (int s2 = 0; s2 < nsys; ++s2) {
      const KPoint& K = c->k[k_of[s2]];
      IKR_REQUIRE(band_of[s2] < K.nocc, IKR_ERR_ARG, "band must be occupied");
      IKR_REQUIRE(tol[s2] > 0.0, IKR_ERR_ARG, "tolerances must be positive");
      nbmax = std::max(nbmax, K.nb);
    }
    IKR_REQUIRE(ld >= nbmax, IKR_ERR_ARG, "ld must be >= the largest basis size");
    ensure_workspace(c, nsys);
    Workspace& w = c->ws;
    const cudaStream_t st = c->stream;
    IKR_CUDA(cudaMemsetAsync(w.Y.p, 0, sizeof(double2) * nsys * c->ld, st));
    for (int s2 = 0; s2 < nsys; ++s2) {
      const int nb = c->k[k_of[s2]].nb;
      IKR_CUDA(cudaMemcpyAsync(w.Y.p + (size_t)s2 * c->ld, static_cast<const double2*>(rhs) + (size_t)s2 * ld,
                               sizeof(double2) * nb, cudaMemcpyDeviceToDevice, st));
    }
    // B = Q rhs
    double2* coef = reinterpret_cast<double2*>(w.coefM.p);
    proj_coef<double>(c, L, w.Y.p, c->ld, nullptr, coef);
    proj_apply<double>(c, L, coef, w.Y.p, 1.0, -1.0, w.B.p, c->ld, nullptr, nullptr, nullptr);
    std::vector<double> shift(nsys), kappa(nsys), t(tol, tol + nsys);
    for (int s2 = 0; s2 < nsys; ++s2) {
      const KPoint& K = c->k[k_of[s2]];
      shift[s2] = K.eps[band_of[s2]];
      int occ_index = 0;
      for (int q = 0; q < k_of[s2]; ++q) occ_index += c->k[q].nocc;
      kappa[s2] = c->h_kappa_occ[occ_index + band_of[s2]];
    }
    CgStats stt = (precision == IKR_MIXED) ? mixed_solve(c, L, w.B.p, w.X.p, shift, kappa, t, maxit)
                                           : cg_solve<double>(c, L, w.B.p, w.X.p, shift, kappa, t, maxit);
    for (int s2 = 0; s2 < nsys; ++s2) {
      const int nb = c->k[k_of[s2]].nb;
      IKR_CUDA(cudaMemcpyAsync(static_cast<double2*>(x) + (size_t)s2 * ld, w.X.p + (size_t)s2 * c->ld,
                               sizeof(double2) * nb, cudaMemcpyDeviceToDevice, st));
      if (iters_out) iters_out[s2] = stt.iters[s2];
      if (resid_out) resid_out[s2] = stt.res[s2];
    }
    IKR_CUDA(cudaStreamSynchronize(st));
    if (stt.numeric) result = IKR_ERR_NUMERIC;
    else if (stt.noconv) result = IKR_ERR_NOCONV;
  });
  return s != IKR_OK ? s : result;
}

ikr_status ikr_apply_chi0(ikr_ctx* c, const double* dV, double* drho, const double* tol, int precision,
                          ikr_report* report, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  RunStats rs;
  const double t0 = wall_ms();
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(dV && drho && dV != drho, IKR_ERR_ARG, "dV and drho must be distinct device pointers");
    const std::vector<double> t = tol_vector(c, tol);
    chi0_core(c, dV, nullptr, t, 1000, precision, drho, rs);
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
  fill_report(report, rs, wall_ms() - t0);
  if (report) report->status = s;
  if (s == IKR_OK && rs.cg_numeric) s = IKR_ERR_NUMERIC;
  if (s == IKR_OK && rs.cg_noconv) s = IKR_ERR_NOCONV;
  return s;
}

ikr_status ikr_apply_dielectric(ikr_ctx* c, const double* v, double* Ev, const double* tol, int precision,
                                ikr_report* report, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  RunStats rs;
  const double t0 = wall_ms();
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(v && Ev && v != Ev, IKR_ERR_ARG, "v and Ev must be distinct device pointers");
    const std::vector<double> t = tol_vector(c, tol);
    dielectric_core(c, v, Ev, [&](double) { return t; }, 1000, precision, rs);
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
  fill_report(report, rs, wall_ms() - t0);
  if (report) report->status = s;
  if (s == IKR_OK && rs.cg_numeric) s = IKR_ERR_NUMERIC;
  if (s == IKR_OK && rs.cg_noconv) s = IKR_ERR_NOCONV;
  return s;
}

ikr_status ikr_solve_response(ikr_ctx* c, int nrhs, const double* b, double* x, const ikr_solve_opts* opts,
                              ikr_report* report, cudaStream_t stream) {
  return solve_any(c, nrhs, b, x, opts, report, stream, false);
}

ikr_status ikr_apply_dielectric_adjoint(ikr_ctx* c, const double* v, double* Ev, const double* tol, int precision,
                                        ikr_report* report, cudaStream_t stream) {
  if (!c) return IKR_ERR_ARG;
  c->stream = stream;
  RunStats rs;
  const double t0 = wall_ms();
  ikr_status s = guarded(c, [&] {
    IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
    IKR_REQUIRE(v && Ev && v != Ev, IKR_ERR_ARG, "v and Ev must be distinct device pointers");
    const std::vector<double> t = tol_vector(c, tol);
    dielectric_adjoint_core(c, v, Ev, [&](double) { return t; }, 1000, precision, rs);
    IKR_CUDA(cudaStreamSynchronize(stream));
  });
  fill_report(report, rs, wall_ms() - t0);
  if (report) report->status = s;
  if (s == IKR_OK && rs.cg_numeric) s = IKR_ERR_NUMERIC;
  if (s == IKR_OK && rs.cg_noconv) s = IKR_ERR_NOCONV;
  return s;
}

ikr_status ikr_solve_response_adjoint(ikr_ctx* c, int nrhs, const double* g, double* lambda,
                                      const ikr_solve_opts* opts, ikr_report* report, cudaStream_t stream) {
  return solve_any(c, nrhs, g, lambda, opts, report, stream, true);
}

void ikr_destroy(ikr_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  delete c;
}

const char* ikr_last_error(const ikr_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

const char* ikr_status_string(int s) {
  switch (s) {
    case IKR_OK: return "IKR_OK";
    case IKR_ERR_ARG: return "IKR_ERR_ARG";
    case IKR_ERR_CUDA: return "IKR_ERR_CUDA";
    case IKR_ERR_OOM: return "IKR_ERR_OOM";
    case IKR_ERR_NOGAP: return "IKR_ERR_NOGAP";
    case IKR_ERR_NOCONV: return "IKR_ERR_NOCONV";
    case IKR_ERR_NUMERIC: return "IKR_ERR_NUMERIC";
    case IKR_ERR_TIMEOUT: return "IKR_ERR_TIMEOUT";
    case IKR_ERR_STATE: return "IKR_ERR_STATE";
    default: return "IKR_UNKNOWN";
  }
}

const char* ikr_version(void) { return "ikr 0.1 (sm_103a)"; }

ikr_status ikr_profile_start(ikr_ctx* c, unsigned mask) {
  if (!c) return IKR_ERR_ARG;
  for (int i = 0; i < kNumKid; ++i) {
    c->prof.launches[i] = 0;
    c->prof.units32[i] = 0;
    c->prof.units64[i] = 0;
    c->prof.used[i] = 0;
    c->prof.used[kNumKid + i] = 0;
  }
  c->prof.mask = mask;
  return IKR_OK;
}

int ikr_profile_read(ikr_ctx* c, ikr_kernel_stat* out, int cap) {
  static const char* names[kNumKid] = {"z_inverse", "plane", "z_forward", "proj_coef", "proj_apply",
                                       "cg_vector", "density", "grid_fft", "grid_ops", "scalar"};
  if (!c) return 0;
  cudaStreamSynchronize(c->stream);
  const int n = cap < (int)kNumKid ? cap : (int)kNumKid;
  for (int i = 0; i < n && out; ++i) {
    out[i].name = names[i];
    out[i].launches = c->prof.launches[i];
    double ms[2] = {0.0, 0.0};
    long long calls[2] = {0, 0};
    for (int prec = 0; prec < 2; ++prec) {
      const int id = i + prec * kNumKid;
      const size_t pairs = c->prof.used[id] / 2;
      for (size_t j = 0; j < pairs; ++j) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->prof.ev[id][2 * j], c->prof.ev[id][2 * j + 1]) == cudaSuccess) ms[prec] += t;
      }
      calls[prec] = (long long)pairs;
    }
    out[i].timed_calls = calls[0] + calls[1];
    out[i].ms = ms[0] + ms[1];
    out[i].ms_fp32 = ms[0];
    out[i].ms_fp64 = ms[1];
    out[i].timed_calls_fp32 = calls[0];
    out[i].timed_calls_fp64 = calls[1];
    out[i].units_fp32 = c->prof.units32[i];
    out[i].units_fp64 = c->prof.units64[i];
  }
  return (int)kNumKid;
}

ikr_status ikr_fft_geometry(const ikr_ctx* c, int* out) {
  if (!c || !out) return IKR_ERR_ARG;
  out[0] = c->N[0];
  out[1] = c->N[1];
  out[2] = c->N[2];
  out[3] = c->nc;
  out[4] = c->nxa;
  return IKR_OK;
}

}  // extern "C"
