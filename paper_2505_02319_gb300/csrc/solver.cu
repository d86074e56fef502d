// Host orchestration of the hot path: H_k applications, the batched
// Sternheimer CG, chi0, the dielectric adjoint E and Algorithm 1.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>

#include "ops.hpp"
#include "solver.hpp"

namespace ikr {

namespace {

template <typename R> struct Bufs;
template <> struct Bufs<double> {
  static CgVecs<double> get(ikr_ctx* c) {
    return {c->ws.X.p, c->ws.R.p, c->ws.P.p, c->ws.Z.p, c->ws.W.p, nullptr};
  }
  static const double* pot(ikr_ctx* c) { return c->d_Vt.p; }
  static double2* b1(ikr_ctx* c) { return c->ws.b1.p; }
  static double2* b4(ikr_ctx* c) { return c->ws.b4.p; }
};
template <> struct Bufs<float> {
  static CgVecs<float> get(ikr_ctx* c) {
    return {c->ws.X32.p, c->ws.R32.p, c->ws.P32.p, c->ws.Z32.p, c->ws.W32.p, nullptr};
  }
  static const float* pot(ikr_ctx* c) { return c->d_Vt32.p; }
  static float2* b1(ikr_ctx* c) { return reinterpret_cast<float2*>(c->ws.b1.p); }
  static float2* b4(ikr_ctx* c) { return reinterpret_cast<float2*>(c->ws.b4.p); }
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// Buffers for n systems of orbital size ld.
void ensure_workspace(ikr_ctx* c, int n) {
  Workspace& w = c->ws;
  const size_t nv = (size_t)std::max(n, 1) * c->ld;
  const size_t nf = (size_t)std::max(n, 1) * c->N[2] * c->ncp;
  w.b1.reserve(nf);
  w.b4.reserve(nf);
  w.b1b.reserve(nf);
  for (auto* b : {&w.X, &w.R, &w.P, &w.Z, &w.W, &w.B, &w.Y}) b->reserve(nv);
  for (auto* b : {&w.X32, &w.R32, &w.P32, &w.Z32, &w.W32, &w.B32}) b->reserve(nv);
  const size_t nm = (size_t)std::max(n, 1) * std::max(std::max(c->noccmax, c->rmax), 1);
  w.coef.reserve(2 * nm);
  w.coefM.reserve(2 * nm);
  w.coefP.reserve(2 * nm);
  const int np = std::max(std::max(proj_chunks(c), cg_chunks(c)), zf_chunks(c));
  w.dpart.reserve((size_t)std::max(n, 1) * np);
  w.sys.reserve((size_t)kSysFields * std::max(n, 1));
  w.val.reserve(std::max(n, 1));
  w.active.reserve(std::max(n, 1));
  w.alist.reserve(std::max(n, 1));
  w.deps.reserve(std::max(n, 1));
  w.ca.reserve(std::max(n, 1));
  w.cb.reserve(std::max(n, 1));
  w.scal.reserve(64);
  for (auto* b : {&w.grid1, &w.grid2, &w.grid3, &w.grid4, &w.grid5, &w.grid6}) b->reserve(c->Ng);
}

// pinned host scratch for n doubles (and 64 ints)
void ensure_pinned(ikr_ctx* c, int n) {
  const size_t need = sizeof(double) * (size_t)std::max(n, 64);
  if (c->pinned_bytes >= need && c->h_pinned) return;
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  c->h_pinned = nullptr;
  void* p = nullptr;
  IKR_CUDA(cudaMallocHost(&p, need + 256));
  c->h_pinned = reinterpret_cast<int*>(p);
  c->h_pinned_d = reinterpret_cast<double*>(reinterpret_cast<char*>(p) + 256);
  c->pinned_bytes = need;
}

// --------------------------------------------------------------- H apply --

template <typename R>
void hamiltonian(ikr_ctx* c, int k, const C_t<R>* psi, C_t<R>* hpsi, int ld, int nvec) {
  const int batch = 512;
  for (int v0 = 0; v0 < nvec; v0 += batch) {
    const int nv = std::min(batch, nvec - v0);
    std::vector<int> kof(nv, k), band(nv, 0);
    SysList L;
    make_syslist(c, L, nv, kof.data(), band.data());
    ensure_workspace(c, nv);
    const C_t<R>* in = psi + (size_t)v0 * ld;
    C_t<R>* out = hpsi + (size_t)v0 * ld;
    launch_z_inverse<R>(c, L, in, ld, nullptr, Bufs<R>::b1(c));
    launch_plane<R>(c, L, Bufs<R>::b1(c), Bufs<R>::pot(c), nullptr, nullptr, Bufs<R>::b4(c));
    launch_z_forward<R>(c, L, Bufs<R>::b4(c), out, ld, in, nullptr, true, nullptr);
    apply_nonlocal<R>(c, L, in, ld, out, nullptr, nullptr, 0);
  }
}
template void hamiltonian<double>(ikr_ctx*, int, const double2*, double2*, int, int);
template void hamiltonian<float>(ikr_ctx*, int, const float2*, float2*, int, int);

// ---------------------------------------------------------- Sternheimer CG --
// Preconditioned CG on A_s = Q_k (H_k - eps_s) Q_k for every system s of L
// (eq. discretised_sternheimer), x0 = 0, >= 1 iteration, absolute stopping
// rule ||r|| <= tol_s.  The preconditioned residual z is re-projected by Q
// every iteration, which keeps the search direction p and the iterate x in
// range(Q) (Remark rmk:sternheimer_solution); A p = (H - eps) p then already
// lies in range(Q) up to the eigenpair residual.  Preconditioner:
// z = Q diag(1/(kappa_s + |k+G|^2/2)) r.  B must be in range(Q).
// zset: project z on the complement of another set of eigenvectors than Phi_k
// (the Schur-complement solves below: Q is then R = 1 - [Phi Psi][Phi Psi]^H
// and B must be in range(R)).
template <typename R>
CgStats cg_solve(ikr_ctx* c, const SysList& L, const C_t<R>* Bv, C_t<R>* Xv, const std::vector<double>& shift,
                 const std::vector<double>& kappa, const std::vector<double>& tol, int maxit, const OrbSet* zset) {
  const int n = L.n;
  CgStats st;
  st.iters.assign(n, 0);
  st.status.assign(n, 1);
  st.res.assign(n, 0.0);
  if (n == 0) return st;
  ensure_workspace(c, n);
  ensure_pinned(c, n);
  Workspace& w = c->ws;
  CgVecs<R> v = Bufs<R>::get(c);
  v.X = Xv;
  v.B = Bv;
  std::vector<double> hs((size_t)kSysFields * n, 0.0);
  for (int s = 0; s < n; ++s) {
    hs[kSysShift * n + s] = shift[s];
    hs[kSysKappa * n + s] = kappa[s];
    hs[kSysTol2 * n + s] = tol[s] * tol[s];
  }
  const cudaStream_t strm = c->stream;
  IKR_CUDA(cudaMemcpyAsync(w.sys.p, hs.data(), sizeof(double) * hs.size(), cudaMemcpyHostToDevice, strm));
  std::vector<int> ones(n, 1), all(n);
  for (int s = 0; s < n; ++s) all[s] = s;
  IKR_CUDA(cudaMemcpyAsync(w.active.p, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, strm));
  IKR_CUDA(cudaMemcpyAsync(w.alist.p, all.data(), sizeof(int) * n, cudaMemcpyHostToDevice, strm));
  double* sys = w.sys.p;
  int* act = w.active.p;
  const int pch = proj_chunks(c, (int)sizeof(R)), cch = cg_chunks(c);
  double2* coef = reinterpret_cast<double2*>(w.coef.p);
  // the masked projections below see at most mask_bound active systems (the count read
  // back after every iteration); cleared when the solve ends
  struct BoundGuard {
    ikr_ctx* c;
    ~BoundGuard() { c->mask_bound = 0; }
  } bound_guard{c};
  c->mask_bound = n;
  // initial state: x = 0, r = b, z = Q M^-1 r, p = z
  cg_xr<R>(c, L, 0, v, sys, act, nullptr);
  proj_coef<R>(c, L, v.Z, c->ld, act, coef, zset);
  proj_apply<R>(c, L, coef, v.Z, R(1), R(-1), v.Z, c->ld, v.R, w.dpart.p, act, zset);
  cg_scalars(c, 0, sys, w.dpart.p, pch, n, maxit, act, nullptr);
  cg_p<R>(c, L, 0, v, sys, act);
  c->active_hint = n;
  int* dcount = reinterpret_cast<int*>(w.scal.p + 40);
  for (int it = 1; it <= maxit; ++it) {
    // W = (H - eps) P and <P, W>.  P is in range(Q) (z is projected below), and
    // Phi^H (H - eps) P = (Lambda - eps) Phi^H P = 0 for the eigenvectors Phi, so
    // Q W = W up to the eigenpair residual: W is not projected again.
    launch_z_inverse<R>(c, L, v.P, c->ld, act, Bufs<R>::b1(c), w.alist.p, c->active_hint);
    launch_plane<R>(c, L, Bufs<R>::b1(c), Bufs<R>::pot(c), nullptr, act, Bufs<R>::b4(c), nullptr, w.alist.p,
                    c->active_hint);
    launch_z_forward<R>(c, L, Bufs<R>::b4(c), v.W, c->ld, v.P, sys + kSysShift * n, true, act, w.dpart.p,
                        w.alist.p, c->active_hint);
    // nonlocal part of A p, and <p, V_nl p> folded into the first <p, Ap> partial
    apply_nonlocal<R>(c, L, v.P, c->ld, v.W, act, w.dpart.p, zf_chunks(c, (int)sizeof(R)));
    bool fused = false;
    if constexpr (sizeof(R) == 4) {
      if (!c->tc_proj) {   // the fused kernel projects on the CUDA cores
        // alpha, x, r, stopping test, z = Q M^-1 r (or R M^-1 r), beta and p in one launch
        ProfScope ps(c, kKidCgVec, 1);
        IKR_CUDA(cudaMemsetAsync(dcount, 0, sizeof(int), strm));
        fused = launch_cg_fused(c, L, v.X, v.R, v.P, v.W, sys, maxit, act, dcount, w.alist.p, w.dpart.p,
                                zf_chunks(c, 4), zset);
      }
    }
    if (!fused) {
      cg_scalars(c, 1, sys, w.dpart.p, zf_chunks(c, (int)sizeof(R)), n, maxit, act, dcount);
      // x += alpha p, r -= alpha W, z = M^-1 r, ||r||^2, stopping test
      cg_xr<R>(c, L, 1, v, sys, act, w.dpart.p);
      cg_scalars(c, 2, sys, w.dpart.p, cch, n, maxit, act, dcount, w.alist.p);
      // z = Q z, beta, p = z + beta p
      proj_coef<R>(c, L, v.Z, c->ld, act, coef, zset);
      proj_apply<R>(c, L, coef, v.Z, R(1), R(-1), v.Z, c->ld, v.R, w.dpart.p, act, zset);
      cg_scalars(c, 3, sys, w.dpart.p, pch, n, maxit, act, nullptr);
      cg_p<R>(c, L, 1, v, sys, act);
    }
    IKR_CUDA(cudaMemcpyAsync(c->h_pinned, dcount, sizeof(int), cudaMemcpyDeviceToHost, strm));
    IKR_CUDA(cudaStreamSynchronize(strm));
    c->active_hint = c->h_pinned[0];
    c->mask_bound = std::max(c->h_pinned[0], 1);
    if (c->h_pinned[0] == 0) break;
  }
  IKR_CUDA(cudaMemcpyAsync(hs.data(), sys, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, strm));
  IKR_CUDA(cudaStreamSynchronize(strm));
  if (c->tc_proj) tc_check(c);
  for (int s = 0; s < n; ++s) {
    st.iters[s] = (int)hs[kSysIters * n + s];
    int code = (int)hs[kSysStatus * n + s];
    if (code == 0) code = 3;   // still running at the cap
    st.status[s] = code;
    st.res[s] = std::sqrt(std::max(0.0, hs[kSysRr * n + s]));
    st.n_ham += st.iters[s];
    st.max_iters = std::max(st.max_iters, st.iters[s]);
    if (code == 3) st.noconv++;
    if (code == 2) st.numeric++;
  }
  return st;
}
template CgStats cg_solve<double>(ikr_ctx*, const SysList&, const double2*, double2*, const std::vector<double>&,
                                  const std::vector<double>&, const std::vector<double>&, int, const OrbSet*);
template CgStats cg_solve<float>(ikr_ctx*, const SysList&, const float2*, float2*, const std::vector<double>&,
                                 const std::vector<double>&, const std::vector<double>&, int, const OrbSet*);

// The Sternheimer solves of chi0: the projected CG above, or (ikr_set_schur)
// its Schur-complement form over the extra computed bands Psi_k (Sec. 3.4.2,
// Sec. 4.1.2).  With R = Q - Psi Psi^H, the solution of Q (H - eps) Q x = b is
//   x = Psi a + y,   a = M^-1 (Psi^H b - W^H y),   M = Psi^H (H - eps) Psi,
//   S y = R b - W M^-1 Psi^H b,   S = R (H - eps) R - W M^-1 W^H,   W = R H Psi,
// and CG runs on S, whose smallest eigenvalue is eps_{Nocc+Nx+1} - eps instead
// of eps_{Nocc+1} - eps.  The extra bands are Rayleigh-Ritz pairs of the
// eigensolver, so M = diag(lambda_j - eps) and W = R (H Psi - Psi Lambda) is
// the size of their residual: the W terms are dropped, and the solve becomes
//   a = (lambda - eps)^-1 Psi^H b,  R (H - eps) R y = R b,  x = y + Psi a.
// B is overwritten with R b.
template <typename R>
CgStats sternheimer_solve(ikr_ctx* c, const SysList& L, C_t<R>* Bv, C_t<R>* Xv, const std::vector<double>& shift,
                          const std::vector<double>& kappa, const std::vector<double>& tol, int maxit) {
  if (!c->schur) return cg_solve<R>(c, L, Bv, Xv, shift, kappa, tol, maxit);
  const int n = L.n;
  if (n == 0) return cg_solve<R>(c, L, Bv, Xv, shift, kappa, tol, maxit);
  const OrbSet xs = extra_set(c), rs = schur_set(c);
  Workspace& w = c->ws;
  w.coefX.reserve((size_t)2 * n * std::max(c->xmax, 1));
  w.xshift.reserve(n);
  double2* a = reinterpret_cast<double2*>(w.coefX.p);
  proj_coef<R>(c, L, Bv, c->ld, nullptr, a, &xs);
  proj_apply<R>(c, L, a, Bv, R(1), R(-1), Bv, c->ld, nullptr, nullptr, nullptr, &xs);
  CgStats st = cg_solve<R>(c, L, Bv, Xv, shift, kappa, tol, maxit, &rs);
  IKR_CUDA(cudaMemcpyAsync(w.xshift.p, shift.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  deflate_coef(c, L, a, w.xshift.p);
  proj_apply<R>(c, L, a, Xv, R(1), R(1), Xv, c->ld, nullptr, nullptr, nullptr, &xs);
  return st;
}
template CgStats sternheimer_solve<double>(ikr_ctx*, const SysList&, double2*, double2*, const std::vector<double>&,
                                           const std::vector<double>&, const std::vector<double>&, int);
template CgStats sternheimer_solve<float>(ikr_ctx*, const SysList&, float2*, float2*, const std::vector<double>&,
                                          const std::vector<double>&, const std::vector<double>&, int);

// ------------------------------------------------------------------- chi0 --
// drho = chi0 (pot_scale * u) for the occupied systems (eqs. chi0, kchi0).
// fp32 = true runs the whole application (right-hand sides, CG, density) in
// FP32 with FP64 accumulation of the density; the callers choose it only when
// the error budget of the application is far above FP32 rounding.
namespace {
struct EmulateScope {   // FP64-accurate passes of the mixed path run in double-float
  ikr_ctx* c;
  bool old;
  EmulateScope(ikr_ctx* c_, bool on) : c(c_), old(c_->emulate_fp64) { c->emulate_fp64 = on; }
  ~EmulateScope() { c->emulate_fp64 = old; }
};
}  // namespace

void chi0_core(ikr_ctx* c, const double* u, const double* pot_scale, const std::vector<double>& tol,
               int maxit, int precision, double* drho, RunStats& rs, bool fp32) {
  IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
  EmulateScope em(c, precision == IKR_MIXED);
  const SysList& L = c->occ;
  const int n = L.n;
  IKR_REQUIRE((int)tol.size() == n, IKR_ERR_ARG, "one tolerance per occupied system is required");
  ensure_workspace(c, n);
  Workspace& w = c->ws;
  const int ld = c->ld;
  double2* M = reinterpret_cast<double2*>(w.coefM.p);
  double2* CP = reinterpret_cast<double2*>(w.coefP.p);
  std::vector<double> shift(n), kappa(n);
  for (int s = 0; s < n; ++s) {
    shift[s] = c->k[L.k[s]].eps[L.band[s]];
    kappa[s] = c->h_kappa_occ[s];
  }
  if (fp32) {
    float* upl = reinterpret_cast<float*>(w.grid1.p);
    float2* Y = w.W32.p;     // consumed before the CG reuses W32
    to_plane_layout<float>(c, u, upl, 1.0 / (double)c->Ng, pot_scale);
    launch_plane<float>(c, L, nullptr, upl, nullptr, nullptr, reinterpret_cast<float2*>(w.b4.p), c->d_psir32.p);
    launch_z_forward<float>(c, L, reinterpret_cast<float2*>(w.b4.p), Y, ld, nullptr, nullptr, false, nullptr);
    proj_coef<float>(c, L, Y, ld, nullptr, M);
    chi0_sys(c, L, M, w.deps.p, CP);
    proj_apply<float>(c, L, M, Y, -1.0f, 1.0f, w.B32.p, ld, nullptr, nullptr, nullptr);
    CgStats st = sternheimer_solve<float>(c, L, w.B32.p, w.X32.p, shift, kappa, tol, maxit);
    st.fp32 = true;
    rs.add(st);
    if (c->T > 0.0) proj_apply<float>(c, L, CP, w.X32.p, 1.0f, 1.0f, w.X32.p, ld, nullptr, nullptr, nullptr);
    occupation_response(c, w.deps.p, w.ca.p, w.cb.p, w.scal.p + 8);
    float2* b1b = reinterpret_cast<float2*>(w.b1b.p);
    launch_z_inverse<float>(c, L, w.X32.p, ld, nullptr, b1b);
    launch_density<float>(c, n, c->d_b1phi32.p, b1b, w.ca.p, w.cb.p, drho, 1.0 / c->volume, c->d_psir32.p);
    if (c->tc_proj) tc_check(c);
    return;
  }
  // y_s = F(u . F^-1 phi_s): plane pass on the cached real-space orbitals
  to_plane_layout<double>(c, u, w.grid1.p, 1.0 / (double)c->Ng, pot_scale);
  launch_plane<double>(c, L, c->d_b1phi.p, w.grid1.p, nullptr, nullptr, w.b4.p, c->d_psir.p);
  launch_z_forward<double>(c, L, w.b4.p, w.Y.p, ld, nullptr, nullptr, false, nullptr);
  // M = Phi^H Y; deps_s = M[s][n_s]; dphi^P coefficients (metals)
  proj_coef<double>(c, L, w.Y.p, ld, nullptr, M);
  chi0_sys(c, L, M, w.deps.p, CP);
  // b_s = -Q y_s
  proj_apply<double>(c, L, M, w.Y.p, -1.0, 1.0, w.B.p, ld, nullptr, nullptr, nullptr);
  CgStats st;
  if (precision == IKR_MIXED) {
    st = mixed_solve(c, L, w.B.p, w.X.p, shift, kappa, tol, maxit, true);
  } else {
    st = sternheimer_solve<double>(c, L, w.B.p, w.X.p, shift, kappa, tol, maxit);
  }
  rs.add(st);
  // dphi = dphi^Q + dphi^P
  if (c->T > 0.0) proj_apply<double>(c, L, CP, w.X.p, 1.0, 1.0, w.X.p, ld, nullptr, nullptr, nullptr);
  // df_s = f'_s (deps_s - deps_F), density coefficients
  occupation_response(c, w.deps.p, w.ca.p, w.cb.p, w.scal.p + 8);
  launch_z_inverse<double>(c, L, w.X.p, ld, nullptr, w.b1b.p);
  launch_density<double>(c, n, c->d_b1phi.p, w.b1b.p, w.ca.p, w.cb.p, drho, 1.0 / c->volume, c->d_psir.p);
  if (c->tc_proj) tc_check(c);   // the tensor-core products after the last CG of this application
}

// Ev = v - ||Kv|| chi0(Kv/||Kv||)  (eq. op_discretised).  tol_fn receives ||Kv||.
// allowed: the absolute error Algorithm 1 grants this application (0: none
// given).  With IKR_MIXED the application runs entirely in FP32 when its
// estimated FP32 rounding error, kFp32Rel ||v - Ev|| of the previous
// application, is at most allowed / 10.
constexpr double kFp32Rel = 1e-6;

void dielectric_core(ikr_ctx* c, const double* v, double* Ev, const TolFn& tol_fn, int maxit, int precision,
                     RunStats& rs, double allowed) {
  Workspace& w = c->ws;
  ensure_workspace(c, c->occ.n);
  double* Kv = w.grid2.p;
  double* nrm = w.scal.p;          // {||Kv||^2, ||Kv||, 1/||Kv||}
  apply_K(c, v, Kv, nrm);
  double h[3];
  IKR_CUDA(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  rs.kv_norm = h[1];
  if (!(h[1] > 0.0)) {
    IKR_CUDA(cudaMemcpyAsync(Ev, v, sizeof(double) * c->Ng, cudaMemcpyDeviceToDevice, c->stream));
    return;
  }
  IKR_REQUIRE(std::isfinite(h[1]), IKR_ERR_NUMERIC, "non-finite ||Kv||");
  const std::vector<double> tol = tol_fn(h[1]);
  const bool fp32 = precision == IKR_MIXED && allowed > 0.0 && rs.last_dEv > 0.0 &&
                    10.0 * kFp32Rel * rs.last_dEv <= allowed;
  chi0_core(c, Kv, nrm + 2, tol, maxit, precision, w.grid3.p, rs, fp32);
  axpy(c, v, w.grid3.p, -1.0, nrm + 1, Ev);
  // ||v - Ev|| = ||Kv|| ||chi0 u|| for the next precision decision
  norm2(c, w.grid3.p, w.scal.p + 48);
  double d3[3];
  IKR_CUDA(cudaMemcpyAsync(d3, w.scal.p + 48, sizeof(d3), cudaMemcpyDeviceToHost, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  rs.last_dEv = h[1] * d3[1];
  rs.e_applies++;
}

// E^T v = v - K chi0 v = v - ||v|| K chi0(v / ||v||): the dielectric operator
// 1 - K chi0, the transpose of E for symmetric chi0 and K (Sec. 2.2).  The
// Sternheimer error enters through K after chi0, so the error bound of Lemma
// cgtol_E holds with ||K v_i|| replaced by ||K|| ||v_i||; tol_fn receives ||K||.
void dielectric_adjoint_core(ikr_ctx* c, const double* v, double* Ev, const TolFn& tol_fn, int maxit,
                             int precision, RunStats& rs, double allowed) {
  Workspace& w = c->ws;
  ensure_workspace(c, c->occ.n);
  double* nrm = w.scal.p;          // {||v||^2, ||v||, 1/||v||}
  norm2(c, v, nrm);
  double h[3];
  IKR_CUDA(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  if (!(h[1] > 0.0)) {
    IKR_CUDA(cudaMemcpyAsync(Ev, v, sizeof(double) * c->Ng, cudaMemcpyDeviceToDevice, c->stream));
    return;
  }
  IKR_REQUIRE(std::isfinite(h[1]), IKR_ERR_NUMERIC, "non-finite ||v||");
  rs.kv_norm = c->knorm;
  const std::vector<double> tol = tol_fn(c->knorm);
  const bool fp32 = precision == IKR_MIXED && allowed > 0.0 && rs.last_dEv > 0.0 &&
                    10.0 * kFp32Rel * rs.last_dEv <= allowed;
  chi0_core(c, v, nrm + 2, tol, maxit, precision, w.grid3.p, rs, fp32);
  apply_K(c, w.grid3.p, w.grid2.p, w.scal.p + 48);          // K chi0(v/||v||)
  axpy(c, v, w.grid2.p, -1.0, nrm + 1, Ev);
  double d3[3];
  IKR_CUDA(cudaMemcpyAsync(d3, w.scal.p + 48, sizeof(d3), cudaMemcpyDeviceToHost, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  rs.last_dEv = h[1] * d3[1];
  rs.e_applies++;
}

// ---------------------------------------------------------- Algorithm 1 --

// smallest singular value of the m x n (m >= n) column-major matrix a by
// one-sided Jacobi rotations (Hestenes).
double sigma_min(std::vector<double> a, int m, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int r = 0; r < m; ++r) {
          al += a[p * m + r] * a[p * m + r];
          be += a[q * m + r] * a[q * m + r];
          ga += a[p * m + r] * a[q * m + r];
        }
        if (ga == 0.0 || std::fabs(ga) <= 1e-17 * std::sqrt(al * be)) continue;
        off = std::max(off, std::fabs(ga) / std::sqrt(al * be));
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < m; ++r) {
          const double up = a[p * m + r], uq = a[q * m + r];
          a[p * m + r] = cs * up - sn * uq;
          a[q * m + r] = sn * up + cs * uq;
        }
      }
    if (off < 1e-15) break;
  }
  double smin = 1e300;
  for (int p = 0; p < n; ++p) {
    double s = 0;
    for (int r = 0; r < m; ++r) s += a[p * m + r] * a[p * m + r];
    smin = std::min(smin, std::sqrt(s));
  }
  return smin;
}


std::vector<double> strategy_tolerances(ikr_ctx* c, const ikr_solve_opts& o, int i, double s, double rprev,
                                        double kv_norm, double b_norm) {
  const SysList& L = c->occ;
  const int n = L.n;
  std::vector<double> t(n);
  const double tau = o.tau;
  int nocc_tot = 0;
  for (auto& K : c->k) nocc_tot += K.nocc;
  const double vol = c->volume, ng = (double)c->Ng, nmp = (double)c->k.size();
  for (int q = 0; q < n; ++q) {
    const KPoint& K = c->k[L.k[q]];
    const int b = L.band[q];
    const double f = K.f[b], wk = K.weight;
    double pf = 1.0;
    switch (o.strategy) {
      case IKR_D10: t[q] = tau / 10.0; continue;
      case IKR_D100: t[q] = tau / 100.0; continue;
      case IKR_D10N: t[q] = tau / (10.0 * b_norm); continue;
      case IKR_FIXED: t[q] = o.fixed_cg_tol; continue;
      case IKR_AGR: pf = 1.0; break;
      case IKR_BAL: pf = vol / (2.0 * f * wk * nocc_tot * std::sqrt(ng)); break;
      case IKR_GRT:
        pf = std::sqrt(vol) / (2.0 * f * wk * std::sqrt(ng) * std::sqrt((double)nocc_tot) * kv_norm * K.rownorm_re);
        break;
      case IKR_GRT_EXACT:
        pf = std::sqrt(vol) * (K.eps[K.nocc] - K.eps[b]) /
             (2.0 * f * wk * kv_norm * K.rownorm * nmp * std::sqrt(ng * K.nocc));
        break;
      default: throw Error(IKR_ERR_ARG, "unknown strategy");
    }
    t[q] = (i == 0) ? pf * tau / 3.0 : pf * s / (3.0 * o.m) * tau / rprev;
  }
  return t;
}

void gmres_solve(ikr_ctx* c, const double* b, double* x, const ikr_solve_opts& o, ikr_report* rep, bool adjoint) {
  IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
  IKR_REQUIRE(o.tau > 0 && o.m >= 1 && o.m <= 200, IKR_ERR_ARG, "invalid tau or m");
  const double t0 = now_ms();
  const int m = o.m;
  const size_t Ng = c->Ng;
  const cudaStream_t strm = c->stream;
  ensure_workspace(c, c->occ.n);
  Workspace& w = c->ws;
  w.gm_V.reserve((size_t)(m + 1) * Ng);
  w.gm_h.reserve(4096 + 304 * 256);
  double* V = w.gm_V.p;
  double* hdev = w.gm_h.p;          // [0, 256): Arnoldi coefficients
  double* wv = w.grid4.p;
  double* bb = w.grid5.p;           // b, or T b with Kerker
  double* r0 = w.grid6.p;
  const bool kerker = o.kerker_alpha > 0.0;
  RunStats rs;
  // norms helper
  auto norm = [&](const double* v) {
    norm2(c, v, w.scal.p + 16);
    double h[3];
    IKR_CUDA(cudaMemcpyAsync(h, w.scal.p + 16, sizeof(h), cudaMemcpyDeviceToHost, strm));
    IKR_CUDA(cudaStreamSynchronize(strm));
    return h[1];
  };
  if (kerker) apply_kerker(c, b, bb, o.kerker_alpha);
  else IKR_CUDA(cudaMemcpyAsync(bb, b, sizeof(double) * Ng, cudaMemcpyDeviceToDevice, strm));
  const double b_norm = norm(b);
  IKR_REQUIRE(std::isfinite(b_norm), IKR_ERR_NUMERIC, "non-finite right-hand side");
  bool x0_nonzero = o.use_x0 != 0;
  if (!x0_nonzero) IKR_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * Ng, strm));
  double s = o.s0 > 0 ? o.s0 : 1.0;
  int restarts = 0, steps = 0;
  double est = 0.0;
  double min_tol = 1e300, max_tol = 0.0;
  std::vector<double> hist;
  ikr_status status = IKR_OK;
  double first_tol = 0.0, first_kvn = 0.0;
  bool first_seen = false;
  auto track = [&](const std::vector<double>& t, double kvn) {
    if (!first_seen) {
      first_seen = true;
      first_kvn = kvn;
      first_tol = 1e300;
      for (double v : t) first_tol = std::min(first_tol, v);
    }
    for (double v : t) {
      min_tol = std::min(min_tol, v);
      max_tol = std::max(max_tol, v);
    }
  };
  bool done = false;
  while (!done) {
    // Line 1: r~0 = b - E~(0) x0 (tolerances C_{0,n} tau / 3)
    if (x0_nonzero) {
      auto tf = [&](double kvn) {
        auto t = strategy_tolerances(c, o, 0, s, 1.0, kvn, b_norm);
        track(t, kvn);
        return t;
      };
      if (adjoint) dielectric_adjoint_core(c, x, wv, tf, o.cg_maxit, o.precision, rs, o.tau / 3.0);
      else dielectric_core(c, x, wv, tf, o.cg_maxit, o.precision, rs, o.tau / 3.0);
      if (kerker) {
        axpy(c, b, wv, -1.0, nullptr, r0);
        apply_kerker(c, r0, r0, o.kerker_alpha);
      } else {
        axpy(c, bb, wv, -1.0, nullptr, r0);
      }
    } else {
      IKR_CUDA(cudaMemcpyAsync(r0, bb, sizeof(double) * Ng, cudaMemcpyDeviceToDevice, strm));
    }
    const double beta = norm(r0);
    est = beta;
    IKR_REQUIRE(std::isfinite(beta), IKR_ERR_NUMERIC, "non-finite residual");
    if (!(beta > 0.0)) break;
    // v_1 = r0 / beta
    w.scal.reserve(64);
    {
      const double inv = 1.0 / beta;
      IKR_CUDA(cudaMemcpyAsync(w.scal.p + 24, &inv, sizeof(double), cudaMemcpyHostToDevice, strm));
      scale_by(c, r0, w.scal.p + 24, V);
    }
    std::vector<double> Hraw((size_t)(m + 1) * m, 0.0);   // column-major (m+1) x m
    std::vector<double> Rm((size_t)(m + 1) * m, 0.0);
    std::vector<double> cs(m), sn(m), g(m + 1, 0.0);
    g[0] = beta;
    double rprev = beta;
    int i = 0;
    for (i = 1; i <= m; ++i) {
      if (o.timeout_s > 0 && (now_ms() - t0) > 1000.0 * o.timeout_s) {
        status = IKR_ERR_TIMEOUT;
        break;
      }
      auto tf = [&](double kvn) {
        auto t = strategy_tolerances(c, o, i, s, rprev, kvn, b_norm);
        track(t, kvn);
        return t;
      };
      if (adjoint)
        dielectric_adjoint_core(c, V + (size_t)(i - 1) * Ng, wv, tf, o.cg_maxit, o.precision, rs,
                                s / (3.0 * m) * o.tau / rprev);
      else
        dielectric_core(c, V + (size_t)(i - 1) * Ng, wv, tf, o.cg_maxit, o.precision, rs,
                        s / (3.0 * m) * o.tau / rprev);
      if (kerker) apply_kerker(c, wv, wv, o.kerker_alpha);
      steps++;
      // classical Gram-Schmidt with one reorthogonalisation pass (FP64)
      multidot(c, V, i, wv, hdev, 0);
      sub_combination(c, V, i, hdev, wv);
      multidot(c, V, i, wv, hdev + 256, 0);
      sub_combination(c, V, i, hdev + 256, wv);
      std::vector<double> h1(i), h2(i);
      IKR_CUDA(cudaMemcpyAsync(h1.data(), hdev, sizeof(double) * i, cudaMemcpyDeviceToHost, strm));
      IKR_CUDA(cudaMemcpyAsync(h2.data(), hdev + 256, sizeof(double) * i, cudaMemcpyDeviceToHost, strm));
      const double hn = norm(wv);
      for (int j = 0; j < i; ++j) Hraw[(size_t)(i - 1) * (m + 1) + j] = h1[j] + h2[j];
      Hraw[(size_t)(i - 1) * (m + 1) + i] = hn;
      if (hn > 0.0) {
        const double inv = 1.0 / hn;
        IKR_CUDA(cudaMemcpyAsync(w.scal.p + 24, &inv, sizeof(double), cudaMemcpyHostToDevice, strm));
        scale_by(c, wv, w.scal.p + 24, V + (size_t)i * Ng);
      }
      // Givens update of the least-squares problem (eq. small_ls)
      for (int j = 0; j <= i; ++j) Rm[(size_t)(i - 1) * (m + 1) + j] = Hraw[(size_t)(i - 1) * (m + 1) + j];
      double* col = &Rm[(size_t)(i - 1) * (m + 1)];
      for (int j = 0; j < i - 1; ++j) {
        const double t = cs[j] * col[j] + sn[j] * col[j + 1];
        col[j + 1] = -sn[j] * col[j] + cs[j] * col[j + 1];
        col[j] = t;
      }
      const double rho = std::hypot(col[i - 1], col[i]);
      cs[i - 1] = rho > 0 ? col[i - 1] / rho : 1.0;
      sn[i - 1] = rho > 0 ? col[i] / rho : 0.0;
      col[i - 1] = rho;
      col[i] = 0.0;
      g[i] = -sn[i - 1] * g[i - 1];
      g[i - 1] = cs[i - 1] * g[i - 1];
      const double rn = std::fabs(g[i]);
      est = rn;
      rprev = rn;
      hist.push_back(rn);
      const bool conv = rn <= o.tau / 3.0;
      if (conv || i == m || hn == 0.0) {
        // sigma_i(H_i), y_i, x = x0 + V_i y_i
        std::vector<double> Hs((size_t)(i + 1) * i);
        for (int q = 0; q < i; ++q)
          for (int r = 0; r <= i; ++r) Hs[(size_t)q * (i + 1) + r] = Hraw[(size_t)q * (m + 1) + r];
        const double sig = sigma_min(Hs, i + 1, i);
        std::vector<double> y(i);
        for (int r = i - 1; r >= 0; --r) {
          double a = g[r];
          for (int q = r + 1; q < i; ++q) a -= Rm[(size_t)q * (m + 1) + r] * y[q];
          y[r] = a / Rm[(size_t)r * (m + 1) + r];
        }
        IKR_CUDA(cudaMemcpyAsync(hdev + 512, y.data(), sizeof(double) * i, cudaMemcpyHostToDevice, strm));
        add_combination(c, V, i, hdev + 512, x0_nonzero ? x : nullptr, x);
        x0_nonzero = true;
        if ((conv || hn == 0.0) && s <= sig) {
          done = true;
        } else {
          s = sig;
          restarts++;
        }
        rs.sigma = sig;
        break;
      }
    }
    if (status != IKR_OK) break;
    if (!done && restarts > o.max_restarts) {
      status = IKR_ERR_NOCONV;
      break;
    }
  }
  IKR_CUDA(cudaStreamSynchronize(strm));
  if (rs.cg_noconv > 0 && status == IKR_OK) status = IKR_OK;  // reported, not fatal
  if (rep) {
    rep->status = status;
    rep->outer_iters = steps;
    rep->restarts = restarts;
    rep->e_applies = rs.e_applies;
    rep->e_applies_fp32 = rs.e_applies_fp32;
    rep->n_ham = rs.n_ham;
    rep->n_ham_fp64 = rs.n_ham_fp64;
    rep->cg_max_iters = rs.cg_max_iters;
    rep->cg_noconv = rs.cg_noconv;
    rep->est_residual = est;
    rep->sigma = s;
    rep->b_norm = b_norm;
    rep->kv_norm = rs.kv_norm;
    rep->min_cg_tol = min_tol;
    rep->max_cg_tol = max_tol;
    rep->first_min_cg_tol = first_tol;
    rep->first_kv_norm = first_kvn;
    rep->ms = now_ms() - t0;
    rep->history_len = 0;
    if (rep->history && rep->history_cap > 0) {
      const int nh = std::min<int>(rep->history_cap, (int)hist.size());
      for (int q = 0; q < nh; ++q) rep->history[q] = hist[q];
      rep->history_len = nh;
    }
  }
  if (status != IKR_OK) throw Error(status, status == IKR_ERR_TIMEOUT ? "timeout" : "GMRES did not converge");
}

}  // namespace ikr
