// Several right-hand sides in lockstep: Algorithm 1 for each of them, with
// the E applications of one round batched.
//
// A batch of perturbations dV_r (the differentiated workload: one response
// per bump or atom displacement) gives independent Dyson equations
// E drho_r = b_r.  Each keeps its own GMRES state (Krylov basis, Hessenberg
// matrix, restarts, tolerances); per round every unfinished one asks for one
// E application (a Krylov step or the residual after a restart).  The
// right-hand-side passes and the densities of these applications run per
// right-hand side, but their Sternheimer equations (S per application) are
// gathered into one k-grouped system list and solved by one batched CG, so
// that a few dozen right-hand sides of a small cell fill the GPU that the S
// systems of one application leave mostly idle.  The arithmetic of every
// system is the same as in a solve of its right-hand side alone.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "solver.hpp"

namespace ikr {

namespace {

struct EmulateOn {   // FP64-accurate passes of the mixed path in double-float
  ikr_ctx* c;
  bool old;
  EmulateOn(ikr_ctx* c_, bool on) : c(c_), old(c_->emulate_fp64) { c->emulate_fp64 = on; }
  ~EmulateOn() { c->emulate_fp64 = old; }
};

// dst[q] = src[map[q]] (gather) or dst[map[q]] = src[q] (scatter), ld complex each
__global__ void k_move_sys(const double2* __restrict__ src, const int* __restrict__ map, int ld, int n, int scatter,
                           double2* __restrict__ dst) {
  const int q = blockIdx.y;
  const int g = blockIdx.x * 256 + threadIdx.x;
  if (q >= n || g >= ld) return;
  const size_t a = (size_t)q * ld + g, b = (size_t)map[q] * ld + g;
  if (scatter) dst[b] = src[a];
  else dst[a] = src[b];
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct BatchItem {
  const double* v = nullptr;   // E (or E^T) is applied to v
  double* Ev = nullptr;
  TolFn tol_fn;
  RunStats* rs = nullptr;
};

// E v_r = v_r - ||K v_r|| chi0(K v_r / ||K v_r||), or with adjoint
// E^T v_r = v_r - ||v_r|| K chi0(v_r / ||v_r||), for every item; one CG for
// the Sternheimer systems of all items.  The right-hand-side and density
// passes are FP64-accurate (double-float in the mixed path) for every item.
void dielectric_batch(ikr_ctx* c, std::vector<BatchItem>& items, int maxit, int precision, bool adjoint) {
  const int nr = (int)items.size();
  if (nr == 0) return;
  const SysList& L = c->occ;
  const int S = L.n, ld = c->ld, nk = (int)c->k.size();
  const size_t Ng = c->Ng;
  const cudaStream_t st = c->stream;
  ensure_workspace(c, S);
  Workspace& w = c->ws;
  EmulateOn em(c, precision == IKR_MIXED);
  const int nm = std::max(c->noccmax, 1);
  w.bu.reserve((size_t)nr * Ng);
  w.bdrho.reserve((size_t)nr * Ng);
  w.bnrm.reserve((size_t)8 * nr);
  w.bB.reserve((size_t)nr * S * ld);
  w.bX.reserve((size_t)nr * S * ld);
  w.bM.reserve((size_t)2 * nr * S * nm);
  w.bCP.reserve((size_t)2 * nr * S * nm);
  w.bdeps.reserve((size_t)nr * S);
  auto u_of = [&](int r) { return w.bu.p + (size_t)r * Ng; };
  auto nrm_of = [&](int r) { return w.bnrm.p + (size_t)8 * r; };   // {|x|^2, |x|, 1/|x|} then {|d|^2, |d|, 1/|d|}
  // 1. the potential chi0 acts on and its scale
  for (int r = 0; r < nr; ++r) {
    if (adjoint) norm2(c, items[r].v, nrm_of(r));
    else apply_K(c, items[r].v, u_of(r), nrm_of(r));
  }
  std::vector<double> hn((size_t)8 * nr);
  IKR_CUDA(cudaMemcpyAsync(hn.data(), w.bnrm.p, sizeof(double) * 8 * nr, cudaMemcpyDeviceToHost, st));
  IKR_CUDA(cudaStreamSynchronize(st));
  std::vector<int> live;
  std::vector<std::vector<double>> tol(nr);
  for (int r = 0; r < nr; ++r) {
    const double a = hn[(size_t)8 * r + 1];
    if (!(a > 0.0)) {   // E v = v
      IKR_CUDA(cudaMemcpyAsync(items[r].Ev, items[r].v, sizeof(double) * Ng, cudaMemcpyDeviceToDevice, st));
      continue;
    }
    IKR_REQUIRE(std::isfinite(a), IKR_ERR_NUMERIC, adjoint ? "non-finite ||v||" : "non-finite ||Kv||");
    items[r].rs->kv_norm = adjoint ? c->knorm : a;
    tol[r] = items[r].tol_fn(adjoint ? c->knorm : a);
    IKR_REQUIRE((int)tol[r].size() == S, IKR_ERR_ARG, "one tolerance per occupied system is required");
    live.push_back(r);
  }
  const int nl = (int)live.size();
  if (nl == 0) return;
  // 2. right-hand sides b_s = -Q F(u . F^-1 phi_s), deps_s and the dphi^P coefficients, per item
  for (int j = 0; j < nl; ++j) {
    const int r = live[j];
    const double* u = adjoint ? items[r].v : u_of(r);
    double2* M = reinterpret_cast<double2*>(w.bM.p) + (size_t)j * S * nm;
    double2* CP = reinterpret_cast<double2*>(w.bCP.p) + (size_t)j * S * nm;
    to_plane_layout<double>(c, u, w.grid1.p, 1.0 / (double)Ng, nrm_of(r) + 2);
    launch_plane<double>(c, L, c->d_b1phi.p, w.grid1.p, nullptr, nullptr, w.b4.p, c->d_psir.p);
    launch_z_forward<double>(c, L, w.b4.p, w.Y.p, ld, nullptr, nullptr, false, nullptr);
    proj_coef<double>(c, L, w.Y.p, ld, nullptr, M);
    chi0_sys(c, L, M, w.bdeps.p + (size_t)j * S, CP);
    proj_apply<double>(c, L, M, w.Y.p, -1.0, 1.0, w.bB.p + (size_t)j * S * ld, ld, nullptr, nullptr, nullptr);
  }
  // 3. one CG over the systems of all items, k-grouped: (k, item, band)
  const int nb = nl * S;
  std::vector<int> kof, band, map;
  std::vector<double> shift, kappa, tl;
  kof.reserve(nb);
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nl; ++j)
      for (int s = L.kstart[k]; s < L.kstart[k] + L.kcount[k]; ++s) {
        kof.push_back(k);
        band.push_back(L.band[s]);
        map.push_back(j * S + s);
        shift.push_back(c->k[k].eps[L.band[s]]);
        kappa.push_back(c->h_kappa_occ[s]);
        tl.push_back(tol[live[j]][s]);
      }
  if (c->batch_items != nl) {
    make_syslist(c, c->batch_list, nb, kof.data(), band.data());
    c->d_batch_map.reserve(nb);
    IKR_CUDA(cudaMemcpyAsync(c->d_batch_map.p, map.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    c->batch_items = nl;
  }
  const SysList& Lb = c->batch_list;
  ensure_workspace(c, nb);
  const dim3 mg((ld + 255) / 256, nb);
  {
    ProfScope ps(c, kKidCgVec, 1);
    k_move_sys<<<mg, 256, 0, st>>>(w.bB.p, c->d_batch_map.p, ld, nb, 0, w.B.p);
    IKR_CUDA(cudaGetLastError());
  }
  CgStats cs = (precision == IKR_MIXED) ? mixed_solve(c, Lb, w.B.p, w.X.p, shift, kappa, tl, maxit, true)
                                        : sternheimer_solve<double>(c, Lb, w.B.p, w.X.p, shift, kappa, tl, maxit);
  {
    ProfScope ps(c, kKidCgVec, 1);
    k_move_sys<<<mg, 256, 0, st>>>(w.X.p, c->d_batch_map.p, ld, nb, 1, w.bX.p);
    IKR_CUDA(cudaGetLastError());
  }
  // statistics of each item: its systems' share of the batched solve
  std::vector<CgStats> per(nl);
  for (auto& p : per) p.fp32 = cs.fp32;
  for (int q = 0; q < nb; ++q) {
    const int j = map[q] / S;
    CgStats& p = per[j];
    const int it = cs.iters[q], chk = cs.checks.empty() ? 0 : cs.checks[q];
    p.n_ham += it + chk;
    p.n_ham_fp64 += cs.fp32 ? chk : it;
    p.max_iters = std::max(p.max_iters, it);
    if (cs.status[q] == 3) p.noconv++;
    if (cs.status[q] == 2) p.numeric++;
  }
  // 4. dphi^P, occupation response and density per item; 5. E v
  ensure_workspace(c, S);
  for (int j = 0; j < nl; ++j) {
    const int r = live[j];
    double2* Xr = w.bX.p + (size_t)j * S * ld;
    const double2* CP = reinterpret_cast<const double2*>(w.bCP.p) + (size_t)j * S * nm;
    double* drho = w.bdrho.p + (size_t)j * Ng;
    if (c->T > 0.0) proj_apply<double>(c, L, CP, Xr, 1.0, 1.0, Xr, ld, nullptr, nullptr, nullptr);
    occupation_response(c, w.bdeps.p + (size_t)j * S, w.ca.p, w.cb.p, w.scal.p + 8);
    launch_z_inverse<double>(c, L, Xr, ld, nullptr, w.b1b.p);
    launch_density<double>(c, S, c->d_b1phi.p, w.b1b.p, w.ca.p, w.cb.p, drho, 1.0 / c->volume, c->d_psir.p);
    if (adjoint) {
      apply_K(c, drho, w.grid2.p, nrm_of(r) + 3);                 // K chi0(v/||v||)
      axpy(c, items[r].v, w.grid2.p, -1.0, nrm_of(r) + 1, items[r].Ev);
    } else {
      norm2(c, drho, nrm_of(r) + 3);                              // ||chi0 u||
      axpy(c, items[r].v, drho, -1.0, nrm_of(r) + 1, items[r].Ev);
    }
  }
  IKR_CUDA(cudaMemcpyAsync(hn.data(), w.bnrm.p, sizeof(double) * 8 * nr, cudaMemcpyDeviceToHost, st));
  IKR_CUDA(cudaStreamSynchronize(st));
  if (c->tc_proj) tc_check(c);
  for (int j = 0; j < nl; ++j) {
    const int r = live[j];
    RunStats& rs = *items[r].rs;
    rs.add(per[j]);
    rs.last_dEv = hn[(size_t)8 * r + 1] * hn[(size_t)8 * r + 4];   // ||x|| ||chi0 u|| (or ||K chi0 u||)
    rs.e_applies++;
  }
}

// ------------------------------------------------------ lockstep GMRES --

namespace {

enum Phase { kStart, kResidual, kStep, kDone };

struct Rhs {
  const double* b;
  double* x;
  double *bb, *r0, *wv, *V;    // device: b or T b, restart residual, E output, Krylov basis (m + 1) x Ng
  double b_norm = 0.0, s = 1.0, est = 0.0, rprev = 0.0, beta = 0.0;
  bool x0_nonzero = false;
  int restarts = 0, steps = 0, i = 0;
  Phase phase = kStart;
  ikr_status status = IKR_OK;
  std::vector<double> Hraw, Rm, cs, sn, g, hist;
  double min_tol = 1e300, max_tol = 0.0;
  double first_tol = 0.0, first_kvn = 0.0;
  bool first_seen = false;
  RunStats rs;
};

}  // namespace

void gmres_solve_batch(ikr_ctx* c, int nrhs, const double* b, double* x, const ikr_solve_opts& o,
                       ikr_report* reps, bool adjoint) {
  IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
  IKR_REQUIRE(o.tau > 0 && o.m >= 1 && o.m <= 200, IKR_ERR_ARG, "invalid tau or m");
  const double t0 = now_ms();
  const int m = o.m;
  const size_t Ng = c->Ng;
  const cudaStream_t strm = c->stream;
  ensure_workspace(c, c->occ.n);
  Workspace& w = c->ws;
  const size_t per = (size_t)(m + 4) * Ng;    // V, bb, r0, wv
  w.bgm.reserve((size_t)nrhs * per);
  w.gm_h.reserve(4096 + 304 * 256);
  double* hdev = w.gm_h.p;
  const bool kerker = o.kerker_alpha > 0.0;
  auto norm = [&](const double* v) {
    norm2(c, v, w.scal.p + 16);
    double h[3];
    IKR_CUDA(cudaMemcpyAsync(h, w.scal.p + 16, sizeof(h), cudaMemcpyDeviceToHost, strm));
    IKR_CUDA(cudaStreamSynchronize(strm));
    return h[1];
  };
  std::vector<Rhs> R(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    Rhs& q = R[r];
    q.b = b + (size_t)r * Ng;
    q.x = x + (size_t)r * Ng;
    double* base = w.bgm.p + (size_t)r * per;
    q.V = base;
    q.bb = base + (size_t)(m + 1) * Ng;
    q.r0 = q.bb + Ng;
    q.wv = q.r0 + Ng;
    if (kerker) apply_kerker(c, q.b, q.bb, o.kerker_alpha);
    else IKR_CUDA(cudaMemcpyAsync(q.bb, q.b, sizeof(double) * Ng, cudaMemcpyDeviceToDevice, strm));
    q.b_norm = norm(q.b);
    IKR_REQUIRE(std::isfinite(q.b_norm), IKR_ERR_NUMERIC, "non-finite right-hand side");
    q.x0_nonzero = o.use_x0 != 0;
    if (!q.x0_nonzero) IKR_CUDA(cudaMemsetAsync(q.x, 0, sizeof(double) * Ng, strm));
    q.s = o.s0 > 0 ? o.s0 : 1.0;
    q.Hraw.assign((size_t)(m + 1) * m, 0.0);
    q.Rm.assign((size_t)(m + 1) * m, 0.0);
    q.cs.assign(m, 0.0);
    q.sn.assign(m, 0.0);
    q.g.assign(m + 1, 0.0);
  }
  auto track = [](Rhs& q, const std::vector<double>& t, double kvn) {
    if (!q.first_seen) {
      q.first_seen = true;
      q.first_kvn = kvn;
      q.first_tol = 1e300;
      for (double v : t) q.first_tol = std::min(q.first_tol, v);
    }
    for (double v : t) {
      q.min_tol = std::min(q.min_tol, v);
      q.max_tol = std::max(q.max_tol, v);
    }
  };
  // a new cycle from r0: beta, v_1 (or the end when r0 = 0)
  auto start_cycle = [&](Rhs& q) {
    q.beta = norm(q.r0);
    q.est = q.beta;
    IKR_REQUIRE(std::isfinite(q.beta), IKR_ERR_NUMERIC, "non-finite residual");
    if (!(q.beta > 0.0)) {
      q.phase = kDone;
      return;
    }
    const double inv = 1.0 / q.beta;
    IKR_CUDA(cudaMemcpyAsync(w.scal.p + 24, &inv, sizeof(double), cudaMemcpyHostToDevice, strm));
    scale_by(c, q.r0, w.scal.p + 24, q.V);
    std::fill(q.Hraw.begin(), q.Hraw.end(), 0.0);
    std::fill(q.Rm.begin(), q.Rm.end(), 0.0);
    std::fill(q.g.begin(), q.g.end(), 0.0);
    q.g[0] = q.beta;
    q.rprev = q.beta;
    q.i = 1;
    q.phase = kStep;
  };
  // Arnoldi step i on wv = E v_i (lines of Algorithm 1 as in the single solver)
  auto arnoldi = [&](Rhs& q) {
    const int i = q.i;
    if (kerker) apply_kerker(c, q.wv, q.wv, o.kerker_alpha);
    q.steps++;
    multidot(c, q.V, i, q.wv, hdev, 0);
    sub_combination(c, q.V, i, hdev, q.wv);
    multidot(c, q.V, i, q.wv, hdev + 256, 0);
    sub_combination(c, q.V, i, hdev + 256, q.wv);
    std::vector<double> h1(i), h2(i);
    IKR_CUDA(cudaMemcpyAsync(h1.data(), hdev, sizeof(double) * i, cudaMemcpyDeviceToHost, strm));
    IKR_CUDA(cudaMemcpyAsync(h2.data(), hdev + 256, sizeof(double) * i, cudaMemcpyDeviceToHost, strm));
    const double hn = norm(q.wv);
    for (int j = 0; j < i; ++j) q.Hraw[(size_t)(i - 1) * (m + 1) + j] = h1[j] + h2[j];
    q.Hraw[(size_t)(i - 1) * (m + 1) + i] = hn;
    if (hn > 0.0) {
      const double inv = 1.0 / hn;
      IKR_CUDA(cudaMemcpyAsync(w.scal.p + 24, &inv, sizeof(double), cudaMemcpyHostToDevice, strm));
      scale_by(c, q.wv, w.scal.p + 24, q.V + (size_t)i * Ng);
    }
    for (int j = 0; j <= i; ++j) q.Rm[(size_t)(i - 1) * (m + 1) + j] = q.Hraw[(size_t)(i - 1) * (m + 1) + j];
    double* col = &q.Rm[(size_t)(i - 1) * (m + 1)];
    for (int j = 0; j < i - 1; ++j) {
      const double t = q.cs[j] * col[j] + q.sn[j] * col[j + 1];
      col[j + 1] = -q.sn[j] * col[j] + q.cs[j] * col[j + 1];
      col[j] = t;
    }
    const double rho = std::hypot(col[i - 1], col[i]);
    q.cs[i - 1] = rho > 0 ? col[i - 1] / rho : 1.0;
    q.sn[i - 1] = rho > 0 ? col[i] / rho : 0.0;
    col[i - 1] = rho;
    col[i] = 0.0;
    q.g[i] = -q.sn[i - 1] * q.g[i - 1];
    q.g[i - 1] = q.cs[i - 1] * q.g[i - 1];
    const double rn = std::fabs(q.g[i]);
    q.est = rn;
    q.rprev = rn;
    q.hist.push_back(rn);
    const bool conv = rn <= o.tau / 3.0;
    if (!(conv || i == m || hn == 0.0)) {
      q.i = i + 1;
      return;
    }
    std::vector<double> Hs((size_t)(i + 1) * i);
    for (int a = 0; a < i; ++a)
      for (int r = 0; r <= i; ++r) Hs[(size_t)a * (i + 1) + r] = q.Hraw[(size_t)a * (m + 1) + r];
    const double sig = sigma_min(Hs, i + 1, i);
    std::vector<double> y(i);
    for (int r = i - 1; r >= 0; --r) {
      double a = q.g[r];
      for (int p = r + 1; p < i; ++p) a -= q.Rm[(size_t)p * (m + 1) + r] * y[p];
      y[r] = a / q.Rm[(size_t)r * (m + 1) + r];
    }
    IKR_CUDA(cudaMemcpyAsync(hdev + 512, y.data(), sizeof(double) * i, cudaMemcpyHostToDevice, strm));
    add_combination(c, q.V, i, hdev + 512, q.x0_nonzero ? q.x : nullptr, q.x);
    q.x0_nonzero = true;
    q.rs.sigma = sig;
    if ((conv || hn == 0.0) && q.s <= sig) {
      q.phase = kDone;
      return;
    }
    q.s = sig;
    q.restarts++;
    if (q.restarts > o.max_restarts) {
      q.status = IKR_ERR_NOCONV;
      q.phase = kDone;
      return;
    }
    q.phase = kStart;
  };
  for (;;) {
    // advance every state to the point where it needs an E application
    std::vector<int> owners;
    std::vector<BatchItem> items;
    for (int r = 0; r < nrhs; ++r) {
      Rhs& q = R[r];
      if (q.phase == kStart) {
        if (q.x0_nonzero) {
          BatchItem it;
          it.v = q.x;
          it.Ev = q.wv;
          it.rs = &q.rs;
          it.tol_fn = [&, r](double kvn) {
            auto t = strategy_tolerances(c, o, 0, R[r].s, 1.0, kvn, R[r].b_norm);
            track(R[r], t, kvn);
            return t;
          };
          items.push_back(it);
          owners.push_back(r);
          q.phase = kResidual;
          continue;
        }
        IKR_CUDA(cudaMemcpyAsync(q.r0, q.bb, sizeof(double) * Ng, cudaMemcpyDeviceToDevice, strm));
        start_cycle(q);
      }
      if (q.phase == kStep) {
        if (o.timeout_s > 0 && (now_ms() - t0) > 1000.0 * o.timeout_s) {
          q.status = IKR_ERR_TIMEOUT;
          q.phase = kDone;
          continue;
        }
        BatchItem it;
        it.v = q.V + (size_t)(q.i - 1) * Ng;
        it.Ev = q.wv;
        it.rs = &q.rs;
        const int i = q.i;
        it.tol_fn = [&, r, i](double kvn) {
          auto t = strategy_tolerances(c, o, i, R[r].s, R[r].rprev, kvn, R[r].b_norm);
          track(R[r], t, kvn);
          return t;
        };
        items.push_back(it);
        owners.push_back(r);
      }
    }
    if (items.empty()) break;
    dielectric_batch(c, items, o.cg_maxit, o.precision, adjoint);
    for (int r : owners) {
      Rhs& q = R[r];
      if (q.phase == kResidual) {
        if (kerker) {
          axpy(c, q.b, q.wv, -1.0, nullptr, q.r0);
          apply_kerker(c, q.r0, q.r0, o.kerker_alpha);
        } else {
          axpy(c, q.bb, q.wv, -1.0, nullptr, q.r0);
        }
        start_cycle(q);
      } else {
        arnoldi(q);
      }
    }
  }
  IKR_CUDA(cudaStreamSynchronize(strm));
  const double ms = now_ms() - t0;
  for (int r = 0; r < nrhs && reps; ++r) {
    Rhs& q = R[r];
    ikr_report* rep = reps + r;
    rep->status = q.status;
    rep->outer_iters = q.steps;
    rep->restarts = q.restarts;
    rep->e_applies = q.rs.e_applies;
    rep->e_applies_fp32 = q.rs.e_applies_fp32;
    rep->n_ham = q.rs.n_ham;
    rep->n_ham_fp64 = q.rs.n_ham_fp64;
    rep->cg_max_iters = q.rs.cg_max_iters;
    rep->cg_noconv = q.rs.cg_noconv;
    rep->est_residual = q.est;
    rep->sigma = q.s;
    rep->b_norm = q.b_norm;
    rep->kv_norm = q.rs.kv_norm;
    rep->min_cg_tol = q.min_tol;
    rep->max_cg_tol = q.max_tol;
    rep->first_min_cg_tol = q.first_tol;
    rep->first_kv_norm = q.first_kvn;
    rep->ms = ms;
    rep->history_len = 0;
    if (rep->history && rep->history_cap > 0) {
      const int nh = std::min((int)q.hist.size(), rep->history_cap);
      std::copy(q.hist.begin(), q.hist.begin() + nh, rep->history);
      rep->history_len = nh;
    }
  }
  for (auto& q : R)
    if (q.status != IKR_OK) throw Error(q.status, q.status == IKR_ERR_TIMEOUT ? "time limit reached"
                                                                              : "GMRES did not converge");
}

}  // namespace ikr
