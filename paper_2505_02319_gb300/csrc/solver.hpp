// Internal interfaces of the solver layer (solver.cu, mixed.cu).
#pragma once

#include <complex>
#include <functional>
#include <vector>

#include "ops.hpp"

namespace ikr {

// Kleinman-Bylander nonlocal part (kb.cu)
void set_nonlocal(ikr_ctx* c, int ncentres, const double* centres, const double* sigma, const double* D);
// out += B diag(D) B^H in for the systems of L (k-grouped); with pap, also
// pap[s * nparts] += <in_s, V_nl in_s> for the active systems
template <typename R>
void apply_nonlocal(ikr_ctx* c, const SysList& L, const C_t<R>* in, int ld, C_t<R>* out, const int* active,
                    double* pap, int nparts);

// ground-state eigensolver (eigen.cu)
struct EigenStats {
  int iters = 0;              // filter + Rayleigh-Ritz cycles
  double max_residual = 0.0;  // largest ||H x - theta x|| of the wanted bands
};
std::vector<EigenStats> compute_eigenpairs(ikr_ctx* c, int nbands, double tol, int maxit, int degree,
                                           std::vector<DBuf<double2>>& vecs, std::vector<double>& eps);
void herm_jacobi(int n, std::vector<std::complex<double>>& A, std::vector<double>& w,
                 std::vector<std::complex<double>>& V);

struct CgStats {
  std::vector<int> iters, status;   // status: 1 converged, 2 numeric, 3 iteration cap
  std::vector<int> checks;          // FP64 residual applications per system (mixed solves)
  std::vector<double> res;          // final recursive residual norms
  long long n_ham = 0, n_ham_fp64 = 0;
  int max_iters = 0, noconv = 0, numeric = 0;
  bool fp32 = false;
};

struct RunStats {
  long long n_ham = 0, n_ham_fp64 = 0;
  int e_applies = 0, e_applies_fp32 = 0;
  int cg_max_iters = 0, cg_noconv = 0, cg_numeric = 0;
  double kv_norm = 0.0, sigma = 0.0;
  double last_dEv = 0.0;            // ||v - Ev|| of the previous E application
  void add(const CgStats& s) {
    n_ham += s.n_ham;
    n_ham_fp64 += s.fp32 ? s.n_ham_fp64 : s.n_ham;
    cg_max_iters = std::max(cg_max_iters, s.max_iters);
    cg_noconv += s.noconv;
    cg_numeric += s.numeric;
    if (s.fp32) e_applies_fp32++;
  }
};

using TolFn = std::function<std::vector<double>(double)>;

void ensure_workspace(ikr_ctx* c, int n);
void ensure_pinned(ikr_ctx* c, int n);
template <typename R>
void hamiltonian(ikr_ctx* c, int k, const C_t<R>* psi, C_t<R>* hpsi, int ld, int nvec);
template <typename R>
CgStats cg_solve(ikr_ctx* c, const SysList& L, const C_t<R>* Bv, C_t<R>* Xv, const std::vector<double>& shift,
                 const std::vector<double>& kappa, const std::vector<double>& tol, int maxit,
                 const OrbSet* zset = nullptr);
// cg_solve, or its Schur-complement form when the context has it enabled (B is then overwritten)
template <typename R>
CgStats sternheimer_solve(ikr_ctx* c, const SysList& L, C_t<R>* Bv, C_t<R>* Xv, const std::vector<double>& shift,
                          const std::vector<double>& kappa, const std::vector<double>& tol, int maxit);
// schur: the FP32 solves take the Schur-complement form when the context has it
// enabled (only for occupied systems, whose shifts lie below the extra bands)
CgStats mixed_solve(ikr_ctx* c, const SysList& L, const double2* Bv, double2* Xv, const std::vector<double>& shift,
                    const std::vector<double>& kappa, const std::vector<double>& tol, int maxit,
                    bool schur = false);
void chi0_core(ikr_ctx* c, const double* u, const double* pot_scale, const std::vector<double>& tol,
               int maxit, int precision, double* drho, RunStats& rs, bool fp32 = false);
void dielectric_core(ikr_ctx* c, const double* v, double* Ev, const TolFn& tol_fn, int maxit, int precision,
                     RunStats& rs, double allowed = 0.0);
// smallest singular value of the m x n column-major matrix a (m >= n)
double sigma_min(std::vector<double> a, int m, int n);
std::vector<double> strategy_tolerances(ikr_ctx* c, const ikr_solve_opts& o, int i, double s, double rprev,
                                        double kv_norm, double b_norm);
void hamiltonian_noalloc(ikr_ctx* c, int k, const double2* psi, double2* hpsi, int nvec);
void dielectric_adjoint_core(ikr_ctx* c, const double* v, double* Ev, const TolFn& tol_fn, int maxit,
                             int precision, RunStats& rs, double allowed = 0.0);
void gmres_solve(ikr_ctx* c, const double* b, double* x, const ikr_solve_opts& o, ikr_report* rep,
                 bool adjoint = false);
// Algorithm 1 for nrhs right-hand sides in lockstep, the E applications of a
// round batched into one CG (batch.cu); reps: nrhs reports or NULL
void gmres_solve_batch(ikr_ctx* c, int nrhs, const double* b, double* x, const ikr_solve_opts& o,
                       ikr_report* reps, bool adjoint = false);

// times the interchangeable kernel variants on the context's systems and keeps the
// fastest (tune.cu); out: 16 doubles, see ikr_autotune
void autotune(ikr_ctx* c, double* out);

}  // namespace ikr
