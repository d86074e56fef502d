// Autotuner of the interchangeable kernel variants of a context.
//
// Several kernels of the H_k application and of the CG have variants that
// compute the same thing with different launch shapes and data layouts; which
// is fastest depends on the grid, the number of systems and the orbital-set
// sizes.  autotune() times them on the context's own systems and keeps the
// fastest:
//   - the FP32 CG iteration (H_k application, projections, vector update) for
//     every combination of the FP32 plane kernel (full-plane k_plane_r, or the
//     compact k_plane_rc bounded to 4 or 5 blocks per SM) and the FP32
//     projection products (CUDA cores with the fused cluster update, or tcgen05
//     tensor cores with the unfused update): a few iterations of the batched
//     CG over all occupied systems, from a fixed right-hand side, projecting on
//     the vector set of the context's solves (Phi_k, or [Phi_k Psi_k] in the
//     Schur-complement form);
//   - with the CUDA cores, the cluster size of the fused update (16, 12, 10 or 8
//     CTAs per k-point: how many SMs work against how much each CTA holds);
//   - the FP64-accurate (double-float) H_k application for the padded and the
//     swizzled plane kernel, where the grid has both (48 x 48 planes).
// Each candidate runs once untimed (allocations, attributes) and then twice
// timed by CUDA events on the context's stream; the smaller time counts.  The
// variants agree to FP32 (respectively double-float) rounding, so the choice
// changes results only at that level.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "solver.hpp"

namespace ikr {

namespace {

template <typename F>
double best_ms(cudaStream_t st, F&& run) {
  run();                                          // untimed: allocations, attributes
  IKR_CUDA(cudaStreamSynchronize(st));
  cudaEvent_t e0, e1;
  IKR_CUDA(cudaEventCreate(&e0));
  IKR_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  for (int rep = 0; rep < 2; ++rep) {
    IKR_CUDA(cudaEventRecord(e0, st));
    run();
    IKR_CUDA(cudaEventRecord(e1, st));
    IKR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    IKR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, (double)ms);
  }
  IKR_CUDA(cudaEventDestroy(e0));
  IKR_CUDA(cudaEventDestroy(e1));
  return best;
}

}  // namespace

void autotune(ikr_ctx* c, double* out) {
  IKR_REQUIRE(c->have_gs, IKR_ERR_STATE, "the ground state is not set");
  const SysList& L = c->occ;
  const int n = L.n;
  for (int i = 0; i < 16; ++i) out[i] = -1.0;
  if (n == 0) return;
  ensure_workspace(c, n);
  Workspace& w = c->ws;
  const cudaStream_t st = c->stream;
  // a fixed right-hand side (every float 0x3c3c3c3c = 0.0115); the work does not depend on it
  IKR_CUDA(cudaMemsetAsync(w.B32.p, 0x3c, sizeof(float2) * (size_t)n * c->ld, st));
  std::vector<double> shift(n), kappa(n), tol(n, 0.0);     // tolerance 0: every iteration runs
  for (int s = 0; s < n; ++s) {
    shift[s] = c->k[L.k[s]].eps[L.band[s]];
    kappa[s] = c->h_kappa_occ[s];
  }
  constexpr int kIters = 4;
  const OrbSet set = c->schur ? schur_set(c) : occ_set(c);
  const int old_rc = c->plane_rc, old_force = c->cgf_force;
  const bool old_tc = c->tc_proj, old_sw = c->plane_sw;
  const int rcs[3] = {0, 4, 5};
  double best = 1e300;
  int best_rc = old_rc;
  bool best_tc = old_tc;
  try {
    for (int tc = 0; tc < 2; ++tc)
      for (int r = 0; r < 3; ++r) {
        c->plane_rc = rcs[r];
        c->tc_proj = tc != 0;
        const double ms = best_ms(st, [&] { cg_solve<float>(c, L, w.B32.p, w.X32.p, shift, kappa, tol, kIters, &set); });
        out[3 * tc + r] = ms / kIters;
        if (ms < best) {
          best = ms;
          best_rc = rcs[r];
          best_tc = tc != 0;
        }
      }
    c->plane_rc = best_rc;
    c->tc_proj = best_tc;
    out[6] = best_rc;
    out[7] = best_tc ? 1.0 : 0.0;
    // the cluster size of the fused CG update
    out[11] = 0.0;
    if (!best_tc) {
      const int sizes[4] = {16, 12, 10, 8};
      double bcs = 1e300;
      int best_cs = 0;
      for (int i = 0; i < 4; ++i) {
        c->cgf_force = sizes[i];
        if (cg_fused_cluster(c, L, set.maxcnt) != sizes[i]) continue;
        const double ms = best_ms(st, [&] { cg_solve<float>(c, L, w.B32.p, w.X32.p, shift, kappa, tol, kIters, &set); });
        out[12 + i] = ms / kIters;
        if (ms < bcs) {
          bcs = ms;
          best_cs = sizes[i];
        }
      }
      c->cgf_force = best_cs;
      out[11] = best_cs;
    }
    // the double-float H_k application (z-passes in FP64, plane pass in double-float)
    if (c->N[0] == 48 && c->N[1] == 48) {
      const bool old_em = c->emulate_fp64;
      c->emulate_fp64 = true;
      IKR_CUDA(cudaMemsetAsync(w.P.p, 0x3c, sizeof(double2) * (size_t)n * c->ld, st));
      double t[2];
      for (int sw = 0; sw < 2; ++sw) {
        c->plane_sw = sw != 0;
        t[sw] = best_ms(st, [&] {
          launch_z_inverse<double>(c, L, w.P.p, c->ld, nullptr, w.b1.p);
          launch_plane<double>(c, L, w.b1.p, c->d_Vt.p, nullptr, nullptr, w.b4.p, nullptr);
          launch_z_forward<double>(c, L, w.b4.p, w.W.p, c->ld, nullptr, nullptr, false, nullptr);
        });
        out[8 + sw] = t[sw];
      }
      c->emulate_fp64 = old_em;
      c->plane_sw = t[1] <= t[0];
    }
    out[10] = c->plane_sw ? 1.0 : 0.0;
    if (c->tc_proj) tc_check(c);
  } catch (...) {
    c->plane_rc = old_rc;
    c->tc_proj = old_tc;
    c->plane_sw = old_sw;
    c->cgf_force = old_force;
    throw;
  }
}

}  // namespace ikr
