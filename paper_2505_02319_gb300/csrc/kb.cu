// Kleinman-Bylander nonlocal part of H_k (the nonlocal term of the GTH
// pseudopotentials of Sec. 4, here with Gaussian projectors):
//   V_nl = sum_j D_j |beta_j><beta_j|,
// an s and three p projectors of unit norm on every centre R,
//   beta_s(r)   = (pi s^2)^{-3/4} exp(-|r|^2 / (2 s^2)),
//   beta_p,a(r) = sqrt(2)/s (pi s^2)^{-3/4} r_a exp(-|r|^2 / (2 s^2)),
// whose Bloch sums have the plane-wave coefficients
//   <e_q | beta> = e^{-i q.R} betahat(q) / sqrt(Omega),  q = k + G,
//   betahat_s(q)   = (4 pi s^2)^{3/4} exp(-s^2 q^2 / 2),
//   betahat_p,a(q) = -i s^2 q_a sqrt(2)/s (pi s^2)^{-3/4} (2 pi s^2)^{3/2} exp(-s^2 q^2 / 2).
// The projector blocks B_k (Nb_k x nproj) are built once on the GPU.  An
// application out += B_k diag(D) B_k^H in treats the projectors of every
// k-point as a vector set, exactly like the occupied orbitals of the
// Q-projection: C = B_k^H in and out += B_k C run on the library's own
// projection kernels (FP64 and double-float on the CUDA cores; FP32 on the
// CUDA cores or, with ikr_set_tensor_cores, as tcgen05 MMAs on the exact
// three-piece bf16 split), all k-points in one launch each; between them a scaling kernel
// applies diag(D) and folds <in, V_nl in> = sum_j D_j |(B^H in)_j|^2 into the
// first <p, Ap> partial of a CG iteration.
#include <cmath>

#include "solver.hpp"

namespace ikr {

namespace {

// B_k for one k-point: projector j = 4 a + ch of centre a (ch: s, p_x, p_y, p_z)
__global__ void k_kb_build(const int* __restrict__ miller, int nb, int ld, double k0, double k1, double k2,
                           const double* __restrict__ recip, const double* __restrict__ centres, int nproj,
                           double ss, double sp, double omega, double2* __restrict__ B, float2* __restrict__ B32) {
  const size_t n = (size_t)nproj * ld;
  const double PI = 3.14159265358979323846;
  const double cs = pow(4.0 * PI * ss * ss, 0.75);
  const double cp = sqrt(2.0) / sp * pow(PI * sp * sp, -0.75) * pow(2.0 * PI * sp * sp, 1.5);
  const double inv_sqrt_omega = 1.0 / sqrt(omega);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ld), g = (int)(e - (size_t)j * ld);
    double2 v = make_double2(0.0, 0.0);
    if (g < nb) {
      const double m0 = miller[3 * g] + k0, m1 = miller[3 * g + 1] + k1, m2 = miller[3 * g + 2] + k2;
      double q[3];
      for (int i = 0; i < 3; ++i) q[i] = recip[3 * i] * m0 + recip[3 * i + 1] * m1 + recip[3 * i + 2] * m2;
      const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
      const int a = j / 4, ch = j - 4 * a;
      const double* R = centres + 3 * a;
      double sn, cn;
      sincos(-(q[0] * R[0] + q[1] * R[1] + q[2] * R[2]), &sn, &cn);   // e^{-i q.R}
      if (ch == 0) {
        const double f = cs * exp(-0.5 * ss * ss * q2) * inv_sqrt_omega;
        v = make_double2(f * cn, f * sn);
      } else {
        // -i f (cn + i sn) = f sn - i f cn
        const double f = sp * sp * cp * q[ch - 1] * exp(-0.5 * sp * sp * q2) * inv_sqrt_omega;
        v = make_double2(f * sn, -f * cn);
      }
    }
    B[e] = v;
    B32[e] = make_float2((float)v.x, (float)v.y);
  }
}

// C_js <- D_j C_js for every system s (coefficients [s][nproj]); with pap,
// also pap[s * nparts] += sum_j D_j |C_js|^2 (before the scaling) for the
// active systems; one warp per system
__global__ void k_kb_scale(double2* __restrict__ Cm, int nproj, int nsys, const double* __restrict__ D,
                           const int* __restrict__ active, double* __restrict__ pap, int nparts) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= nsys) return;
  if (active && !active[s]) return;
  double2* col = Cm + (size_t)s * nproj;
  double acc = 0.0;
  for (int j = lane; j < nproj; j += 32) {
    const double2 v = col[j];
    const double d = D[j];
    acc += d * (v.x * v.x + v.y * v.y);
    col[j] = make_double2(d * v.x, d * v.y);
  }
  acc = warp_sum(acc);
  if (pap && lane == 0) pap[(size_t)s * nparts] += acc;
}

}  // namespace

void set_nonlocal(ikr_ctx* c, int ncentres, const double* centres, const double* sigma, const double* D) {
  IKR_REQUIRE(ncentres >= 0, IKR_ERR_ARG, "ncentres must be >= 0");
  c->nproj = 0;
  if (ncentres == 0) return;
  IKR_REQUIRE(centres && sigma && D, IKR_ERR_ARG, "NULL argument");
  IKR_REQUIRE(sigma[0] > 0.0 && sigma[1] > 0.0, IKR_ERR_ARG, "projector widths must be positive");
  const int nproj = 4 * ncentres, nk = (int)c->k.size();
  const size_t per_k = (size_t)nproj * c->ld;
  c->d_kb.reserve(per_k * nk);
  c->d_kb32.reserve(per_k * nk);
  DBuf<double> dcen, drec;
  dcen.reserve(3 * (size_t)ncentres);
  drec.reserve(9);
  IKR_CUDA(cudaMemcpyAsync(dcen.p, centres, sizeof(double) * 3 * ncentres, cudaMemcpyHostToDevice, c->stream));
  IKR_CUDA(cudaMemcpyAsync(drec.p, c->recip, sizeof(double) * 9, cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < nk; ++k) {
    const KPoint& K = c->k[k];
    DBuf<int> dm;
    dm.reserve(K.miller.size());
    IKR_CUDA(cudaMemcpyAsync(dm.p, K.miller.data(), sizeof(int) * K.miller.size(), cudaMemcpyHostToDevice,
                             c->stream));
    const size_t n = per_k;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    k_kb_build<<<blocks, 256, 0, c->stream>>>(dm.p, K.nb, c->ld, K.kfrac[0], K.kfrac[1], K.kfrac[2], drec.p, dcen.p,
                                             nproj, sigma[0], sigma[1], c->volume, c->d_kb.p + k * per_k,
                                             c->d_kb32.p + k * per_k);
    IKR_CUDA(cudaGetLastError());
    IKR_CUDA(cudaStreamSynchronize(c->stream));   // dm is released at the end of the iteration
  }
  std::vector<double> dd(nproj);
  for (int a = 0; a < ncentres; ++a)
    for (int ch = 0; ch < 4; ++ch) dd[4 * a + ch] = ch == 0 ? D[0] : D[1];
  std::vector<int> koff(nk), kcnt(nk, nproj);
  for (int k = 0; k < nk; ++k) koff[k] = k * nproj;      // projector j of k-point k is row k nproj + j
  c->d_kboff.reserve(nk);
  c->d_kbcnt.reserve(nk);
  IKR_CUDA(cudaMemcpyAsync(c->d_kboff.p, koff.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, c->stream));
  IKR_CUDA(cudaMemcpyAsync(c->d_kbcnt.p, kcnt.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, c->stream));
  c->d_kbD.reserve(nproj);
  IKR_CUDA(cudaMemcpyAsync(c->d_kbD.p, dd.data(), sizeof(double) * nproj, cudaMemcpyHostToDevice, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  c->nproj = nproj;
  c->kb_dmax = std::max(D[0], D[1]);
}

OrbSet kb_set(ikr_ctx* c) {
  OrbSet o;
  o.phi = c->d_kb.p;
  o.phi32 = c->d_kb32.p;
  o.off = c->d_kboff.p;
  o.cnt = c->d_kbcnt.p;
  o.maxcnt = c->nproj;
  return o;
}

template <typename R>
void apply_nonlocal(ikr_ctx* c, const SysList& L, const C_t<R>* in, int ld, C_t<R>* out, const int* active,
                    double* pap, int nparts) {
  if (c->nproj == 0 || L.n == 0) return;
  const OrbSet kb = kb_set(c);
  c->ws.kbc.reserve((size_t)L.n * c->nproj);
  double2* Cm = c->ws.kbc.p;
  proj_coef<R>(c, L, in, ld, active, Cm, &kb);
  {
    ProfScope ps(c, kKidProjApply, 1);
    k_kb_scale<<<(L.n * 32 + 255) / 256, 256, 0, c->stream>>>(Cm, c->nproj, L.n, c->d_kbD.p, active, pap, nparts);
    IKR_CUDA(cudaGetLastError());
    c->tc_coef32_of = nullptr;   // scaled in place: the FP32 copy of the coefficients is stale
  }
  proj_apply<R>(c, L, Cm, out, R(1), R(1), out, ld, nullptr, nullptr, active, &kb);
}
template void apply_nonlocal<double>(ikr_ctx*, const SysList&, const double2*, int, double2*, const int*, double*,
                                     int);
template void apply_nonlocal<float>(ikr_ctx*, const SysList&, const float2*, int, float2*, const int*, double*, int);

}  // namespace ikr
