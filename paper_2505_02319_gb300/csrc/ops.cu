// Occupied-space projections, CG vector updates with deterministic per-system
// dot products, the Hartree-exchange kernel K^Hxc, the Kerker preconditioner
// and the FP64 Arnoldi kernels.
#include "ops.hpp"

namespace ikr {

// ------------------------------------------------------------ projections --
// For the systems s of k-point k (grouped: L.kstart[k] .. + L.kcount[k]):
//   coef[s][m] = <phi_m, y_s> = sum_G conj(Phi_k[m][G]) y_s[G]       (Phi^H Y)
// as a split-K product: every CTA owns a chunk of kKC plane waves of one
// k-point and all (m, s) pairs, with the chunk of Phi and Y staged in shared
// memory and a 2 x 2 register tile of outputs per thread; the per-chunk
// partial sums are then added in fixed order (deterministic).

// coef[s][m] = sum over the chunk partials, one warp per (s, m): lanes take
// chunks lane, lane + 32, ... and a fixed shuffle tree adds them.
__global__ void k_proj_reduce(const double2* __restrict__ part, int nchunks, int kc, int nsys, int noccmax,
                              const int* __restrict__ sys_k, const int* __restrict__ nocc_k,
                              const int* __restrict__ nb_k, const int* __restrict__ active,
                              double2* __restrict__ coef) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nsys * noccmax) return;
  const int s = warp / noccmax, m = warp - s * noccmax;
  if (active && !active[s]) return;
  const int k = sys_k[s];
  if (m >= nocc_k[k]) return;
  const int nch = min((nb_k[k] + kc - 1) / kc, nchunks);
  double ax = 0, ay = 0;
  for (int c = lane; c < nch; c += 32) {
    const double2 v = part[((size_t)c * nsys + s) * noccmax + m];
    ax += v.x;
    ay += v.y;
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  if (lane == 0) coef[warp] = make_double2(ax, ay);
}

// FP64 variants: one warp per system, lanes over m (Phi^H Y) or over G (Y - Phi C),
// chunks of 32 plane waves; on this part's FP64 pipe they run faster than the
// register-tiled FP32 kernels below.
constexpr int kPC = 32;

template <typename R>
__global__ void __launch_bounds__(256) k_proj_partial_w(const typename io<R>::cx* __restrict__ phi_all, int ld,
                                                        const int* __restrict__ phi_off,
                                                        const int* __restrict__ nocc_k,
                                                        const int* __restrict__ nb_k,
                                                        const int* __restrict__ kstart,
                                                        const int* __restrict__ kcount,
                                                        const typename io<R>::cx* __restrict__ Y, int ldy,
                                                        const int* __restrict__ active, int nsys,
                                                        int noccmax, double2* __restrict__ part) {
  using C = C_t<R>;
  const int k = blockIdx.y, chunk = blockIdx.x;
  const int ns = kcount[k];
  if (ns == 0) return;
  const int nocc = nocc_k[k], nb = nb_k[k];
  const int g0 = chunk * kPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ph = reinterpret_cast<C*>(smem_raw);           // [g][m], kPC x nocc
  C* ys = ph + kPC * nocc;                          // per warp kPC entries
  const typename io<R>::cx* phi = phi_all + (size_t)phi_off[k] * ld;
  for (int idx = threadIdx.x; idx < kPC * nocc; idx += blockDim.x) {
    const int m = idx / kPC, g = idx - m * kPC;
    ph[g * nocc + m] = (g0 + g < nb) ? to_c<C>(phi[(size_t)m * ld + g0 + g]) : mk<C>(0, 0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  C* yw = ys + warp * kPC;
  const int s0 = kstart[k];
  for (int sl = warp; sl < ns; sl += nw) {
    const int s = s0 + sl;
    if (active && !active[s]) continue;
    yw[lane] = (g0 + lane < nb) ? to_c<C>(Y[(size_t)s * ldy + g0 + lane]) : mk<C>(0, 0);
    __syncwarp();
    for (int m = lane; m < nocc; m += 32) {
      R ax = R(0), ay = R(0);
#pragma unroll 8
      for (int g = 0; g < kPC; ++g) {
        const C p = ph[g * nocc + m], y = yw[g];
        ax += p.x * y.x + p.y * y.y;
        ay += p.x * y.y - p.y * y.x;
      }
      part[((size_t)chunk * nsys + s) * noccmax + m] = make_double2(to_d(ax), to_d(ay));
    }
    __syncwarp();
  }
}

// out[s][G] = alpha * in[s][G] + beta * sum_m Phi_k[m][G] coef[s][m]
// optionally dpart[s][chunk] = sum_{G in chunk} Re(conj(dv[s][G]) out[s][G]).
template <typename R>
__global__ void __launch_bounds__(256) k_proj_apply_w(const typename io<R>::cx* __restrict__ phi_all, int ld,
                                                      const int* __restrict__ phi_off,
                                                      const int* __restrict__ nocc_k,
                                                      const int* __restrict__ nb_k,
                                                      const int* __restrict__ kstart,
                                                      const int* __restrict__ kcount,
                                                      const double2* __restrict__ coef, int noccmax,
                                                      const typename io<R>::cx* in, double alpha, double beta,
                                                      typename io<R>::cx* out, int ldy,
                                                      const typename io<R>::cx* __restrict__ dv,
                                                      double* __restrict__ dpart, int nparts,
                                                      const int* __restrict__ active) {
  using C = C_t<R>;
  const int k = blockIdx.y, chunk = blockIdx.x;
  const int ns = kcount[k];
  if (ns == 0) return;
  const int nocc = nocc_k[k], nb = nb_k[k];
  const int g0 = chunk * kPC;
  if (g0 >= nb) {
    // chunk beyond this k-point's basis: still define the dot partials
    if (dpart)
      for (int sl = threadIdx.x; sl < ns; sl += blockDim.x) dpart[(size_t)(kstart[k] + sl) * nparts + chunk] = 0.0;
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ph = reinterpret_cast<C*>(smem_raw);           // [m][g]
  C* cwall = ph + kPC * nocc;                       // per warp: the coefficients of its system
  const typename io<R>::cx* phi = phi_all + (size_t)phi_off[k] * ld;
  for (int idx = threadIdx.x; idx < kPC * nocc; idx += blockDim.x) {
    const int m = idx / kPC, g = idx - m * kPC;
    ph[m * kPC + g] = (g0 + g < nb) ? to_c<C>(phi[(size_t)m * ld + g0 + g]) : mk<C>(0, 0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  C* cw = cwall + warp * nocc;
  const int s0 = kstart[k];
  const R ra = to_r<R>(alpha), rb = to_r<R>(beta);
  for (int sl = warp; sl < ns; sl += nw) {
    const int s = s0 + sl;
    if (active && !active[s]) continue;
    const double2* cf = coef + (size_t)s * noccmax;
    // each coefficient is converted once, by one lane
    for (int m = lane; m < nocc; m += 32) {
      const double2 cd = cf[m];
      cw[m] = mk<C>(to_r<R>(cd.x), to_r<R>(cd.y));
    }
    __syncwarp();
    R ax = R(0), ay = R(0);
    for (int m = 0; m < nocc; ++m) {
      const C p = ph[m * kPC + lane];
      const C cc = cw[m];
      ax += p.x * cc.x - p.y * cc.y;
      ay += p.x * cc.y + p.y * cc.x;
    }
    __syncwarp();
    const int g = g0 + lane;
    double d = 0.0;
    if (g < nb) {
      const size_t o = (size_t)s * ldy + g;
      C v = mk<C>(rb * ax, rb * ay);
      if (alpha != 0.0) {
        const C x = to_c<C>(in[o]);
        v.x += ra * x.x;
        v.y += ra * x.y;
      }
      out[o] = from_c(v);
      if (dv) {
        const auto w = dv[o];
        d = (double)w.x * to_d(v.x) + (double)w.y * to_d(v.y);
      }
    }
    if (dpart) {
      d = warp_sum(d);
      if (lane == 0) dpart[(size_t)s * nparts + chunk] = d;
    }
  }
}

// ------------------------------------------------------- per-system sums --
// out[s] = sum_{c < nparts} part[s][c] in fixed order.
__global__ void k_sys_reduce(const double* __restrict__ part, int nparts, int nsys,
                             const int* __restrict__ active, double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  if (active && !active[s]) return;
  double a = 0.0;
  for (int c = 0; c < nparts; ++c) a += part[(size_t)s * nparts + c];
  out[s] = a;
}

// ------------------------------------------------------------- CG kernels --
// Per-system scalars live in sys[field * nsys + s].

constexpr int kEC = 256;  // element chunk of the CG vector kernels

// Z = M^-1 R with M^-1 = 1/(kappa_s + |k+G|^2/2); dpart = <R, Z> partials are
// not formed here (Z is projected afterwards).  Mode 0: initialisation
// (X = 0, R = B).  Mode 1: X += alpha P, R -= alpha W, and ||R||^2 partials.
template <typename R>
__global__ void __launch_bounds__(kEC) k_cg_xr(int mode, C_t<R>* __restrict__ X, C_t<R>* __restrict__ Rv,
                                               const C_t<R>* __restrict__ Pv, const C_t<R>* __restrict__ W,
                                               const C_t<R>* __restrict__ Bv, C_t<R>* __restrict__ Z,
                                               int ld, const int* __restrict__ sys_k,
                                               const int* __restrict__ nb_k, const R* __restrict__ kin_all,
                                               const double* __restrict__ sys, int nsys,
                                               const int* __restrict__ active,
                                               double* __restrict__ dpart, int nparts) {
  using C = C_t<R>;
  const int s = blockIdx.y, chunk = blockIdx.x;
  if (active && !active[s]) return;
  __shared__ double sh[kEC / 32];
  const int k = sys_k[s], nb = nb_k[k];
  const int g = chunk * kEC + threadIdx.x;
  const R kappa = (R)sys[kSysKappa * nsys + s];
  double rr = 0.0;
  if (g < nb) {
    const size_t o = (size_t)s * ld + g;
    C r;
    if (mode == 0) {
      X[o] = mk<C>(0, 0);
      r = Bv[o];
    } else {
      const R a = (R)sys[kSysAlpha * nsys + s];
      const C p = Pv[o], w = W[o];
      C x = X[o];
      x.x += a * p.x;
      x.y += a * p.y;
      X[o] = x;
      r = Rv[o];
      r.x -= a * w.x;
      r.y -= a * w.y;
    }
    Rv[o] = r;
    const R mi = R(1) / (kappa + kin_all[(size_t)k * ld + g]);
    Z[o] = mk<C>(r.x * mi, r.y * mi);
    if constexpr (sizeof(R) == 8) rr = (double)r.x * r.x + (double)r.y * r.y;
    else rr = (double)fmaf(r.x, r.x, r.y * r.y);
  }
  if (mode == 1 && dpart) {
    if constexpr (sizeof(R) == 4) {
      // FP32 within the warp, FP64 across the warps (FP64 arithmetic is slow here)
      const float wsum = warp_sum((float)rr);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)wsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEC / 32; ++w) t += sh[w];
        dpart[(size_t)s * nparts + chunk] = t;
      }
    } else {
      rr = block_sum(rr, sh);
      if (threadIdx.x == 0) dpart[(size_t)s * nparts + chunk] = rr;
    }
  }
}

// P = Z + beta P (mode 1) or P = Z (mode 0)
template <typename R>
__global__ void __launch_bounds__(kEC) k_cg_p(int mode, C_t<R>* __restrict__ Pv, const C_t<R>* __restrict__ Z,
                                              int ld, const int* __restrict__ sys_k,
                                              const int* __restrict__ nb_k, const double* __restrict__ sys,
                                              int nsys, const int* __restrict__ active) {
  using C = C_t<R>;
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int nb = nb_k[sys_k[s]];
  const int g = blockIdx.x * kEC + threadIdx.x;
  if (g >= nb) return;
  const size_t o = (size_t)s * ld + g;
  const C z = Z[o];
  if (mode == 0) {
    Pv[o] = z;
  } else {
    const R b = (R)sys[kSysBeta * nsys + s];
    const C p = Pv[o];
    Pv[o] = mk<C>(z.x + b * p.x, z.y + b * p.y);
  }
}

// Scalar steps of the CG recurrences, one warp per system.  The warp first
// sums its system's nparts partial dot products (lane c takes c, c + 32, ...,
// then a fixed shuffle tree: the same order on every run); lane 0 then runs
// the stage.
//   stage 0 (init):  rz = <r, z>;  iters = 0;  status = 0
//   stage 1 (alpha): alpha = rz / <p, Ap>   (non-positive or non-finite -> numeric stop);
//                    resets the active counter
//   stage 2 (check): iters += 1; stop when ||r||^2 <= tol^2 or iters >= maxit;
//                    counts the systems that stay active and, given a list,
//                    writes their indices to it (compacted, in arrival order)
//   stage 3 (beta):  beta = rz_new / rz; rz = rz_new
__global__ void k_cg_scalars(int stage, double* __restrict__ sys, const double* __restrict__ part, int nparts,
                             int nsys, int maxit, int* __restrict__ active, int* __restrict__ counter,
                             int* __restrict__ list) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (stage == 1 && s == 0 && lane == 0 && counter) *counter = 0;
  if (s >= nsys || !active[s]) return;   // uniform over the warp
  double val = 0.0;
  for (int c = lane; c < nparts; c += 32) val += part[(size_t)s * nparts + c];
  val = warp_sum(val);
  if (lane != 0) return;
  double* f = sys;
  if (stage == 0) {
    f[kSysRz * nsys + s] = val;
    f[kSysIters * nsys + s] = 0;
    f[kSysStatus * nsys + s] = 0;
  } else if (stage == 1) {
    const double pap = val;
    f[kSysPap * nsys + s] = pap;
    const double a = f[kSysRz * nsys + s] / pap;
    if (!(pap > 0.0) || !isfinite(a)) {
      f[kSysStatus * nsys + s] = 2;
      f[kSysAlpha * nsys + s] = 0.0;
      active[s] = 0;
      return;
    }
    f[kSysAlpha * nsys + s] = a;
  } else if (stage == 2) {
    const double rr = val;
    f[kSysRr * nsys + s] = rr;
    const double it = f[kSysIters * nsys + s] + 1;
    f[kSysIters * nsys + s] = it;
    if (!isfinite(rr)) {
      f[kSysStatus * nsys + s] = 2;
      active[s] = 0;
    } else if (rr <= f[kSysTol2 * nsys + s]) {
      f[kSysStatus * nsys + s] = 1;
      active[s] = 0;
    } else if (it >= maxit) {
      f[kSysStatus * nsys + s] = 3;
      active[s] = 0;
    } else if (counter) {
      const int slot = atomicAdd(counter, 1);
      if (list) list[slot] = s;   // any order: each system's work is independent of its slot
    }
  } else {
    const double rz = val;
    const double b = rz / f[kSysRz * nsys + s];
    f[kSysBeta * nsys + s] = isfinite(b) ? b : 0.0;
    f[kSysRz * nsys + s] = rz;
  }
}

__global__ void k_count_active(const int* __restrict__ active, int n, int* __restrict__ out) {
  __shared__ int sh[32];
  int c = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c += active[i] ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

// ----------------------------------------------------------- chi0 pieces --
// Per system s = (k, n) of the occupied list: deps_s = Re M[s][n] and, for
// metals, the dphi^P coefficients coefP[s][m] = c_nm M[s][m] (m != n),
// c_nm = f_n/(f_n^2+f_m^2) (f_n-f_m)/(eps_n-eps_m), f' limit for |de| < 1e-10.
__global__ void k_chi0_sys(const double2* __restrict__ M, int noccmax, const int* __restrict__ sys_k,
                           const int* __restrict__ band, const int* __restrict__ nocc_k,
                           const int* __restrict__ kstart_occ, const double* __restrict__ eps_occ,
                           const double* __restrict__ f_occ, const double* __restrict__ fp_occ,
                           int nsys, int metal, double* __restrict__ deps,
                           double2* __restrict__ coefP) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsys * noccmax) return;
  const int s = idx / noccmax, m = idx - s * noccmax;
  const int k = sys_k[s], n = band[s];
  const int nocc = nocc_k[k];
  const double2 v = M[idx];
  if (m == n) deps[s] = v.x;
  double2 out = make_double2(0.0, 0.0);
  if (metal && m < nocc && m != n) {
    const int on = kstart_occ[k] + n, om = kstart_occ[k] + m;
    const double fn = f_occ[on], fm = f_occ[om];
    const double den = fn * fn + fm * fm;
    if (den > 0.0) {
      const double de = eps_occ[on] - eps_occ[om];
      const double D = (fabs(de) < 1e-10) ? 0.5 * (fp_occ[on] + fp_occ[om]) : (fn - fm) / de;
      const double c = fn / den * D;
      out = make_double2(c * v.x, c * v.y);
    }
  }
  coefP[idx] = out;
}

// One block: deps_F = sum w f' deps / sum w f' (0 if the denominator is 0),
// coef_a[s] = 2 w_k f_s, coef_b[s] = w_k f'_s (deps_s - deps_F).
__global__ void k_occupation_response(const double* __restrict__ deps, const double* __restrict__ w_s,
                                      const double* __restrict__ f_s, const double* __restrict__ fp_s,
                                      int nsys, double* __restrict__ coef_a, double* __restrict__ coef_b,
                                      double* __restrict__ deF_out) {
  __shared__ double sh[32];
  double num = 0.0, den = 0.0;
  // fixed-order strided partial sums
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    num += w_s[s] * fp_s[s] * deps[s];
    den += w_s[s] * fp_s[s];
  }
  num = block_sum(num, sh);
  __syncthreads();
  den = block_sum(den, sh);
  __shared__ double deF;
  if (threadIdx.x == 0) {
    deF = (den != 0.0) ? num / den : 0.0;
    if (deF_out) *deF_out = deF;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    coef_a[s] = 2.0 * w_s[s] * f_s[s];
    coef_b[s] = w_s[s] * fp_s[s] * (deps[s] - deF);
  }
}

// ------------------------------------------------------- grid operations --

__global__ void k_real_to_complex(const double* __restrict__ v, size_t n, double2* __restrict__ c) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c[i] = make_double2(v[i], 0.0);
}

__global__ void k_scale_complex(double2* __restrict__ c, const double* __restrict__ f, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = c[i];
    c[i] = make_double2(v.x * f[i], v.y * f[i]);
  }
}

// Kerker factor D = |G|^2/(|G|^2 + alpha^2) with D(0) = 1, divided by Ng.
__global__ void k_kerker_scale(double2* __restrict__ c, const double* __restrict__ G2, double alpha2,
                               double inv_ng, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double g2 = G2[i];
    const double d = (i == 0) ? 1.0 : g2 / (g2 + alpha2);
    const double2 v = c[i];
    c[i] = make_double2(v.x * d * inv_ng, v.y * d * inv_ng);
  }
}

// out = Re(c) + kxc * v, with per-block partial ||out||^2
__global__ void k_finish_K(const double2* __restrict__ c, const double* __restrict__ kxc,
                           const double* __restrict__ v, size_t n, double* __restrict__ out,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double o = c[i].x + kxc[i] * v[i];
    out[i] = o;
    a += o * o;
  }
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_complex_real_part(const double2* __restrict__ c, size_t n, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = c[i].x;
}

// partial sums of x*y
__global__ void k_dot_part(const double* __restrict__ x, const double* __restrict__ y, size_t n,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// single block: out[0] = sum part, out[1] = sqrt(out[0]), out[2] = 1/out[1] (0 if 0)
__global__ void k_finish_norm(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = sqrt(a);
    out[2] = a > 0.0 ? 1.0 / sqrt(a) : 0.0;
  }
}

// out = x + a * y with a = sa * (*da) (da may be null)
__global__ void k_axpy(const double* __restrict__ x, const double* __restrict__ y, double sa,
                       const double* __restrict__ da, size_t n, double* __restrict__ out) {
  const double a = sa * (da ? *da : 1.0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = x[i] + a * y[i];
}

// ---------------------------------------------------------------- Arnoldi --
// h_part[j][block] = sum_{i in block's range} V[j][i] w[i], j < nv
constexpr int kArnBlocks = 304;   // 2 per SM

__global__ void __launch_bounds__(256) k_multidot(const double* __restrict__ V, int nv, size_t n,
                                                  const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t i0 = blockIdx.x * per, i1 = (i0 + per < n) ? i0 + per : n;
  for (int j = 0; j < nv; ++j) {
    double a = 0.0;
    for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) a += V[(size_t)j * n + i] * w[i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = a;
    __syncthreads();
  }
}

// h[j] (+)= sum_b part[j][b], j < nv  (one block per j)
__global__ void k_multidot_finish(const double* __restrict__ part, int nb, int nv, int accumulate,
                                  double* __restrict__ h) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[(size_t)j * nb + b];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) h[j] = accumulate ? h[j] + a : a;
}

// w -= sum_j V[j] * h[j]
__global__ void k_sub_combination(const double* __restrict__ V, int nv, size_t n,
                                  const double* __restrict__ h, double* __restrict__ w) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double a = w[i];
    for (int j = 0; j < nv; ++j) a -= V[(size_t)j * n + i] * h[j];
    w[i] = a;
  }
}

// x = x0 + sum_j V[j] y[j]
__global__ void k_add_combination(const double* __restrict__ V, int nv, size_t n,
                                  const double* __restrict__ y, const double* __restrict__ x0,
                                  double* __restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double a = x0 ? x0[i] : 0.0;
    for (int j = 0; j < nv; ++j) a += V[(size_t)j * n + i] * y[j];
    x[i] = a;
  }
}

// v_out = w * (*dinv)
__global__ void k_scale_by(const double* __restrict__ w, const double* __restrict__ dinv, size_t n,
                           double* __restrict__ out) {
  const double a = *dinv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = w[i] * a;
}

// ------------------------------------------------------------------ misc --

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, size_t n, B* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    out[i].x = in[i].x;
    out[i].y = in[i].y;
  }
}

// max over the grid of rows norms: out = max_r acc[r] (single block, fixed order)
__global__ void k_max(const double* __restrict__ v, size_t n, double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
    *out = t;
  }
}

// kxc = -(1/3)(3/pi)^{1/3} rho^{-2/3} where rho >= 1e-10, else 0 (LDA exchange)
__global__ void k_exchange_kernel(const double* __restrict__ rho, size_t n, double* __restrict__ kxc) {
  const double c = -(1.0 / 3.0) * cbrt(3.0 / 3.14159265358979323846);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[i];
    kxc[i] = (r >= 1e-10) ? c / cbrt(r * r) : 0.0;
  }
}

// ========================================================== host wrappers ==

static inline int grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

template <typename R> const C_t<R>* phi_ptr(ikr_ctx* c);
template <> const double2* phi_ptr<double>(ikr_ctx* c) { return c->d_phi_all.p; }
template <> const float2* phi_ptr<float>(ikr_ctx* c) { return c->d_phi_all32.p; }

static void set_smem_attr(const void* f, size_t bytes) {
  IKR_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

int proj_chunks(ikr_ctx* c, int fp_bytes) {
  const int g = fp_bytes == 4 ? proj_chunks32() : kPC;
  return (c->ld + g - 1) / g;
}
int proj_chunks(ikr_ctx* c) { return std::max(proj_chunks(c, 4), proj_chunks(c, 8)); }
int cg_chunks(ikr_ctx* c) { return (c->ld + kEC - 1) / kEC; }

OrbSet occ_set(ikr_ctx* c) {
  OrbSet o;
  o.phi = c->d_phi_all.p;
  o.phi32 = c->d_phi_all32.p;
  o.off = c->d_phi_off.p;
  o.cnt = c->d_nocc.p;
  o.maxcnt = c->noccmax;
  return o;
}
OrbSet schur_set(ikr_ctx* c) {
  OrbSet o;
  o.phi = c->d_rset.p;
  o.phi32 = c->d_rset32.p;
  o.off = c->d_roff.p;
  o.cnt = c->d_rcnt.p;
  o.maxcnt = c->rmax;
  return o;
}
OrbSet extra_set(ikr_ctx* c) {
  OrbSet o;
  o.phi = c->d_rset.p;
  o.phi32 = c->d_rset32.p;
  o.off = c->d_xoff.p;
  o.cnt = c->d_xcnt.p;
  o.maxcnt = c->xmax;
  return o;
}

template <typename R>
void proj_coef(ikr_ctx* c, const SysList& L, const C_t<R>* Y, int ldy, const int* active, double2* coef,
               const OrbSet* set) {
  ProfScope ps(c, kKidProjCoef, 2, L.n, (int)sizeof(R));
  const OrbSet os = set ? *set : occ_set(c);
  c->tc_coef32_of = nullptr;   // a tensor-core product below makes the FP32 copy current again
  if (sizeof(R) == 8) {
    const int nch = (c->ld + kPC - 1) / kPC;
    const int nm = os.maxcnt;
    c->ws.cpart.reserve((size_t)nch * L.n * nm * 2);
    double2* part = reinterpret_cast<double2*>(c->ws.cpart.p);
    const size_t smem = sizeof(double2) * (kPC * nm + 8 * kPC);
    dim3 grid(nch, (unsigned)c->k.size());
    const double2* Yd = reinterpret_cast<const double2*>(Y);
    if (c->emulate_fp64) {   // FP64-accurate products of the mixed path on the FP32 units
      set_smem_attr((const void*)k_proj_partial_w<dfloat>, smem);
      k_proj_partial_w<dfloat><<<grid, 256, smem, c->stream>>>(os.phi, c->ld, os.off, os.cnt,
                                                                c->d_nb.p, L.d_kstart.p, L.d_kcount.p, Yd, ldy,
                                                                active, L.n, nm, part);
    } else {
      set_smem_attr((const void*)k_proj_partial_w<double>, smem);
      k_proj_partial_w<double><<<grid, 256, smem, c->stream>>>(os.phi, c->ld, os.off, os.cnt,
                                                                c->d_nb.p, L.d_kstart.p, L.d_kcount.p, Yd, ldy,
                                                                active, L.n, nm, part);
    }
    IKR_CUDA(cudaGetLastError());
    const long long threads = 32LL * L.n * nm;
    k_proj_reduce<<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(part, nch, kPC, L.n, nm, L.d_k.p,
                                                                            os.cnt, c->d_nb.p, active, coef);
    IKR_CUDA(cudaGetLastError());
    return;
  }
  if constexpr (sizeof(R) == 4) proj_coef32(c, L, Y, ldy, active, coef, os);
}

template <typename R>
void proj_apply(ikr_ctx* c, const SysList& L, const double2* coef, const C_t<R>* in, R alpha, R beta,
                C_t<R>* out, int ldy, const C_t<R>* dv, double* dpart, const int* active, const OrbSet* set) {
  ProfScope ps(c, kKidProjApply, 1, L.n, (int)sizeof(R));
  const OrbSet os = set ? *set : occ_set(c);
  if (sizeof(R) == 8) {
    const int nch = proj_chunks(c, 8);
    const size_t smem = sizeof(double2) * ((kPC + 8) * os.maxcnt);
    dim3 grid(nch, (unsigned)c->k.size());
    const double2* ind = reinterpret_cast<const double2*>(in);
    double2* outd = reinterpret_cast<double2*>(out);
    const double2* dvd = reinterpret_cast<const double2*>(dv);
    if (c->emulate_fp64) {
      set_smem_attr((const void*)k_proj_apply_w<dfloat>, smem);
      k_proj_apply_w<dfloat><<<grid, 256, smem, c->stream>>>(os.phi, c->ld, os.off, os.cnt,
                                                              c->d_nb.p, L.d_kstart.p, L.d_kcount.p, coef, os.maxcnt,
                                                              ind, (double)alpha, (double)beta, outd, ldy, dvd, dpart,
                                                              nch, active);
    } else {
      set_smem_attr((const void*)k_proj_apply_w<double>, smem);
      k_proj_apply_w<double><<<grid, 256, smem, c->stream>>>(os.phi, c->ld, os.off, os.cnt,
                                                              c->d_nb.p, L.d_kstart.p, L.d_kcount.p, coef, os.maxcnt,
                                                              ind, (double)alpha, (double)beta, outd, ldy, dvd, dpart,
                                                              nch, active);
    }
    IKR_CUDA(cudaGetLastError());
    return;
  }
  if constexpr (sizeof(R) == 4) proj_apply32(c, L, coef, in, alpha, beta, out, ldy, dv, dpart, active, os);
}

void sys_reduce(ikr_ctx* c, const double* part, int nparts, int nsys, const int* active, double* out) {
  ProfScope ps(c, kKidScalar, 1);
  k_sys_reduce<<<(nsys + 127) / 128, 128, 0, c->stream>>>(part, nparts, nsys, active, out);
  IKR_CUDA(cudaGetLastError());
}

template <typename R> const R* kin_ptr(ikr_ctx* c);
template <> const double* kin_ptr<double>(ikr_ctx* c) { return c->d_kin_all.p; }
template <> const float* kin_ptr<float>(ikr_ctx* c) { return c->d_kin_all32.p; }

template <typename R>
void cg_xr(ikr_ctx* c, const SysList& L, int mode, CgVecs<R>& v, const double* sys, const int* active,
           double* dpart) {
  ProfScope ps(c, kKidCgVec, 1);
  const int nch = cg_chunks(c);
  dim3 grid(nch, L.n);
  k_cg_xr<R><<<grid, kEC, 0, c->stream>>>(mode, v.X, v.R, v.P, v.W, v.B, v.Z, c->ld, L.d_k.p, c->d_nb.p,
                                          kin_ptr<R>(c), sys, L.n, active, dpart, nch);
  IKR_CUDA(cudaGetLastError());
}

template <typename R>
void cg_p(ikr_ctx* c, const SysList& L, int mode, CgVecs<R>& v, const double* sys, const int* active) {
  ProfScope ps(c, kKidCgVec, 1);
  dim3 grid(cg_chunks(c), L.n);
  k_cg_p<R><<<grid, kEC, 0, c->stream>>>(mode, v.P, v.Z, c->ld, L.d_k.p, c->d_nb.p, sys, L.n, active);
  IKR_CUDA(cudaGetLastError());
}

void cg_scalars(ikr_ctx* c, int stage, double* sys, const double* part, int nparts, int nsys, int maxit,
                int* active, int* counter, int* list) {
  ProfScope ps(c, kKidScalar, 1);
  k_cg_scalars<<<(nsys + 3) / 4, 128, 0, c->stream>>>(stage, sys, part, nparts, nsys, maxit, active, counter, list);
  IKR_CUDA(cudaGetLastError());
}

void count_active(ikr_ctx* c, const int* active, int n, int* dout) {
  ProfScope ps(c, kKidScalar, 1);
  k_count_active<<<1, 1024, 0, c->stream>>>(active, n, dout);
  IKR_CUDA(cudaGetLastError());
}

void chi0_sys(ikr_ctx* c, const SysList& L, const double2* M, double* deps, double2* coefP) {
  ProfScope ps(c, kKidScalar, 1);
  const int tot = L.n * c->noccmax;
  k_chi0_sys<<<(tot + 255) / 256, 256, 0, c->stream>>>(
      M, c->noccmax, L.d_k.p, L.d_band.p, c->d_nocc.p, c->d_occ_kstart.p, c->d_eps_occ.p, c->d_f_occ.p,
      c->d_fp_occ.p, L.n, c->T > 0.0 ? 1 : 0, deps, coefP);
  IKR_CUDA(cudaGetLastError());
}

// a[s][j] = <psi_j, b_s> / (lambda_j - eps_s): the Psi_k component of the
// Schur-complement solution (lambda_j >= eps_{Nocc+1,k} > eps_s, checked when
// the eigenpairs were set).
__global__ void k_deflate_coef(double2* __restrict__ a, int xmax, int nsys, const int* __restrict__ sys_k,
                               const int* __restrict__ xcnt, const int* __restrict__ xoff,
                               const double* __restrict__ reps, const double* __restrict__ shift) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsys * xmax) return;
  const int s = idx / xmax, j = idx - s * xmax;
  const int k = sys_k[s];
  if (j >= xcnt[k]) return;
  const double inv = 1.0 / (reps[xoff[k] + j] - shift[s]);
  const double2 v = a[idx];
  a[idx] = make_double2(v.x * inv, v.y * inv);
}

void deflate_coef(ikr_ctx* c, const SysList& L, double2* a, const double* shift) {
  c->tc_coef32_of = nullptr;   // the coefficients change: their FP32 copy is stale
  ProfScope ps(c, kKidScalar, 1);
  const int tot = L.n * c->xmax;
  if (tot == 0) return;
  k_deflate_coef<<<(tot + 255) / 256, 256, 0, c->stream>>>(a, c->xmax, L.n, L.d_k.p, c->d_xcnt.p, c->d_xoff.p,
                                                           c->d_reps.p, shift);
  IKR_CUDA(cudaGetLastError());
}

void occupation_response(ikr_ctx* c, const double* deps, double* coef_a, double* coef_b, double* deF) {
  ProfScope ps(c, kKidScalar, 1);
  k_occupation_response<<<1, 1024, 0, c->stream>>>(deps, c->d_w_occ.p, c->d_f_occ.p, c->d_fp_occ.p,
                                                   c->occ.n, coef_a, coef_b, deF);
  IKR_CUDA(cudaGetLastError());
}

// K v = K^H v + K^xc v; d_norm receives {||Kv||^2, ||Kv||, 1/||Kv||}.
void apply_K(ikr_ctx* c, const double* v, double* Kv, double* d_norm) {
  ProfScope ps(c, kKidGridOps, 4);
  const size_t n = c->Ng;
  c->ws.cgrid.reserve(n);
  c->ws.gm_h.reserve(4096);
  double2* cg = c->ws.cgrid.p;
  const int nb = grid_for(n, 256);
  k_real_to_complex<<<nb, 256, 0, c->stream>>>(v, n, cg);
  full_fft(c, cg, false);
  k_scale_complex<<<nb, 256, 0, c->stream>>>(cg, c->d_coul.p, n);
  full_fft(c, cg, true);
  double* part = c->ws.gm_h.p + 2048;
  k_finish_K<<<nb, 256, 0, c->stream>>>(cg, c->d_kxc.p, v, n, Kv, part);
  k_finish_norm<<<1, 256, 0, c->stream>>>(part, nb, d_norm);
  IKR_CUDA(cudaGetLastError());
}

void apply_kerker(ikr_ctx* c, const double* v, double* Tv, double alpha) {
  ProfScope ps(c, kKidGridOps, 3);
  const size_t n = c->Ng;
  c->ws.cgrid.reserve(n);
  double2* cg = c->ws.cgrid.p;
  const int nb = grid_for(n, 256);
  k_real_to_complex<<<nb, 256, 0, c->stream>>>(v, n, cg);
  full_fft(c, cg, false);
  k_kerker_scale<<<nb, 256, 0, c->stream>>>(cg, c->d_G2.p, alpha * alpha, 1.0 / (double)n, n);
  full_fft(c, cg, true);
  k_complex_real_part<<<nb, 256, 0, c->stream>>>(cg, n, Tv);
  IKR_CUDA(cudaGetLastError());
}

void norm2(ikr_ctx* c, const double* x, double* d_out3) {
  ProfScope ps(c, kKidGridOps, 2);
  const size_t n = c->Ng;
  c->ws.gm_h.reserve(4096);
  double* part = c->ws.gm_h.p + 2048;
  const int nb = grid_for(n, 256);
  k_dot_part<<<nb, 256, 0, c->stream>>>(x, x, n, part);
  k_finish_norm<<<1, 256, 0, c->stream>>>(part, nb, d_out3);
  IKR_CUDA(cudaGetLastError());
}

void axpy(ikr_ctx* c, const double* x, const double* y, double sa, const double* da, double* out) {
  ProfScope ps(c, kKidGridOps, 1);
  k_axpy<<<grid_for(c->Ng, 256), 256, 0, c->stream>>>(x, y, sa, da, c->Ng, out);
  IKR_CUDA(cudaGetLastError());
}

void scale_by(ikr_ctx* c, const double* w, const double* dinv, double* out) {
  ProfScope ps(c, kKidGridOps, 1);
  k_scale_by<<<grid_for(c->Ng, 256), 256, 0, c->stream>>>(w, dinv, c->Ng, out);
  IKR_CUDA(cudaGetLastError());
}

// h[0..nv) (+)= V[0..nv)^T w  (deterministic two-stage reduction)
void multidot(ikr_ctx* c, const double* V, int nv, const double* w, double* h, int accumulate) {
  ProfScope ps(c, kKidGridOps, 2);
  c->ws.gm_h.reserve(4096 + (size_t)kArnBlocks * 64);
  double* part = c->ws.gm_h.p + 4096;
  k_multidot<<<kArnBlocks, 256, 0, c->stream>>>(V, nv, c->Ng, w, part);
  k_multidot_finish<<<nv, 256, 0, c->stream>>>(part, kArnBlocks, nv, accumulate, h);
  IKR_CUDA(cudaGetLastError());
}

void sub_combination(ikr_ctx* c, const double* V, int nv, const double* h, double* w) {
  ProfScope ps(c, kKidGridOps, 1);
  k_sub_combination<<<grid_for(c->Ng, 256), 256, 0, c->stream>>>(V, nv, c->Ng, h, w);
  IKR_CUDA(cudaGetLastError());
}

void add_combination(ikr_ctx* c, const double* V, int nv, const double* y, const double* x0, double* x) {
  ProfScope ps(c, kKidGridOps, 1);
  k_add_combination<<<grid_for(c->Ng, 256), 256, 0, c->stream>>>(V, nv, c->Ng, y, x0, x);
  IKR_CUDA(cudaGetLastError());
}

void exchange_kernel(ikr_ctx* c) {
  k_exchange_kernel<<<grid_for(c->Ng, 256), 256, 0, c->stream>>>(c->d_rho.p, c->Ng, c->d_kxc.p);
  IKR_CUDA(cudaGetLastError());
}

void grid_max(ikr_ctx* c, const double* v, size_t n, double* dout) {
  k_max<<<1, 1024, 0, c->stream>>>(v, n, dout);
  IKR_CUDA(cudaGetLastError());
}

void to_fp32(ikr_ctx* c, const double2* in, size_t n, float2* out) {
  ProfScope ps(c, kKidCgVec, 1);
  k_convert<double2, float2><<<grid_for(n, 256), 256, 0, c->stream>>>(in, n, out);
  IKR_CUDA(cudaGetLastError());
}

void to_fp64(ikr_ctx* c, const float2* in, size_t n, double2* out) {
  ProfScope ps(c, kKidCgVec, 1);
  k_convert<float2, double2><<<grid_for(n, 256), 256, 0, c->stream>>>(in, n, out);
  IKR_CUDA(cudaGetLastError());
}

#define IKR_INST(R)                                                                                \
  template void proj_coef<R>(ikr_ctx*, const SysList&, const C_t<R>*, int, const int*, double2*,  \
                             const OrbSet*);                                                       \
  template void proj_apply<R>(ikr_ctx*, const SysList&, const double2*, const C_t<R>*, R, R,      \
                              C_t<R>*, int, const C_t<R>*, double*, const int*, const OrbSet*);   \
  template void cg_xr<R>(ikr_ctx*, const SysList&, int, CgVecs<R>&, const double*, const int*,     \
                         double*);                                                                 \
  template void cg_p<R>(ikr_ctx*, const SysList&, int, CgVecs<R>&, const double*, const int*);
IKR_INST(double)
IKR_INST(float)
#undef IKR_INST

}  // namespace ikr
