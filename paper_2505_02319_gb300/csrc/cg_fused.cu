// Fused FP32 update of the projected Sternheimer CG (eq. discretised_sternheimer,
// preconditioned CG of the Sternheimer solves) after the H_k application of an
// iteration: alpha from <p, Ap>, x += alpha p, r -= alpha Ap, the stopping
// test on ||r||, z = Q M^-1 r with Q = 1 - Phi_k Phi_k^H, beta = <r, z>_new /
// <r, z>_old and p = z + beta p, for all systems of a k-point in one launch.
//
// One thread-block cluster per k-point; CTA r of the cluster owns the plane
// waves [r sl, (r + 1) sl) of every system of the k-point, keeps their z and
// the matching slice of Phi_k in shared memory, and exchanges only the
// cross-slice sums (||r||^2, the N_occ x n_sys coefficients Phi^H z, <r, z>)
// through distributed shared memory: each CTA writes its partial sums, the
// cluster barrier publishes them, and every CTA adds the partials of all ranks
// in rank order, so the sums (and the decisions taken on them) are identical
// in every CTA and on every run.  The coefficients are reduced distributed:
// rank q mod CS adds entry q over the ranks, then every CTA gathers the
// reduced entries.  Rank 0 writes the per-system scalars, the active flags
// and the compacted list of the systems that continue.
#include <cooperative_groups.h>

#include <cstdlib>

#include "ops.hpp"

namespace cg = cooperative_groups;

namespace ikr {

namespace {
constexpr int kFT = 512;   // threads per CTA (16 warps)
constexpr int kFW = kFT / 32;
constexpr int kFU = 8;     // slice elements per lane (slices of at most 256 plane waves)
}  // namespace

struct CgFusedArgs {
  float2* X;
  float2* Rv;
  float2* P;
  const float2* W;
  const float2* phi_all;
  const int* phi_off;
  const float* kin_all;
  const int* nb_k;
  const int* nocc_k;
  const int* kstart;
  const int* kcount;
  double* sys;
  int nsys, maxit;
  int* active;
  int* counter;
  int* list;
  const double* zpart;   // <p, Ap> partials [s][nzf] of the forward z-pass
  int nzf, ld, sl, lds, nsmax, noccmax;
};

// shared-memory layout (bytes), the same on host and device
struct CgFusedLayout {
  size_t zs, phs, cpart, cred, cfull, sd, si, total;
  __host__ __device__ CgFusedLayout(int nsmax, int noccmax, int lds) {
    zs = 0;
    phs = zs + sizeof(float2) * (size_t)nsmax * lds;
    cpart = phs + sizeof(float2) * (size_t)noccmax * lds;
    cred = cpart + sizeof(float2) * (size_t)noccmax * nsmax;
    cfull = cred + sizeof(float2) * (size_t)noccmax * nsmax;
    sd = cfull + sizeof(float2) * (size_t)noccmax * nsmax;   // 7 x nsmax doubles
    si = sd + sizeof(double) * 7 * (size_t)nsmax;             // 2 x nsmax ints
    total = si + sizeof(int) * 2 * (size_t)nsmax;
  }
};

__global__ void __launch_bounds__(kFT, 1) k_cg_fused(CgFusedArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), CS = (int)cluster.num_blocks();
  const int k = blockIdx.y;
  const int ns = a.kcount[k], s0 = a.kstart[k], nb = a.nb_k[k], nocc = a.nocc_k[k];
  const int g0 = rank * a.sl, ng = max(min(a.sl, nb - g0), 0);   // this CTA's plane waves
  const int lds = a.lds, nsm = a.nsmax, nsys = a.nsys;
  const CgFusedLayout L(a.nsmax, a.noccmax, lds);
  extern __shared__ float4 smem_f[];
  unsigned char* base = reinterpret_cast<unsigned char*>(smem_f);
  float2* zs = reinterpret_cast<float2*>(base + L.zs);
  float2* phs = reinterpret_cast<float2*>(base + L.phs);
  float2* cpart = reinterpret_cast<float2*>(base + L.cpart);
  float2* cred = reinterpret_cast<float2*>(base + L.cred);
  float2* cfull = reinterpret_cast<float2*>(base + L.cfull);
  double* alpha_s = reinterpret_cast<double*>(base + L.sd);
  double* rrp = alpha_s + nsm;
  double* rzp = rrp + nsm;
  double* beta_s = rzp + nsm;
  // the per-system scalars as they were when the launch began: rank 0 updates
  // them in global memory while the other CTAs of the cluster still decide on them
  double* rz0 = beta_s + nsm;
  double* it0 = rz0 + nsm;
  double* tol2 = it0 + nsm;
  int* on_s = reinterpret_cast<int*>(base + L.si);    // active at the start of the iteration
  int* cont_s = on_s + nsm;                            // still active after the stopping test
  double* f = a.sys;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // the Phi_k slice is copied while the scalars and the vector update run
  const float2* phi = a.phi_all + (size_t)a.phi_off[k] * a.ld + g0;
  for (int e = threadIdx.x; e < nocc * ng; e += kFT) {
    const int m = e / ng, gi = e - m * ng;
    cp_async8(phs + (size_t)m * lds + gi, phi + (size_t)m * a.ld + gi);
  }

  // alpha = <r, z> / <p, Ap> (the partials of the forward z-pass, in order)
  for (int t = threadIdx.x; t < nsm; t += kFT) {
    int on = 0;
    double al = 0.0;
    double rz = 0.0, its = 0.0, t2 = 0.0;
    if (t < ns) {
      const int s = s0 + t;
      rz = f[kSysRz * nsys + s];
      its = f[kSysIters * nsys + s];
      t2 = f[kSysTol2 * nsys + s];
      on = a.active[s];
      if (on) {
        double pap = 0.0;
        for (int c = 0; c < a.nzf; ++c) pap += a.zpart[(size_t)s * a.nzf + c];
        al = rz / pap;
        if (!(pap > 0.0) || !isfinite(al)) {   // numeric stop
          on = 0;
          if (rank == 0) {
            f[kSysPap * nsys + s] = pap;
            f[kSysStatus * nsys + s] = 2;
            f[kSysAlpha * nsys + s] = 0.0;
            a.active[s] = 0;
          }
        } else if (rank == 0) {
          f[kSysPap * nsys + s] = pap;
          f[kSysAlpha * nsys + s] = al;
        }
      }
    }
    on_s[t] = on;
    cont_s[t] = 0;
    alpha_s[t] = al;
    rz0[t] = rz;
    it0[t] = its;
    tol2[t] = t2;
    rrp[t] = 0.0;
    rzp[t] = 0.0;
  }
  __syncthreads();

  // x += alpha p, r -= alpha Ap, z = M^-1 r (kept in shared memory), ||r||^2 of the slice
  // (a lane loads all of its elements first, so their latencies overlap)
  for (int j = warp; j < ns; j += kFW) {
    if (!on_s[j]) continue;
    const int s = s0 + j;
    const float al = (float)alpha_s[j];
    const float kappa = (float)f[kSysKappa * nsys + s];
    const size_t ob = (size_t)s * a.ld + g0;
    float2 p[kFU], w[kFU], x[kFU], r[kFU];
    float kn[kFU];
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) {
        p[u] = a.P[ob + gi];
        w[u] = a.W[ob + gi];
        x[u] = a.X[ob + gi];
        r[u] = a.Rv[ob + gi];
        kn[u] = a.kin_all[(size_t)k * a.ld + g0 + gi];
      }
    }
    // FP32 per lane (at most 2 kFU terms), FP64 across the lanes and ranks: FP64 arithmetic runs
    // at a small fraction of the FP32 rate, and the FP32 vectors carry FP32 rounding already
    float rrf = 0.f;
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) {
        x[u].x += al * p[u].x;
        x[u].y += al * p[u].y;
        r[u].x -= al * w[u].x;
        r[u].y -= al * w[u].y;
        a.X[ob + gi] = x[u];
        a.Rv[ob + gi] = r[u];
        const float mi = 1.f / (kappa + kn[u]);
        zs[(size_t)j * lds + gi] = make_float2(r[u].x * mi, r[u].y * mi);
        rrf = fmaf(r[u].x, r[u].x, fmaf(r[u].y, r[u].y, rrf));
      }
    }
    const double rr = warp_sum((double)rrf);
    if (lane == 0) rrp[j] = rr;
  }
  cluster.sync();

  // stopping test on ||r||^2 summed over the ranks in order (the same in every CTA)
  for (int t = threadIdx.x; t < ns; t += kFT) {
    if (!on_s[t]) continue;
    double rr = 0.0;
    for (int q = 0; q < CS; ++q) rr += cluster.map_shared_rank(rrp, q)[t];
    const int s = s0 + t;
    const double it = it0[t] + 1;
    int status = 0;
    if (!isfinite(rr)) status = 2;
    else if (rr <= tol2[t]) status = 1;
    else if (it >= a.maxit) status = 3;
    cont_s[t] = status == 0;
    if (rank == 0) {
      f[kSysRr * nsys + s] = rr;
      f[kSysIters * nsys + s] = it;
      if (status) {
        f[kSysStatus * nsys + s] = status;
        a.active[s] = 0;
      } else {
        const int slot = atomicAdd(a.counter, 1);
        a.list[slot] = s;   // any order: each system's work is independent of its slot
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // Phi^H z over the slice: 3 orbitals x 1 system per thread (FP32 within the slice)
  {
    const int nmt = (nocc + 2) / 3;
    for (int tile = threadIdx.x; tile < nmt * ns; tile += kFT) {
      const int mt = tile % nmt, j = tile / nmt;
      float ax[3] = {0.f, 0.f, 0.f}, ay[3] = {0.f, 0.f, 0.f};
      const int mm = min(3, nocc - 3 * mt);
      const float2* pr[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) pr[u] = phs + (size_t)(3 * mt + min(u, mm - 1)) * lds;
      const float2* zr = zs + (size_t)j * lds;
#pragma unroll 4
      for (int gi = 0; gi < ng; ++gi) {
        const float2 z = zr[gi];
#pragma unroll
        for (int u = 0; u < 3; ++u) {   // conj(phi) z
          const float2 q = pr[u][gi];
          ax[u] += q.x * z.x + q.y * z.y;
          ay[u] += q.x * z.y - q.y * z.x;
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (u < mm) cpart[(size_t)(3 * mt + u) * nsm + j] = make_float2(ax[u], ay[u]);
    }
  }
  cluster.sync();

  // distributed reduction of the coefficients: rank q mod CS adds entry q over the ranks
  const int ncoef = nocc * nsm;
  for (int q = rank + CS * threadIdx.x; q < ncoef; q += CS * kFT) {
    if (q % nsm >= ns) continue;
    double sx = 0.0, sy = 0.0;
    for (int r = 0; r < CS; ++r) {
      const float2 v = cluster.map_shared_rank(cpart, r)[q];
      sx += v.x;
      sy += v.y;
    }
    cred[q] = make_float2((float)sx, (float)sy);
  }
  cluster.sync();
  for (int q = threadIdx.x; q < ncoef; q += kFT) {
    if (q % nsm >= ns) continue;
    cfull[q] = cluster.map_shared_rank(cred, q % CS)[q];
  }
  __syncthreads();

  // z -= Phi_k C on the slice, <r, z> of the slice
  for (int j = warp; j < ns; j += kFW) {
    if (!cont_s[j]) continue;
    const int s = s0 + j;
    const size_t ob = (size_t)s * a.ld + g0;
    float2 z[kFU], r[kFU];
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) {
        z[u] = zs[(size_t)j * lds + gi];
        r[u] = a.Rv[ob + gi];
      }
    }
    for (int m = 0; m < nocc; ++m) {
      const float2 c = cfull[(size_t)m * nsm + j];
      const float2* pm = phs + (size_t)m * lds;
#pragma unroll
      for (int u = 0; u < kFU; ++u) {
        const int gi = lane + 32 * u;
        if (gi < ng) {
          const float2 q = pm[gi];
          z[u].x -= q.x * c.x - q.y * c.y;
          z[u].y -= q.x * c.y + q.y * c.x;
        }
      }
    }
    float rzf = 0.f;                                              // FP32 per lane, as ||r||^2
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) {
        zs[(size_t)j * lds + gi] = z[u];
        rzf = fmaf(r[u].x, z[u].x, fmaf(r[u].y, z[u].y, rzf));
      }
    }
    const double rz = warp_sum((double)rzf);
    if (lane == 0) rzp[j] = rz;
  }
  cluster.sync();

  // beta = <r, z>_new / <r, z>_old, summed over the ranks in order
  for (int t = threadIdx.x; t < ns; t += kFT) {
    if (!cont_s[t]) continue;
    double rz = 0.0;
    for (int q = 0; q < CS; ++q) rz += cluster.map_shared_rank(rzp, q)[t];
    const int s = s0 + t;
    double b = rz / rz0[t];
    b = isfinite(b) ? b : 0.0;
    beta_s[t] = b;
    if (rank == 0) {
      f[kSysBeta * nsys + s] = b;
      f[kSysRz * nsys + s] = rz;
    }
  }
  __syncthreads();

  // p = z + beta p
  for (int j = warp; j < ns; j += kFW) {
    if (!cont_s[j]) continue;
    const int s = s0 + j;
    const float b = (float)beta_s[j];
    const size_t ob = (size_t)s * a.ld + g0;
    float2 p[kFU];
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) p[u] = a.P[ob + gi];
    }
#pragma unroll
    for (int u = 0; u < kFU; ++u) {
      const int gi = lane + 32 * u;
      if (gi < ng) {
        const float2 z = zs[(size_t)j * lds + gi];
        a.P[ob + gi] = make_float2(z.x + b * p[u].x, z.y + b * p[u].y);
      }
    }
  }
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
}

namespace {

struct FusedPlan {
  bool ok = false;
  int cs = 0, sl = 0, lds = 0, nsmax = 0;
  size_t smem = 0;
};

FusedPlan plan_fused(ikr_ctx* c, const SysList& L, int maxcnt) {
  FusedPlan p;
  for (int v : L.kcount) p.nsmax = std::max(p.nsmax, v);
  if (c->cgf_nsmax == p.nsmax && c->cgf_maxcnt == maxcnt && c->cgf_planned_force == c->cgf_force) {
    // planned before for this shape
    p.ok = c->cgf_ok;
    p.cs = c->cgf_cs;
    p.sl = c->cgf_sl;
    p.lds = c->cgf_lds;
    p.smem = c->cgf_smem;
    return p;
  }
  c->cgf_nsmax = p.nsmax;
  c->cgf_maxcnt = maxcnt;
  c->cgf_planned_force = c->cgf_force;
  c->cgf_ok = false;
  if (p.nsmax == 0 || p.nsmax > 64 || maxcnt > 64) return p;
  // IKR_CG_FUSED=0 selects the unfused sequence of kernels (read when a context plans)
  if (const char* e = std::getenv("IKR_CG_FUSED"))
    if (e[0] == '0') return p;
  int max_optin = 0, dev = 0;
  IKR_CUDA(cudaGetDevice(&dev));
  IKR_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the cluster size with the fewest waves of clusters (all k-points at once
  // when possible; a GPC holds one cluster of 16 CTAs of this size), then the
  // largest size
  const int nk = (int)c->k.size();
  int best_waves = 0;
  for (int cs : {16, 12, 10, 8}) {
    if (c->cgf_force > 0 && cs != c->cgf_force) continue;   // the autotuner's choice only
    const int sl = (c->ld + cs - 1) / cs;
    if (sl > 32 * kFU) continue;
    const int lds = sl | 1;
    const CgFusedLayout lay(p.nsmax, maxcnt, lds);
    if (lay.total > (size_t)max_optin) continue;
    if (cs > 8) IKR_CUDA(cudaFuncSetAttribute(k_cg_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    IKR_CUDA(cudaFuncSetAttribute(k_cg_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs, (unsigned)nk, 1);
    cfg.blockDim = dim3(kFT, 1, 1);
    cfg.dynamicSmemBytes = lay.total;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_cg_fused, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (nclusters < 1) continue;
    const int waves = (nk + nclusters - 1) / nclusters;
    if (p.ok && waves >= best_waves) continue;
    best_waves = waves;
    p.ok = true;
    p.cs = cs;
    p.sl = sl;
    p.lds = lds;
    p.smem = lay.total;
  }
  if (p.ok) {
    // the attributes of the chosen size
    IKR_CUDA(cudaFuncSetAttribute(k_cg_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    c->cgf_ok = true;
    c->cgf_cs = p.cs;
    c->cgf_sl = p.sl;
    c->cgf_lds = p.lds;
    c->cgf_smem = p.smem;
  }
  return p;
}

}  // namespace

int cg_fused_cluster(ikr_ctx* c, const SysList& L, int maxcnt) {
  const FusedPlan p = plan_fused(c, L, maxcnt);
  return p.ok ? p.cs : 0;
}

bool launch_cg_fused(ikr_ctx* c, const SysList& L, float2* X, float2* Rv, float2* P, const float2* W, double* sys,
                     int maxit, int* active, int* counter, int* list, const double* zpart, int nzf,
                     const OrbSet* set) {
  const OrbSet os = set ? *set : occ_set(c);
  const FusedPlan p = plan_fused(c, L, os.maxcnt);
  if (!p.ok) return false;
  CgFusedArgs a;
  a.X = X;
  a.Rv = Rv;
  a.P = P;
  a.W = W;
  a.phi_all = os.phi32;
  a.phi_off = os.off;
  a.kin_all = c->d_kin_all32.p;
  a.nb_k = c->d_nb.p;
  a.nocc_k = os.cnt;
  a.kstart = L.d_kstart.p;
  a.kcount = L.d_kcount.p;
  a.sys = sys;
  a.nsys = L.n;
  a.maxit = maxit;
  a.active = active;
  a.counter = counter;
  a.list = list;
  a.zpart = zpart;
  a.nzf = nzf;
  a.ld = c->ld;
  a.sl = p.sl;
  a.lds = p.lds;
  a.nsmax = p.nsmax;
  a.noccmax = os.maxcnt;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(p.cs, (unsigned)c->k.size(), 1);
  cfg.blockDim = dim3(kFT, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = c->stream;
  // the attributes belong to the kernel, not to this context: another context's plan may
  // have set a smaller shared-memory size since this plan was made
  if (p.cs > 8) IKR_CUDA(cudaFuncSetAttribute(k_cg_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  IKR_CUDA(cudaFuncSetAttribute(k_cg_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  IKR_CUDA(cudaLaunchKernelEx(&cfg, k_cg_fused, a));
  return true;
}

}  // namespace ikr
