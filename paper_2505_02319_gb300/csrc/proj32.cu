// FP32 projections of the Sternheimer CG (the Q = 1 - Phi_k Phi_k^H of
// eq. discretised_sternheimer applied to the preconditioned residual):
//   C = Phi_k^H Y             (k_pc32 partial sums over chunks of kKG plane
//                              waves, k_pr: a warp per coefficient sums the
//                              chunks with a fixed shuffle tree)
//   out = alpha in + beta Phi_k C, and Re <dv, out> per chunk     (k_pa32)
// Both are skinny products (N_occ,k rows against Nb_k plane waves, a few dozen
// systems per k-point), so the kernels are register-tiled CUDA-core GEMMs whose
// tiles are staged in shared memory by cp.async: k_pc32 keeps 3 orbitals x 4
// systems per thread (7 shared loads per 12 complex FMAs), k_pa32 4 plane
// waves x 2 systems (6 loads per 8).  Partial sums are FP32 within a chunk and
// FP64 across chunks, in a fixed order.
#include "ops.hpp"

namespace ikr {

namespace {
constexpr int kPG = 64;          // plane waves per apply block (and dot-partial chunk)
constexpr int kKG = 32;          // plane waves per coefficient block (chunk of the partial sums)
constexpr int kLP = kKG + 1;     // padded row of a staged tile (odd: conflict-free columns)
constexpr int kCM = 36;          // orbitals per coefficient block (12 groups of 3)
constexpr int kCS = 32;          // systems per coefficient block (8 groups of 4)
constexpr int kCT = 96;          // threads of a coefficient block
constexpr int kAS = 16;          // systems per apply block (8 groups of 2)
constexpr int kAT = 128;         // threads of an apply block (16 plane-wave lanes x 8 system groups)
}  // namespace

__global__ void __launch_bounds__(kCT)
    k_pc32(const float2* __restrict__ phi_all, int ld, const int* __restrict__ phi_off,
           const int* __restrict__ nocc_k, const int* __restrict__ nb_k, const int* __restrict__ kstart,
           const int* __restrict__ kcount, const float2* __restrict__ Y, int ldy, const int* __restrict__ active,
           int nsys, int noccmax, int nst, int nch, double2* __restrict__ part) {
  __shared__ float2 ph[kCM][kLP];
  __shared__ float2 ys[kCS][kLP];
  const int k = blockIdx.y, chunk = blockIdx.x;
  const int mt = blockIdx.z / nst, st = blockIdx.z - mt * nst;
  const int ns = kcount[k], nocc = nocc_k[k], nb = nb_k[k];
  const int m0 = mt * kCM, sl0 = st * kCS, g0 = chunk * kKG;
  if (m0 >= nocc || sl0 >= ns || g0 >= nb) return;   // uniform over the block
  const int s0 = kstart[k] + sl0;
  const float2* phi = phi_all + ((size_t)phi_off[k] + m0) * ld;
  for (int e = threadIdx.x; e < kCM * kKG; e += kCT) {
    const int r = e / kKG, g = e - r * kKG;
    const bool ok = m0 + r < nocc && g0 + g < nb;
    cp_async8_zfill(&ph[r][g], phi + (ok ? (size_t)r * ld + g0 + g : 0), ok);
  }
  for (int e = threadIdx.x; e < kCS * kKG; e += kCT) {
    const int r = e / kKG, g = e - r * kKG;
    const bool ok = sl0 + r < ns && g0 + g < nb;
    cp_async8_zfill(&ys[r][g], Y + (ok ? (size_t)(s0 + r) * ldy + g0 + g : 0), ok);
  }
  cp_async_wait_all();
  __syncthreads();
  const int mi = threadIdx.x % 12, si = threadIdx.x / 12;
  float ax[3][4], ay[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) ax[a][b] = ay[a][b] = 0.f;
#pragma unroll 4
  for (int g = 0; g < kKG; ++g) {
    float2 p[3], y[4];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = ph[3 * mi + a][g];
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = ys[4 * si + b][g];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {   // conj(p) y
        ax[a][b] += p[a].x * y[b].x + p[a].y * y[b].y;
        ay[a][b] += p[a].x * y[b].y - p[a].y * y[b].x;
      }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int m = m0 + 3 * mi + a, sl = sl0 + 4 * si + b;
      if (m < nocc && sl < ns && (!active || active[s0 - sl0 + sl]))
        part[((size_t)(s0 - sl0 + sl) * noccmax + m) * nch + chunk] = make_double2(ax[a][b], ay[a][b]);
    }
}

// coef[s][m] = sum over the chunks c < ceil(Nb_k / kKG) of part[s][m][c]: one
// warp per coefficient, lane l adds chunks l, l + 32, ... (coalesced), then a
// fixed shuffle tree
__global__ void k_pr(const double2* __restrict__ part, int nsys, int noccmax, int nch, const int* __restrict__ sys_k,
                     const int* __restrict__ nocc_k, const int* __restrict__ nb_k, const int* __restrict__ active,
                     double2* __restrict__ coef) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nsys * noccmax) return;   // uniform over the warp
  const int s = (int)(w / noccmax), m = (int)(w - (long long)s * noccmax);
  if (active && !active[s]) return;
  const int k = sys_k[s];
  if (m >= nocc_k[k]) return;
  const int nc = (nb_k[k] + kKG - 1) / kKG;
  const double2* p = part + ((size_t)s * noccmax + m) * nch;
  double ax = 0.0, ay = 0.0;
  for (int c = lane; c < nc; c += 32) {
    const double2 v = p[c];
    ax += v.x;
    ay += v.y;
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  if (lane == 0) coef[w] = make_double2(ax, ay);
}

__global__ void __launch_bounds__(kAT)
    k_pa32(const float2* __restrict__ phi_all, int ld, const int* __restrict__ phi_off,
           const int* __restrict__ nocc_k, const int* __restrict__ nb_k, const int* __restrict__ kstart,
           const int* __restrict__ kcount, const double2* __restrict__ coef, int noccmax, const float2* in,
           float alpha, float beta, float2* out, int ldy, const float2* __restrict__ dv, double* __restrict__ dpart,
           int nparts, const int* __restrict__ active) {
  extern __shared__ float4 smem_pa[];
  float2* ph = reinterpret_cast<float2*>(smem_pa);   // [nocc][kPG]
  float2* cf = ph + (size_t)noccmax * kPG;          // [nocc][kAS]
  const int k = blockIdx.y, chunk = blockIdx.x;
  const int ns = kcount[k], nocc = nocc_k[k], nb = nb_k[k];
  const int sl0 = blockIdx.z * kAS, g0 = chunk * kPG;
  if (sl0 >= ns) return;   // uniform
  const int s0 = kstart[k] + sl0, nsl = min(kAS, ns - sl0);
  const int live = threadIdx.x < nsl && (!active || active[s0 + threadIdx.x]);
  if (!__syncthreads_or(live)) return;   // a tile of converged systems
  const float2* phi = phi_all + (size_t)phi_off[k] * ld;
  for (int e = threadIdx.x; e < nocc * kPG; e += kAT) {
    const int r = e / kPG, g = e - r * kPG;
    const bool ok = g0 + g < nb;
    cp_async8_zfill(ph + e, phi + (ok ? (size_t)r * ld + g0 + g : 0), ok);
  }
  for (int e = threadIdx.x; e < nocc * kAS; e += kAT) {
    const int m = e / kAS, j = e - m * kAS;
    float2 v = make_float2(0.f, 0.f);
    if (j < nsl) {
      const double2 d = coef[(size_t)(s0 + j) * noccmax + m];
      v = make_float2((float)d.x, (float)d.y);
    }
    cf[e] = v;
  }
  cp_async_wait_all();
  __syncthreads();
  const int tg = threadIdx.x & 15, ts = threadIdx.x >> 4;
  // the epilogue's operands are loaded now, so their latency overlaps the sums
  float2 xin[4][2], wdv[4][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int sl = 2 * ts + j;
    const bool on = sl < nsl && (!active || active[s0 + sl]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = g0 + tg + 16 * i;
      const size_t o = (size_t)(s0 + sl) * ldy + g;
      const bool ld_ok = on && g < nb;
      xin[i][j] = (ld_ok && alpha != 0.f) ? in[o] : make_float2(0.f, 0.f);
      wdv[i][j] = (ld_ok && dv) ? dv[o] : make_float2(0.f, 0.f);
    }
  }
  float2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int m = 0; m < nocc; ++m) {
    float2 p[4], c[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = ph[m * kPG + tg + 16 * i];
#pragma unroll
    for (int j = 0; j < 2; ++j) c[j] = cf[m * kAS + 2 * ts + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        acc[i][j].x += p[i].x * c[j].x - p[i].y * c[j].y;
        acc[i][j].y += p[i].x * c[j].y + p[i].y * c[j].x;
      }
  }
  float dd[2] = {0.f, 0.f};   // FP32 over the thread's plane waves and the 16 lanes, stored in FP64
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int sl = 2 * ts + j;
    const int s = s0 + sl;
    const bool on = sl < nsl && (!active || active[s]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = g0 + tg + 16 * i;
      if (on && g < nb) {
        const size_t o = (size_t)s * ldy + g;
        float2 v = make_float2(beta * acc[i][j].x, beta * acc[i][j].y);
        if (alpha != 0.f) {
          v.x += alpha * xin[i][j].x;
          v.y += alpha * xin[i][j].y;
        }
        out[o] = v;
        if (dv) dd[j] = fmaf(wdv[i][j].x, v.x, fmaf(wdv[i][j].y, v.y, dd[j]));
      }
    }
  }
  if (dpart) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float t = dd[j];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int sl = 2 * ts + j;
      if (tg == 0 && sl < nsl && (!active || active[s0 + sl])) dpart[(size_t)(s0 + sl) * nparts + chunk] = (double)t;
    }
  }
}

int proj_chunks32() { return kPG; }

void proj_coef32(ikr_ctx* c, const SysList& L, const float2* Y, int ldy, const int* active, double2* coef,
                 const OrbSet& set) {
  // the tensor-core coefficient kernel reads two plane waves per 16-byte load: even strides
  // only (vectors in a caller's layout, e.g. Nb_k-strided, take the CUDA cores)
  if (tc_proj_ok(c, set) && ldy % 2 == 0) {
    proj_coef_tc(c, L, Y, ldy, active, coef, set);
    return;
  }
  const int nch = (c->ld + kKG - 1) / kKG;
  const int nm = set.maxcnt;
  c->ws.cpart.reserve((size_t)nch * L.n * nm * 2);
  double2* part = reinterpret_cast<double2*>(c->ws.cpart.p);
  int maxns = 0;
  for (int v : L.kcount) maxns = std::max(maxns, v);
  const int nst = std::max(1, (maxns + kCS - 1) / kCS), nmt = std::max(1, (nm + kCM - 1) / kCM);
  dim3 grid(nch, (unsigned)c->k.size(), nst * nmt);
  k_pc32<<<grid, kCT, 0, c->stream>>>(set.phi32, c->ld, set.off, set.cnt, c->d_nb.p,
                                      L.d_kstart.p, L.d_kcount.p, Y, ldy, active, L.n, nm, nst, nch, part);
  IKR_CUDA(cudaGetLastError());
  const long long threads = 32LL * L.n * nm;
  k_pr<<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(part, L.n, nm, nch, L.d_k.p, set.cnt,
                                                                  c->d_nb.p, active, coef);
  IKR_CUDA(cudaGetLastError());
}

void proj_apply32(ikr_ctx* c, const SysList& L, const double2* coef, const float2* in, float alpha, float beta,
                  float2* out, int ldy, const float2* dv, double* dpart, const int* active, const OrbSet& set) {
  if (tc_proj_ok(c, set)) {
    proj_apply_tc(c, L, coef, in, alpha, beta, out, ldy, dv, dpart, active, set);
    return;
  }
  const int nch = (c->ld + kPG - 1) / kPG;
  const int nm = std::max(set.maxcnt, 1);
  int maxns = 0;
  for (int v : L.kcount) maxns = std::max(maxns, v);
  const size_t smem = sizeof(float2) * (size_t)nm * (kPG + kAS);
  IKR_CUDA(cudaFuncSetAttribute(k_pa32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(nch, (unsigned)c->k.size(), std::max(1, (maxns + kAS - 1) / kAS));
  k_pa32<<<grid, kAT, smem, c->stream>>>(set.phi32, c->ld, set.off, set.cnt, c->d_nb.p,
                                         L.d_kstart.p, L.d_kcount.p, coef, set.maxcnt, in, alpha, beta, out, ldy, dv,
                                         dpart, nch, active);
  IKR_CUDA(cudaGetLastError());
}

}  // namespace ikr
