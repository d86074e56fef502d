// FP32 plane pass of the batched H_k application with one thread per line.
//
// Same result as k_plane_t (fft_plane.cu): for each system and z-plane,
// the inverse y-transforms of the active x positions, the inverse x-transforms
// of every row, the product with the potential row, and the forward
// transforms back, restricted to the sphere columns (the y/x part of the
// pruned F^-1 V F of eq. fft_ifft).  Here a whole line of length N <= 48 lives
// in the registers of one thread, so a transform needs no exchange between
// threads: the shared-memory traffic is one load and one store per element and
// phase, and every twiddle factor is a compile-time constant (ct_trig.hpp).
// Loads and stores are also pruned to the elements that can be non-zero:
//   - a y-line reads only the y-interval of its sphere column and writes back
//     only that interval after the forward transform;
//   - an x-line reads and writes only the active x positions (all positions
//     when the input is a real-space plane).
// One block holds one z-plane of PL systems and the potential plane, staged
// once for the PL systems.  Shared-memory layout (bank-conflict free for all
// phases with PL = 16 / (lanes per row group)): column x of a row is stored
// at (x + NX/2) mod NX, which makes the active x positions of a centred sphere
// contiguous; the row stride ldp is odd and the plane stride is 16/PL modulo
// 16 elements.
#include "ct_trig.hpp"
#include "ops.hpp"

namespace ikr {

namespace {

// a * W_N^X (forward W = e^{-2 pi i/N}; conjugate for the inverse)
template <typename C, int N, int X, bool INV>
__device__ __forceinline__ C twmul(C a) {
  constexpr int x = X % N;
  if constexpr (x == 0) {
    return a;
  } else if constexpr (2 * x == N) {
    return mk<C>(-a.x, -a.y);
  } else if constexpr (4 * x == N) {
    return rot<C, INV>(a);
  } else if constexpr (4 * x == 3 * N) {
    return rot<C, !INV>(a);
  } else {
    using R = decltype(C::x);
    constexpr double c = CtTwiddle<N, x>::c;
    constexpr double s = INV ? CtTwiddle<N, x>::s : -CtTwiddle<N, x>::s;
    const R cr = R(c), sr = R(s);
    return mk<C>(a.x * cr - a.y * sr, a.x * sr + a.y * cr);
  }
}

// u[p][k2] *= W_E^{p k2} for p in [p0, P), k2 in [k, Q), unrolled at compile time
template <typename C, int E, int P, int Q, bool INV, int p, int k>
struct TwiddlePass {
  __device__ __forceinline__ static void run(C (&u)[P][Q]) {
    if constexpr (p < P) {
      if constexpr (k < Q) {
        u[p][k] = twmul<C, E, p * k, INV>(u[p][k]);
        TwiddlePass<C, E, P, Q, INV, p, k + 1>::run(u);
      } else {
        TwiddlePass<C, E, P, Q, INV, p + 1, 1>::run(u);
      }
    }
  }
};

// E-point DFT in registers, natural order in and out, compile-time twiddles.
// E = P Q with the factors of fft_plane.cu's Split (4 first, then 2, 3, 5):
//   X_{k2 + Q k1} = sum_p W_P^{p k1} W_E^{p k2} sum_q x_{p + P q} W_Q^{q k2}.
template <int E> struct CtSplit {
  static constexpr bool base = (E == 2 || E == 3 || E == 4 || E == 5);
  static constexpr int P = base ? E : (E % 4 == 0) ? 4 : (E % 2 == 0) ? 2 : (E % 3 == 0) ? 3 : 5;
  static constexpr int Q = E / P;
};

template <typename C, int E, bool INV> struct CtFft {
  __device__ __forceinline__ static void run(C* v) {
    constexpr int P = CtSplit<E>::P, Q = CtSplit<E>::Q;
    if constexpr (Q == 1) {
      Dft<C, E, INV>::run(v);
    } else {
      C u[P][Q];
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int q = 0; q < Q; ++q) u[p][q] = v[p + P * q];
#pragma unroll
      for (int p = 0; p < P; ++p) CtFft<C, Q, INV>::run(u[p]);
      TwiddlePass<C, E, P, Q, INV, 1, 1>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        C w[P];
#pragma unroll
        for (int p = 0; p < P; ++p) w[p] = u[p][k2];
        Dft<C, P, INV>::run(w);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) v[k2 + Q * k1] = w[k1];
      }
    }
  }
};
template <typename C, bool INV> struct CtFft<C, 1, INV> {
  __device__ __forceinline__ static void run(C*) {}
};

}  // namespace

template <int NX, int NY> struct RegGeom {
  static constexpr int PL = NY >= 32 ? 4 : (NY >= 16 ? 8 : 16);   // systems per block
  static constexpr int ldp = NX | 1;                                // odd row stride
  static constexpr int ps0 = NY * ldp;
  static constexpr int PS = ps0 + (((16 / PL) - ps0) % 16 + 16) % 16;   // plane stride = 16/PL mod 16
  static constexpr int NTH = (PL * NY + 31) / 32 * 32;
  static constexpr int SH = NX / 2;
  static constexpr size_t smem(int nxa) {
    return sizeof(float2) * (size_t)PL * PS + sizeof(float) * (size_t)NY * ldp + sizeof(int) * 3 * (size_t)nxa;
  }
};

template <int NX, int NY>
__global__ void __launch_bounds__(RegGeom<NX, NY>::NTH)
    k_plane_r(const float2* __restrict__ b1, int nc, int ncp, const int* __restrict__ col_xy,
              const int* __restrict__ xr, int nxa, unsigned long long xmask, int Nz,
              const float* __restrict__ pot, const double* __restrict__ pot_scale,
              const int* __restrict__ active, int nsys, const int* __restrict__ list,
              float2* __restrict__ b4, const float2* __restrict__ real_in) {
  using G = RegGeom<NX, NY>;
  constexpr int PL = G::PL, ldp = G::ldp, PS = G::PS, NTH = G::NTH, SH = G::SH;
  const int iz = blockIdx.x;
  __shared__ int live[PL];   // system of slot j, or -1
  extern __shared__ float4 smem_r[];
  float2* planes = reinterpret_cast<float2*>(smem_r);
  float* pot_s = reinterpret_cast<float*>(planes + PL * PS);
  int* xr_s = reinterpret_cast<int*>(pot_s + NY * ldp);
  if (threadIdx.x < PL) {
    const int i = blockIdx.y * PL + threadIdx.x;
    int s = -1;
    if (i < nsys) {
      s = list ? list[i] : i;
      if (active && !active[s]) s = -1;
    }
    live[threadIdx.x] = s;
  }
  __syncthreads();
  int nlive = 0;
#pragma unroll
  for (int j = 0; j < PL; ++j) nlive += live[j] >= 0;
  if (nlive == 0) return;   // uniform over the block
  const float2 zero = make_float2(0.f, 0.f);
  const int2* cxy = reinterpret_cast<const int2*>(col_xy);
#pragma unroll 4
  for (int e = threadIdx.x; e < NY * NX; e += NTH) {
    const int iy = e / NX, ix = e - iy * NX;
    cp_async4(pot_s + iy * ldp + ix, pot + (size_t)iz * NY * NX + e);
  }
  for (int e = threadIdx.x; e < 3 * nxa; e += NTH) cp_async4(xr_s + e, xr + e);
  if (real_in) {
#pragma unroll 4
    for (int e = threadIdx.x; e < PL * NY * NX; e += NTH) {
      const int j = e / (NY * NX), r = e - j * (NY * NX);
      if (live[j] < 0) continue;
      const int iy = r / NX, ix = r - iy * NX;
      const int px = ix + SH >= NX ? ix + SH - NX : ix + SH;
      cp_async8(planes + j * PS + iy * ldp + px, real_in + ((size_t)live[j] * Nz + iz) * NY * NX + r);
    }
  } else {
#pragma unroll 4
    for (int e = threadIdx.x; e < PL * nc; e += NTH) {
      const int j = e / nc, col = e - j * nc;
      if (live[j] < 0) continue;
      const int2 xy = cxy[col];
      const int px = xy.x + SH >= NX ? xy.x + SH - NX : xy.x + SH;
      cp_async8(planes + j * PS + xy.y * ldp + px, b1 + ((size_t)live[j] * Nz + iz) * ncp + col);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // inverse y-lines of the active x positions: only the column's y-interval is non-zero
  if (!real_in) {
    for (int it = threadIdx.x; it < PL * nxa; it += NTH) {
      const int l = it / PL, j = it - l * PL;
      if (live[j] < 0) continue;
      const int px = xr_s[3 * l], ylo = xr_s[3 * l + 1], span = xr_s[3 * l + 2];
      float2* colp = planes + j * PS + px;
      float2 v[NY];
#pragma unroll
      for (int y = 0; y < NY; ++y) {
        int d = y - ylo;
        d += d < 0 ? NY : 0;
        v[y] = d <= span ? colp[y * ldp] : zero;
      }
      CtFft<float2, NY, true>::run(v);
#pragma unroll
      for (int y = 0; y < NY; ++y) colp[y * ldp] = v[y];
    }
    __syncthreads();
  }
  // x-lines: inverse transform (unless real-space input), potential, forward transform
  {
    const float sc = pot_scale ? (float)*pot_scale : 1.f;
    const unsigned long long m = real_in ? ~0ull : xmask;
    for (int it = threadIdx.x; it < PL * NY; it += NTH) {
      const int iy = it / PL, j = it - iy * PL;
      if (live[j] < 0) continue;
      float2* row = planes + j * PS + iy * ldp;
      const float* prow = pot_s + iy * ldp;
      float2 v[NX];
#pragma unroll
      for (int x = 0; x < NX; ++x) v[x] = ((m >> x) & 1ull) ? row[(x + SH) % NX] : zero;
      if (!real_in) CtFft<float2, NX, true>::run(v);
#pragma unroll
      for (int x = 0; x < NX; ++x) v[x] = cscale(v[x], prow[x] * sc);
      CtFft<float2, NX, false>::run(v);
#pragma unroll
      for (int x = 0; x < NX; ++x)
        if ((xmask >> x) & 1ull) row[(x + SH) % NX] = v[x];
    }
  }
  __syncthreads();
  // forward y-lines of the active x positions; only the sphere interval is kept
  for (int it = threadIdx.x; it < PL * nxa; it += NTH) {
    const int l = it / PL, j = it - l * PL;
    if (live[j] < 0) continue;
    const int px = xr_s[3 * l], ylo = xr_s[3 * l + 1], span = xr_s[3 * l + 2];
    float2* colp = planes + j * PS + px;
    float2 v[NY];
#pragma unroll
    for (int y = 0; y < NY; ++y) v[y] = colp[y * ldp];
    CtFft<float2, NY, false>::run(v);
#pragma unroll
    for (int y = 0; y < NY; ++y) {
      int d = y - ylo;
      d += d < 0 ? NY : 0;
      if (d <= span) colp[y * ldp] = v[y];
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < PL * nc; e += NTH) {
    const int j = e / nc, col = e - j * nc;
    if (live[j] < 0) continue;
    const int2 xy = cxy[col];
    const int px = xy.x + SH >= NX ? xy.x + SH - NX : xy.x + SH;
    b4[((size_t)live[j] * Nz + iz) * ncp + col] = planes[j * PS + xy.y * ldp + px];
  }
}

// Compact variant for z-transformed input (the CG's H_k applications): shared
// memory holds only the nxa active x positions of every row, column l at
// shifted position pxlo + l (setup checks that the active positions form one
// run).  The y-lines act only on those columns, and an x-line reads and writes
// only them as well (its inactive inputs are zero, its inactive outputs are
// dropped), so nothing else of the plane is ever needed: ~42 KB per block of
// PL = 4 systems instead of ~85 KB.  With PL NY / 2 threads every thread takes
// two rows of the x phase and at most one line of each y phase (544 line
// transforms in 6 transform-times for 96 threads, against 4 for 192 threads
// with 58 % of them idle in the y phases), and five blocks fit an SM.
// Bank layout as RegGeom: odd row stride, plane stride 4 mod 16 elements.
template <int NX, int NY> struct RcGeom {
  static constexpr int PL = 4;
  static constexpr int NTH = (PL * NY / 2 + 31) / 32 * 32;
  static constexpr int ldp = NX | 1;                      // potential row stride
  static constexpr int SH = NX / 2;
  __host__ __device__ static constexpr int ldc(int nxa) { return nxa | 1; }
  __host__ __device__ static constexpr int ps(int nxa) {
    return NY * (nxa | 1) + ((4 - NY * (nxa | 1)) % 16 + 16) % 16;
  }
  static size_t smem(int nxa) {
    return sizeof(float2) * (size_t)PL * ps(nxa) + sizeof(float) * (size_t)NY * ldp + sizeof(int) * 3 * (size_t)nxa;
  }
};

template <int NX, int NY, int MINB>
__global__ void __launch_bounds__(RcGeom<NX, NY>::NTH, MINB)
    k_plane_rc(const float2* __restrict__ b1, int nc, int ncp, const int* __restrict__ col_xy,
               const int* __restrict__ xr, int nxa, int pxlo, unsigned long long xmask, int Nz,
               const float* __restrict__ pot, const double* __restrict__ pot_scale,
               const int* __restrict__ active, int nsys, const int* __restrict__ list,
               float2* __restrict__ b4) {
  static_assert(NX == NY, "one transform body serves both line directions");
  using G = RcGeom<NX, NY>;
  constexpr int PL = G::PL, NTH = G::NTH, ldp = G::ldp, SH = G::SH, N = NX;
  const int ldc = G::ldc(nxa), PS = G::ps(nxa);
  const int iz = blockIdx.x;
  __shared__ int live[PL];   // system of slot j, or -1
  extern __shared__ float4 smem_rc[];
  float2* planes = reinterpret_cast<float2*>(smem_rc);
  float* pot_s = reinterpret_cast<float*>(planes + PL * PS);
  int* xr_s = reinterpret_cast<int*>(pot_s + NY * ldp);
  if (threadIdx.x < PL) {
    const int i = blockIdx.y * PL + threadIdx.x;
    int s = -1;
    if (i < nsys) {
      s = list ? list[i] : i;
      if (active && !active[s]) s = -1;
    }
    live[threadIdx.x] = s;
  }
  __syncthreads();
  int nlive = 0;
#pragma unroll
  for (int j = 0; j < PL; ++j) nlive += live[j] >= 0;
  if (nlive == 0) return;   // uniform over the block
  const float2 zero = make_float2(0.f, 0.f);
  const int2* cxy = reinterpret_cast<const int2*>(col_xy);
  for (int e = threadIdx.x; e < NY * NX; e += NTH) {
    const int iy = e / NX, ix = e - iy * NX;
    cp_async4(pot_s + iy * ldp + ix, pot + (size_t)iz * NY * NX + e);
  }
  for (int e = threadIdx.x; e < 3 * nxa; e += NTH) cp_async4(xr_s + e, xr + e);
  for (int e = threadIdx.x; e < PL * nc; e += NTH) {
    const int j = e / nc, col = e - j * nc;
    if (live[j] < 0) continue;
    const int2 xy = cxy[col];
    const int px = xy.x + SH >= NX ? xy.x + SH - NX : xy.x + SH;
    cp_async8(planes + j * PS + xy.y * ldc + (px - pxlo), b1 + ((size_t)live[j] * Nz + iz) * ncp + col);
  }
  cp_async_wait_all();
  __syncthreads();
  const float sc = pot_scale ? (float)*pot_scale : 1.f;
  // Three phases with one forward-transform code site between them (the whole
  // kernel issues one copy of the unrolled FFT, so every warp, whatever its
  // phase, runs the same instructions): an inverse transform is
  // conj(FFT(conj(x))).
  //   phase 0: inverse y-lines of the active columns (input: the column's y-interval)
  //   phase 1: x-lines, two passes: inverse, then conj, times the potential row,
  //            forward; the active x positions are read and written
  //   phase 2: forward y-lines, only the column's interval is kept
#pragma unroll 1
  for (int ph = 0; ph < 3; ++ph) {
    const bool xph = ph == 1;
    const int items = xph ? PL * NY : PL * nxa;
    for (int it = threadIdx.x; it < items; it += NTH) {
      const int line = it / PL, j = it - line * PL;
      if (live[j] < 0) continue;
      float2 v[N];
      float2* colp = planes + j * PS + line;                        // y-line of column `line`
      const int base = j * PS + line * ldc - pxlo;                  // x-line of row `line`
      int ylo = 0, span = N - 1;
      if (!xph) {
        ylo = xr_s[3 * line + 1];
        span = xr_s[3 * line + 2];
      }
      if (xph) {
#pragma unroll
        for (int x = 0; x < N; ++x) {
          const float2 a = ((xmask >> x) & 1ull) ? planes[base + (x + SH) % NX] : zero;
          v[x] = make_float2(a.x, -a.y);
        }
      } else if (ph == 0) {
#pragma unroll
        for (int y = 0; y < N; ++y) {
          int d = y - ylo;
          d += d < 0 ? N : 0;
          const float2 a = d <= span ? colp[y * ldc] : zero;
          v[y] = make_float2(a.x, -a.y);
        }
      } else {
#pragma unroll
        for (int y = 0; y < N; ++y) v[y] = colp[y * ldc];
      }
      const int npass = xph ? 2 : 1;
#pragma unroll 1
      for (int pass = 0; pass < npass; ++pass) {
        if (pass == 1) {
          const float* prow = pot_s + line * ldp;
#pragma unroll
          for (int x = 0; x < N; ++x) {
            const float p = prow[x] * sc;
            v[x] = make_float2(v[x].x * p, -v[x].y * p);
          }
        }
        CtFft<float2, N, false>::run(v);
      }
      if (xph) {
#pragma unroll
        for (int x = 0; x < N; ++x)
          if ((xmask >> x) & 1ull) planes[base + (x + SH) % NX] = v[x];
      } else if (ph == 0) {
#pragma unroll
        for (int y = 0; y < N; ++y) colp[y * ldc] = make_float2(v[y].x, -v[y].y);
      } else {
#pragma unroll
        for (int y = 0; y < N; ++y) {
          int d = y - ylo;
          d += d < 0 ? N : 0;
          if (d <= span) colp[y * ldc] = v[y];
        }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < PL * nc; e += NTH) {
    const int j = e / nc, col = e - j * nc;
    if (live[j] < 0) continue;
    const int2 xy = cxy[col];
    const int px = xy.x + SH >= NX ? xy.x + SH - NX : xy.x + SH;
    b4[((size_t)live[j] * Nz + iz) * ncp + col] = planes[j * PS + xy.y * ldc + (px - pxlo)];
  }
}

namespace {

template <int NX, int NY>
bool try_reg(ikr_ctx* c, int nsys, const float2* b1, const float* pot, const double* pot_scale, const int* active,
             float2* b4, const float2* real_in, const int* list) {
  if (c->N[0] != NX || c->N[1] != NY) return false;
  if constexpr (NX == NY) {
  if (!real_in && c->xr_contig && c->plane_rc) {
    using H = RcGeom<NX, NY>;
    const size_t smem = H::smem(c->nxa);
    if (smem <= 200 * 1024) {
      auto launch = [&](auto kern) {
        IKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dim3 grid(c->N[2], (nsys + H::PL - 1) / H::PL);
        kern<<<grid, H::NTH, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xr.p, c->nxa, c->pxlo,
                                               c->xmask, c->N[2], pot, pot_scale, active, nsys, list, b4);
        IKR_CUDA(cudaGetLastError());
      };
      // register bound: 5 blocks per SM (128 registers) or 4 (up to 168)
      if (c->plane_rc == 4) launch(k_plane_rc<NX, NY, 4>);
      else launch(k_plane_rc<NX, NY, 5>);
      return true;
    }
  }
  }
  using G = RegGeom<NX, NY>;
  const size_t smem = G::smem(c->nxa);
  if (smem > 200 * 1024) return false;
  IKR_CUDA(cudaFuncSetAttribute(k_plane_r<NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int Nz = c->N[2];
  dim3 grid(Nz, (nsys + G::PL - 1) / G::PL);
  k_plane_r<NX, NY><<<grid, G::NTH, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xr.p, c->nxa,
                                                       c->xmask, Nz, pot, pot_scale, active, nsys, list, b4,
                                                       real_in);
  IKR_CUDA(cudaGetLastError());
  return true;
}

}  // namespace

bool launch_plane_reg(ikr_ctx* c, int nsys, const float2* b1, const float* pot, const double* pot_scale,
                      const int* active, float2* b4, const float2* real_in, const int* list, int nlist) {
  if (!c->reg_plane_ok || nsys == 0) return false;
  if (list) {
    if (nlist <= 0) return true;   // nothing active
    nsys = nlist;
  }
  return try_reg<48, 48>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list) ||
         try_reg<32, 32>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list) ||
         try_reg<40, 40>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list) ||
         try_reg<24, 24>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list) ||
         try_reg<12, 12>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list) ||
         try_reg<10, 12>(c, nsys, b1, pot, pot_scale, active, b4, real_in, list);
}


// ------------------------------------------------------------------ z-pass --
// FP32 z-transforms of the sphere columns with one thread per column: the
// column's run of plane waves (consecutive z from its z start, cyclic) becomes
// a z-line in registers, transformed with compile-time twiddles, and written as
// row iz of b1[s][iz][column] (coalesced over the block's columns); the forward
// pass reads the rows back, transforms, and keeps the run.  The columns of a
// block are consecutive, and so are their runs in the sphere order (both are
// lexicographic in (j1, j2)): the block's slice [pre[c0], pre[c1]) of the
// orbital-sized vectors moves through shared memory with coalesced copies.

template <int NZ>
__global__ void __launch_bounds__(kZC)
    k_zi_r(const float2* __restrict__ sphere, int ld, const int* __restrict__ sys_k,
           const int* __restrict__ colinfo, const int* __restrict__ colpre, int nc, int ncp,
           const int* __restrict__ active, const int* __restrict__ list, int nsys, float2* __restrict__ b1) {
  extern __shared__ float4 smem_z[];
  float2* sv = reinterpret_cast<float2*>(smem_z);
  const int i = blockIdx.y;
  if (i >= nsys) return;
  const int s = list ? list[i] : i;
  if (active && !active[s]) return;
  const int k = sys_k[s];
  const int c0 = blockIdx.x * kZC, c1 = min(c0 + kZC, nc);
  const int* pre = colpre + (size_t)k * (nc + 1);
  const int base = pre[c0], span = pre[c1] - base;
  const float2* src = sphere + (size_t)s * ld + base;
  for (int e = threadIdx.x; e < span; e += kZC) cp_async8(sv + e, src + e);
  cp_async_wait_all();
  __syncthreads();
  const int col = c0 + threadIdx.x;
  if (col >= nc) return;
  const int* inf = colinfo + ((size_t)k * nc + col) * 3;
  const int rel = inf[0] - base, cnt = inf[1], zs = inf[2];
  const float2 zero = make_float2(0.f, 0.f);
  float2 v[NZ];
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    int t = z - zs;
    t += t < 0 ? NZ : 0;
    v[z] = t < cnt ? sv[rel + t] : zero;
  }
  CtFft<float2, NZ, true>::run(v);
  float2* dst = b1 + (size_t)s * NZ * ncp + col;
#pragma unroll
  for (int iz = 0; iz < NZ; ++iz) dst[(size_t)iz * ncp] = v[iz];
}

// out = F_z(b4) on the sphere; with psi: out += (|k+G|^2/2 - shift_s) psi and
// dpart[s][block] = Re <psi, out> over the block's plane waves (one warp: a
// fixed shuffle tree).
template <int NZ>
__global__ void __launch_bounds__(kZC)
    k_zf_r(const float2* __restrict__ b4, int nc, int ncp, const int* __restrict__ sys_k,
           const int* __restrict__ colinfo, const int* __restrict__ colpre, int zspan, float2* __restrict__ out,
           int ld, int ldk, const float2* __restrict__ psi, const double* __restrict__ shift,
           const float* __restrict__ kin_all, const int* __restrict__ active, const int* __restrict__ list,
           int nsys, double* __restrict__ dpart) {
  extern __shared__ float4 smem_z[];
  float2* so = reinterpret_cast<float2*>(smem_z);
  float2* sp = so + zspan;
  float* sk = reinterpret_cast<float*>(sp + zspan);
  const int i = blockIdx.y;
  if (i >= nsys) return;
  const int s = list ? list[i] : i;
  if (active && !active[s]) return;
  const int k = sys_k[s];
  const int c0 = blockIdx.x * kZC, c1 = min(c0 + kZC, nc);
  const int* pre = colpre + (size_t)k * (nc + 1);
  const int base = pre[c0], span = pre[c1] - base;
  const float* kin = kin_all ? kin_all + (size_t)k * ldk + base : nullptr;
  if (psi) {
    const float2* ps = psi + (size_t)s * ld + base;
    for (int e = threadIdx.x; e < span; e += kZC) {
      cp_async8(sp + e, ps + e);
      if (kin) cp_async4(sk + e, kin + e);
    }
  }
  const int col = c0 + threadIdx.x;
  float2 v[NZ];
  if (col < nc) {
    const float2* srcc = b4 + (size_t)s * NZ * ncp + col;
#pragma unroll
    for (int iz = 0; iz < NZ; ++iz) v[iz] = srcc[(size_t)iz * ncp];
    CtFft<float2, NZ, false>::run(v);
  }
  cp_async_wait_all();
  __syncthreads();
  float dotf = 0.f;   // FP32 over the column's run, FP64 across the columns (FP64 is slow here)
  if (col < nc) {
    const int* inf = colinfo + ((size_t)k * nc + col) * 3;
    const int rel = inf[0] - base, cnt = inf[1], zs = inf[2];
    const float sh = shift ? (float)shift[s] : 0.f;
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      int t = z - zs;
      t += t < 0 ? NZ : 0;
      if (t < cnt) {
        float2 val = v[z];
        if (psi) {
          const float d = (kin ? sk[rel + t] : 0.f) - sh;
          const float2 p = sp[rel + t];
          val.x += d * p.x;
          val.y += d * p.y;
          dotf = fmaf(p.x, val.x, fmaf(p.y, val.y, dotf));
        }
        so[rel + t] = val;
      }
    }
  }
  __syncthreads();
  float2* dst = out + (size_t)s * ld + base;
  for (int e = threadIdx.x; e < span; e += kZC) dst[e] = so[e];
  if (dpart) {
    const double dot = warp_sum((double)dotf);
    if (threadIdx.x == 0) dpart[(size_t)s * gridDim.x + blockIdx.x] = dot;
  }
}

namespace {

template <int NZ>
bool try_zi(ikr_ctx* c, int nsys, const int* d_k, const float2* sphere, int ld, const int* active, const int* list,
            float2* b1) {
  if (c->N[2] != NZ) return false;
  const size_t smem = sizeof(float2) * (size_t)c->zspan;
  if (smem > 48 * 1024) return false;
  dim3 grid((c->nc + kZC - 1) / kZC, nsys);
  k_zi_r<NZ><<<grid, kZC, smem, c->stream>>>(sphere, ld, d_k, c->k_colinfo.p, c->d_colpre.p, c->nc, c->ncp,
                                              active, list, nsys, b1);
  IKR_CUDA(cudaGetLastError());
  return true;
}

template <int NZ>
bool try_zf(ikr_ctx* c, int nsys, const int* d_k, const float2* b4, float2* out, int ld, const float2* psi,
            const double* shift, const float* kin, const int* active, const int* list, double* dpart) {
  if (c->N[2] != NZ) return false;
  const size_t smem = (2 * sizeof(float2) + sizeof(float)) * (size_t)c->zspan;
  if (smem > 48 * 1024) return false;
  dim3 grid((c->nc + kZC - 1) / kZC, nsys);
  k_zf_r<NZ><<<grid, kZC, smem, c->stream>>>(b4, c->nc, c->ncp, d_k, c->k_colinfo.p, c->d_colpre.p, c->zspan,
                                              out, ld, c->ld, psi, shift, kin, active, list, nsys, dpart);
  IKR_CUDA(cudaGetLastError());
  return true;
}

}  // namespace

bool z_reg_ok(ikr_ctx* c) {
  const int nz = c->N[2];
  return c->zreg_ok && (nz == 48 || nz == 32 || nz == 40 || nz == 24 || nz == 16 || nz == 12);
}
int z_reg_chunks(ikr_ctx* c) { return (c->nc + kZC - 1) / kZC; }

bool launch_z_inverse_reg(ikr_ctx* c, int nsys, const int* d_k, const float2* sphere, int ld, const int* active,
                          const int* list, float2* b1) {
  if (!z_reg_ok(c) || nsys == 0) return false;
  return try_zi<48>(c, nsys, d_k, sphere, ld, active, list, b1) ||
         try_zi<32>(c, nsys, d_k, sphere, ld, active, list, b1) ||
         try_zi<40>(c, nsys, d_k, sphere, ld, active, list, b1) ||
         try_zi<24>(c, nsys, d_k, sphere, ld, active, list, b1) ||
         try_zi<16>(c, nsys, d_k, sphere, ld, active, list, b1) ||
         try_zi<12>(c, nsys, d_k, sphere, ld, active, list, b1);
}

bool launch_z_forward_reg(ikr_ctx* c, int nsys, const int* d_k, const float2* b4, float2* out, int ld,
                          const float2* psi, const double* shift, const float* kin, const int* active,
                          const int* list, double* dpart) {
  if (!z_reg_ok(c) || nsys == 0) return false;
  return try_zf<48>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart) ||
         try_zf<32>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart) ||
         try_zf<40>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart) ||
         try_zf<24>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart) ||
         try_zf<16>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart) ||
         try_zf<12>(c, nsys, d_k, b4, out, ld, psi, shift, kin, active, list, dpart);
}

}  // namespace ikr
