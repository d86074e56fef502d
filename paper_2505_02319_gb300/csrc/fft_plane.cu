// Plane pass of the batched H_k application with compile-time line lengths.
//
// Same computation as k_plane in fft.cu (y-lines of the active x positions,
// x-lines of all rows, the product with the potential, and back), but each
// line of length N is transformed by T threads that hold E = N / T elements
// in registers:
//   1. thread t loads x[t + T q], q < E, and takes the E-point DFT in
//      registers (a recursive four-step split E = P Q with P in {4, 2, 3, 5});
//   2. it multiplies by W_N^{t k2} and writes Y_t[k2] to shared memory;
//   3. after a warp barrier, thread t takes the T-point DFTs of the k2 = t + T j
//      and writes X[k2 + E k1] (natural order).
// With n = p + P q and k = k2 + Q k1 the DFT factorises as
//   X_{k2 + Q k1} = sum_p W_P^{p k1} W_N^{p k2} sum_q x_{p + P q} W_Q^{q k2},
// the textbook Cooley-Tukey split, applied at both levels.  All index
// arithmetic is resolved at compile time; only warp barriers separate the
// steps of one line, and an x-line runs inverse FFT, potential product and
// forward FFT without leaving its warp.
#include "ops.hpp"

namespace ikr {

namespace {

// W_L^x (L = table length) for sub-transform size M, x = index in [0, M)
template <typename C, int L, int M, bool INV>
__device__ __forceinline__ C tw(const C* tab, int x) {
  C w = tab[x * (L / M)];
  if (INV) w.y = -w.y;
  return w;
}

// E = P Q: the base lengths 2..5 are one register DFT (P = E, Q = 1),
// otherwise the first factor is taken from 4, 2, 3, 5 in that order.
template <int E> struct Split {
  static constexpr bool base = (E == 2 || E == 3 || E == 4 || E == 5);
  static constexpr int P = base ? E : (E % 4 == 0) ? 4 : (E % 2 == 0) ? 2 : (E % 3 == 0) ? 3 : 5;
  static constexpr int Q = E / P;
};

// In-register DFT of length E (natural order in and out), twiddles from a
// table of W_L, E | L.
template <typename C, int E, int L, bool INV> struct RegFft {
  __device__ __forceinline__ static void run(C* v, const C* tab) {
    constexpr int P = Split<E>::P, Q = Split<E>::Q;
    if constexpr (Q == 1) {
      Dft<C, E, INV>::run(v);
    } else {
      C u[P][Q];
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int q = 0; q < Q; ++q) u[p][q] = v[p + P * q];
#pragma unroll
      for (int p = 0; p < P; ++p) RegFft<C, Q, L, INV>::run(u[p], tab);
#pragma unroll
      for (int p = 1; p < P; ++p)
#pragma unroll
        for (int k2 = 1; k2 < Q; ++k2) u[p][k2] = cmul(u[p][k2], tw<C, L, E, INV>(tab, p * k2));
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
template <typename C, int L, bool INV> struct RegFft<C, 1, L, INV> {
  __device__ __forceinline__ static void run(C*, const C*) {}
};

// Threads per line for a line length N: a power of two T with T^2 | N where
// that keeps E = N / T <= 32 registers of data (then a thread's inverse-FFT
// outputs are exactly its forward-FFT inputs, see line_fft_ivf), else the
// largest power of two dividing N (up to 8).
template <int N> struct Tpl {
  static constexpr int v = (N % 64 == 0 && N / 8 <= 32) ? 8
                         : (N % 16 == 0 && N / 4 <= 32) ? 4
                         : (N % 4 == 0 && N / 2 <= 32) ? 2
                         : (N % 8 == 0) ? 8 : (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2 : 1;
  static constexpr bool fused = (N / v) % v == 0;
};

// FFT of one line held in shared memory (element stride es) by the T lanes
// t = 0..T-1 of a group; `mask` holds the lanes of the warp taking part.
template <typename C, int N, bool INV>
__device__ __forceinline__ void line_fft(C* line, int es, const C* tab, int t, unsigned mask) {
  constexpr int T = Tpl<N>::v;
  constexpr int E = N / T;
  C v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = line[(t + T * q) * es];
  RegFft<C, E, N, INV>::run(v, tab);
  if constexpr (T == 1) {
#pragma unroll
    for (int k = 0; k < E; ++k) line[k * es] = v[k];
  } else {
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) {
      C w = tab[t * k2];
      if (INV) w.y = -w.y;
      v[k2] = cmul(v[k2], w);
    }
    __syncwarp(mask);
#pragma unroll
    for (int k2 = 0; k2 < E; ++k2) line[(k2 * T + t) * es] = v[k2];
    __syncwarp(mask);
    constexpr int J = (E + T - 1) / T;
    C w[J][T];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k2 = t + T * j;
      if (k2 < E) {
#pragma unroll
        for (int tp = 0; tp < T; ++tp) w[j][tp] = line[(k2 * T + tp) * es];
        RegFft<C, T, N, INV>::run(w[j], tab);
      }
    }
    __syncwarp(mask);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k2 = t + T * j;
      if (k2 < E) {
#pragma unroll
        for (int k1 = 0; k1 < T; ++k1) line[(k2 + E * k1) * es] = w[j][k1];
      }
    }
    __syncwarp(mask);
  }
}

// Row stride: with T lanes per x-line reading T consecutive elements, rows
// that are 4 elements (8 banks of 8-byte data) apart in bank space let 8
// lines of a warp share the minimum of 2 wavefronts; odd strides otherwise.
// Second half of a line FFT (steps 2 and 3 of the header) on values the
// thread already holds: v[q] = Y_t[k2 = q] after the E-point DFT.  Writes the
// result X in natural order to the line.
template <typename C, int N, bool INV>
__device__ __forceinline__ void line_fft_finish(C* v, C* line, int es, const C* tab, int t, unsigned mask) {
  constexpr int T = Tpl<N>::v;
  constexpr int E = N / T;
#pragma unroll
  for (int k2 = 1; k2 < E; ++k2) {
    C w = tab[t * k2];
    if (INV) w.y = -w.y;
    v[k2] = cmul(v[k2], w);
  }
  __syncwarp(mask);
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) line[(k2 * T + t) * es] = v[k2];
  __syncwarp(mask);
  constexpr int J = E / T;
  C w[J][T];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k2 = t + T * j;
#pragma unroll
    for (int tp = 0; tp < T; ++tp) w[j][tp] = line[(k2 * T + tp) * es];
    RegFft<C, T, N, INV>::run(w[j], tab);
  }
  __syncwarp(mask);
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int k1 = 0; k1 < T; ++k1) line[(t + T * j + E * k1) * es] = w[j][k1];
  __syncwarp(mask);
}

// x-line: inverse FFT (unless the line is already in real space), product
// with the potential row, forward FFT.  Requires T | E: thread t's inverse
// outputs X[t + T j + E k1] = X[t + T (j + J k1)] are its forward inputs
// x[t + T q], so the product happens in registers.
template <typename R, int N>
__device__ __forceinline__ void line_fft_ivf(C_t<R>* line, const C_t<R>* tab, int t, unsigned mask,
                                             const typename io<R>::real* __restrict__ pot_row, R sc,
                                             bool in_real) {
  using C = C_t<R>;
  constexpr int T = Tpl<N>::v;
  constexpr int E = N / T;
  constexpr int J = E / T;
  C v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = line[t + T * q];
  if (!in_real) {
    RegFft<C, E, N, true>::run(v, tab);
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) {
      C w = tab[t * k2];
      w.y = -w.y;
      v[k2] = cmul(v[k2], w);
    }
    __syncwarp(mask);
#pragma unroll
    for (int k2 = 0; k2 < E; ++k2) line[k2 * T + t] = v[k2];
    __syncwarp(mask);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      C w[T];
      const int k2 = t + T * j;
#pragma unroll
      for (int tp = 0; tp < T; ++tp) w[tp] = line[k2 * T + tp];
      RegFft<C, T, N, true>::run(w, tab);
#pragma unroll
      for (int k1 = 0; k1 < T; ++k1) v[j + J * k1] = w[k1];
    }
  }
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = cscale(v[q], to_r<R>(__ldg(pot_row + t + T * q)) * sc);
  RegFft<C, E, N, false>::run(v, tab);
  line_fft_finish<C, N, false>(v, line, 1, tab, t, mask);
}

template <typename C, int NX, int NY>
struct PlaneGeom {
  static constexpr int ldp = (NX % 16 == 0) ? NX + 4 : (NX % 2 == 0 ? NX + 1 : NX);
  static constexpr int plane = NY * ldp;
  static constexpr int bytes = plane * (int)sizeof(C);
  static constexpr int PL = (65536 / bytes) >= 3 ? 3 : ((65536 / bytes) >= 2 ? 2 : 1);
};

}  // namespace

template <typename R, int NX, int NY>
__global__ void __launch_bounds__(256) k_plane_t(const typename io<R>::cx* __restrict__ b1, int nc, int ncp,
                                                 const int* __restrict__ col_xy, const int* __restrict__ xpos,
                                                 int nxa, int Nz, const typename io<R>::cx* __restrict__ twx,
                                                 const typename io<R>::cx* __restrict__ twy,
                                                 const typename io<R>::real* __restrict__ pot,
                                                 const double* __restrict__ pot_scale,
                                                 const int* __restrict__ active, typename io<R>::cx* __restrict__ b4,
                                                 const typename io<R>::cx* __restrict__ real_in) {
  using C = C_t<R>;
  using G = PlaneGeom<C, NX, NY>;
  constexpr int ldp = G::ldp, PL = G::PL;
  constexpr int TX = Tpl<NX>::v, TY = Tpl<NY>::v;
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int iz0 = blockIdx.x * PL;
  const int npl = min(PL, Nz - iz0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + NX;
  C* planes = ty + NY;
  int* xp = reinterpret_cast<int*>(planes + PL * G::plane);
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tx[i] = to_c<C>(twx[i]);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) ty[i] = to_c<C>(twy[i]);
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  const int lane = threadIdx.x & 31;
  if (real_in) {
    for (int e = threadIdx.x; e < npl * NY * NX; e += blockDim.x) {
      const int p = e / (NY * NX), r = e - p * (NY * NX);
      const int iy = r / NX, ix = r - iy * NX;
      planes[p * G::plane + iy * ldp + ix] = to_c<C>(real_in[((size_t)s * Nz + iz0 + p) * NY * NX + r]);
    }
    __syncthreads();
  } else {
    for (int i = threadIdx.x; i < npl * G::plane; i += blockDim.x) planes[i] = mk<C>(0, 0);
    __syncthreads();
    for (int e = threadIdx.x; e < npl * nc; e += blockDim.x) {
      const int p = e / nc, col = e - p * nc;
      planes[p * G::plane + col_xy[2 * col + 1] * ldp + col_xy[2 * col]] =
          to_c<C>(b1[((size_t)s * Nz + iz0 + p) * ncp + col]);
    }
    __syncthreads();
    // inverse y-lines of the active x positions
    {
      const int slots = blockDim.x / TY, slot = threadIdx.x / TY, t = threadIdx.x % TY;
      const int items = npl * nxa;
      const int rounds = (items + slots - 1) / slots;
      for (int r = 0; r < rounds; ++r) {
        const int it = r * slots + slot;
        const bool ok = it < items;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int p = it / nxa, l = it - p * nxa;
          line_fft<C, NY, true>(planes + p * G::plane + xp[l], ldp, ty, t, mask);
        }
      }
    }
    __syncthreads();
  }
  // x-lines: inverse FFT, potential product, forward FFT, all within the line's lanes
  {
    const R sc = pot_scale ? to_r<R>(*pot_scale) : R(1);
    const int slots = blockDim.x / TX, slot = threadIdx.x / TX, t = threadIdx.x % TX;
    const int items = npl * NY;
    const int rounds = (items + slots - 1) / slots;
    for (int r = 0; r < rounds; ++r) {
      const int it = r * slots + slot;
      const bool ok = it < items;
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int p = it / NY, iy = it - p * NY;
        C* line = planes + p * G::plane + iy * ldp;
        const typename io<R>::real* pp = pot + ((size_t)(iz0 + p) * NY + iy) * NX;
        if constexpr (Tpl<NX>::fused) {
          line_fft_ivf<R, NX>(line, tx, t, mask, pp, sc, real_in != nullptr);
        } else {
          if (!real_in) line_fft<C, NX, true>(line, 1, tx, t, mask);   // real_in: already in real space
#pragma unroll
          for (int ix = t; ix < NX; ix += TX) line[ix] = cscale(line[ix], to_r<R>(pp[ix]) * sc);
          __syncwarp(mask);
          line_fft<C, NX, false>(line, 1, tx, t, mask);
        }
      }
    }
  }
  __syncthreads();
  // forward y-lines of the active x positions
  {
    const int slots = blockDim.x / TY, slot = threadIdx.x / TY, t = threadIdx.x % TY;
    const int items = npl * nxa;
    const int rounds = (items + slots - 1) / slots;
    for (int r = 0; r < rounds; ++r) {
      const int it = r * slots + slot;
      const bool ok = it < items;
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int p = it / nxa, l = it - p * nxa;
        line_fft<C, NY, false>(planes + p * G::plane + xp[l], ldp, ty, t, mask);
      }
    }
  }
  __syncthreads();
  (void)lane;
  for (int e = threadIdx.x; e < npl * nc; e += blockDim.x) {
    const int p = e / nc, col = e - p * nc;
    b4[((size_t)s * Nz + iz0 + p) * ncp + col] =
        from_c(planes[p * G::plane + col_xy[2 * col + 1] * ldp + col_xy[2 * col]]);
  }
}

// ---------------------------------------------------------------------------
// FP64-accurate plane pass in double-float with a swizzled plane (the pass the
// mixed path runs for its right-hand sides and defect-correction residuals).
// Same result as k_plane_t<dfloat>, organised for the 48 x 48 planes:
//   - y-lines take 8 lanes (E = 6 elements each), so the 20 or so active
//     columns keep 160 of the 192 threads busy and take about half the time of
//     4-lane lines; x-lines keep 4 lanes (E = 12, inverse FFT, potential,
//     forward FFT in registers);
//   - element (y, x) of the plane sits at y NX + (x ^ r(y) ^ 2 bit3(x)) with
//     r(y) = G[y mod 8] ^ H[y / 8], G = (0 1 2 3 5 4 7 6), H = (0 1 2 4 5 6),
//     and the two x-lines of a quarter-warp are rows 8b + j and 8b + j + 4:
//     with 16-byte elements every load and store of every step (both line
//     directions, the transposes included) is served by one 128-byte
//     wavefront per quarter-warp (checked for all access patterns on the
//     host when the layout was chosen), against 2-way conflicts of the padded
//     row-major layout.
// The swizzle only permutes positions within aligned groups of 8 elements of
// a row, so a row stays a row: NX % 16 == 0 (4-lane x-lines with T | E) and
// NY % 8 == 0, NY <= 48 (the H table).

__device__ __forceinline__ int sw_row(int y) {
  return (int)(((0x67453210u >> ((y & 7) * 4)) ^ (0x654210u >> ((y >> 3) * 4))) & 7u);
}
template <int NX>
__device__ __forceinline__ int sw_at(int y, int x, int ry) {
  return y * NX + (x ^ ry ^ (((x >> 3) & 1) << 1));
}

// Addresses.  The swizzle changes only the low 3 bits of x, so every access
// pattern is one per-lane value XOR a compile-time constant:
//   y-line of column x, cx = x ^ 2 bit3(x):
//     y = t + 8 q:  y NX + ((cx ^ G[t]) ^ H[q])
//     y = 8 t + p:  y NX + ((cx ^ H[t]) ^ G[p])
//   x-line of row y, r = r(y), lanes t < 4:
//     x = t + 4 k:           y NX + 8 (k >> 1) + ((t ^ r) ^ (4 (k & 1) ^ 2 ((k >> 1) & 1)))
//     x = 4 t + 16 j + p:    y NX + 8 (t >> 1) + 16 j + (m ^ p),  m = 4 (t & 1) ^ r ^ 2 ((t >> 1) & 1)
__device__ __forceinline__ int sw_g(int i) { return (int)((0x67453210u >> (4 * i)) & 7u); }
__device__ __forceinline__ int sw_h(int i) { return (int)((0x654210u >> (4 * i)) & 7u); }

// y-line of column x: 8 lanes, lane t holds x[t + 8 q]; then the 8-point DFTs of
// k2 = t < E (E <= 8) across the lanes; natural order out.  Forward transform;
// cj = true gives the inverse as conj(FFT(conj x)) (conjugated load and store).
template <int NX, int NY>
__device__ __forceinline__ void yline_sw(dfloat2* P, int x, const dfloat2* tab, int t, unsigned mask, bool cj) {
  using C = dfloat2;
  constexpr int T = 8, E = NY / T;
  static_assert(E <= T, "one 8-point DFT per lane");
  const int cx = x ^ (((x >> 3) & 1) << 1);
  const int a = cx ^ sw_g(t);                 // rows y = t + 8 q
  C* col = P + t * NX;
  C v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    v[q] = col[8 * q * NX + (a ^ ((0x654210 >> (4 * q)) & 7))];
    if (cj) v[q].y = -v[q].y;
  }
  RegFft<C, E, NY, false>::run(v, tab);
#pragma unroll
  for (int k2 = 1; k2 < E; ++k2) v[k2] = cmul(v[k2], tab[t * k2]);
  __syncwarp(mask);
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) col[8 * k2 * NX + (a ^ ((0x654210 >> (4 * k2)) & 7))] = v[k2];
  __syncwarp(mask);
  C w[T];
  if (t < E) {
    const int b = cx ^ sw_h(t);               // rows y = 8 t + p
    const C* blk = P + 8 * t * NX;
#pragma unroll
    for (int tp = 0; tp < T; ++tp) w[tp] = blk[tp * NX + (b ^ ((0x67453210 >> (4 * tp)) & 7))];
    RegFft<C, T, NY, false>::run(w, tab);
  }
  __syncwarp(mask);
  if (t < E) {
#pragma unroll
    for (int k1 = 0; k1 < T; ++k1) {
      const int y = t + E * k1;
      C o = w[k1];
      if (cj) o.y = -o.y;
      P[y * NX + (cx ^ sw_row(y))] = o;
    }
  }
  __syncwarp(mask);
}

// x-line of row y: 4 lanes; two passes of one forward pipeline (E-point DFT,
// twiddles, transpose through the row, T-point DFTs): pass 0 transforms the
// conjugated row (the inverse FFT, conjugated back in registers) unless the row
// is already in real space, pass 1 the product with the potential row, whose
// result is written back in natural order
template <int NX>
__device__ __forceinline__ void xline_ivf_sw(dfloat2* P, int y, const dfloat2* tab, int t, unsigned mask,
                                             const double* __restrict__ pot_row, dfloat sc, bool in_real) {
  using C = dfloat2;
  constexpr int T = 4, E = NX / T, J = E / T;
  static_assert(E % T == 0, "x-lines need T | E");
  const int ry = sw_row(y);
  C* row = P + y * NX;
  const int u = t ^ ry;                                               // x = t + 4 k
  C* rowt = row + 8 * (t >> 1);                                       // x = 4 t + 16 j + p
  const int m = (4 * (t & 1)) ^ ry ^ (2 * ((t >> 1) & 1));
#define IKR_SW_LIN(k) (8 * ((k) >> 1) + (u ^ ((4 * ((k) & 1)) ^ (2 * (((k) >> 1) & 1)))))
  C v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    v[q] = row[IKR_SW_LIN(q)];
    if (!in_real) v[q].y = -v[q].y;
  }
  C w[J][T];
#pragma unroll 1
  for (int pass = in_real ? 1 : 0; pass < 2; ++pass) {
    if (pass == 1) {
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const dfloat p = to_r<dfloat>(__ldg(pot_row + t + T * q)) * sc;
        C a = v[q];
        if (!in_real) a.y = -a.y;                   // conj of the inverse pass's output
        v[q] = cscale(a, p);
      }
    }
    RegFft<C, E, NX, false>::run(v, tab);
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) v[k2] = cmul(v[k2], tab[t * k2]);
    __syncwarp(mask);
#pragma unroll
    for (int k2 = 0; k2 < E; ++k2) row[IKR_SW_LIN(k2)] = v[k2];
    __syncwarp(mask);
#pragma unroll
    for (int j = 0; j < J; ++j) {
#pragma unroll
      for (int tp = 0; tp < T; ++tp) w[j][tp] = rowt[16 * j + (m ^ tp)];
      RegFft<C, T, NX, false>::run(w[j], tab);
    }
    // the outputs X[t + T j + E k1] = X[t + T (j + J k1)] are the next pass's inputs
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int k1 = 0; k1 < T; ++k1) v[j + J * k1] = w[j][k1];
  }
  __syncwarp(mask);
#pragma unroll
  for (int q = 0; q < E; ++q) row[IKR_SW_LIN(q)] = v[q];
  __syncwarp(mask);
#undef IKR_SW_LIN
}

template <int NX, int NY>
__global__ void __launch_bounds__(192, 3) k_plane_sw(const double2* __restrict__ b1, int nc, int ncp,
                                                  const int* __restrict__ col_xy, const int* __restrict__ xpos,
                                                  int nxa, int Nz, const double2* __restrict__ twx,
                                                  const double2* __restrict__ twy, const double* __restrict__ pot,
                                                  const double* __restrict__ pot_scale,
                                                  const int* __restrict__ active, double2* __restrict__ b4,
                                                  const double2* __restrict__ real_in) {
  static_assert(NX % 16 == 0 && NY % 8 == 0 && NY <= 48, "swizzled plane shape");
  using C = dfloat2;
  const int iz = blockIdx.x, s = blockIdx.y;
  if (active && !active[s]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + NX;
  C* P = ty + NY;
  int* xp = reinterpret_cast<int*>(P + NX * NY);
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tx[i] = to_c<C>(twx[i]);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) ty[i] = to_c<C>(twy[i]);
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  const size_t plane = (size_t)s * Nz + iz;
  if (real_in) {
    for (int e = threadIdx.x; e < NY * NX; e += blockDim.x) {
      const int y = e / NX, x = e - y * NX;
      P[sw_at<NX>(y, x, sw_row(y))] = to_c<C>(real_in[plane * NY * NX + e]);
    }
  } else {
    for (int i = threadIdx.x; i < NX * NY; i += blockDim.x) P[i] = mk<C>(dfloat(0), dfloat(0));
    __syncthreads();
    for (int col = threadIdx.x; col < nc; col += blockDim.x) {
      const int x = col_xy[2 * col], y = col_xy[2 * col + 1];
      P[sw_at<NX>(y, x, sw_row(y))] = to_c<C>(b1[plane * ncp + col]);
    }
  }
  __syncthreads();
  const dfloat sc = pot_scale ? to_r<dfloat>(*pot_scale) : dfloat(1);
  // phase 0: inverse y-lines (not for real-space input), 1: x-lines, 2: forward y-lines;
  // one y-line and one x-line code site (the transforms are unrolled once each)
#pragma unroll 1
  for (int ph = real_in ? 1 : 0; ph < 3; ++ph) {
    if (ph != 1) {
      const int slots = blockDim.x / 8, slot = threadIdx.x / 8, t = threadIdx.x % 8;
      const int rounds = (nxa + slots - 1) / slots;
      for (int r = 0; r < rounds; ++r) {
        const int l = r * slots + slot;
        const bool ok = l < nxa;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) yline_sw<NX, NY>(P, xp[l], ty, t, mask, ph == 0);
      }
    } else {
      const int slots = blockDim.x / 4, slot = threadIdx.x / 4, t = threadIdx.x % 4;
      const int rounds = (NY + slots - 1) / slots;
      for (int r = 0; r < rounds; ++r) {
        const int it = r * slots + slot;
        const bool ok = it < NY;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int y = 8 * (it >> 3) + ((it & 7) >> 1) + 4 * (it & 1);   // quarter-warp rows y, y + 4
          xline_ivf_sw<NX>(P, y, tx, t, mask, pot + ((size_t)iz * NY + y) * NX, sc, real_in != nullptr);
        }
      }
    }
    __syncthreads();
  }
  for (int col = threadIdx.x; col < nc; col += blockDim.x) {
    const int x = col_xy[2 * col], y = col_xy[2 * col + 1];
    b4[plane * ncp + col] = from_c(P[sw_at<NX>(y, x, sw_row(y))]);
  }
}

// Real-space planes of the sphere vectors (same result as k_synth_planes in
// fft.cu, which it replaces for the supported grids): the z-transformed
// columns b1 scattered into a plane, inverse y-lines of the active x
// positions, inverse x-lines, written out.  One plane in shared memory, the
// lines transformed in place (the generic kernel needs two plane buffers).
template <typename R, int NX, int NY>
__global__ void __launch_bounds__(256) k_synth_t(const typename io<R>::cx* __restrict__ b1, int nc, int ncp,
                                                 const int* __restrict__ col_xy, const int* __restrict__ xpos,
                                                 int nxa, int Nz, const typename io<R>::cx* __restrict__ twx,
                                                 const typename io<R>::cx* __restrict__ twy,
                                                 typename io<R>::cx* __restrict__ out) {
  using C = C_t<R>;
  using G = PlaneGeom<C, NX, NY>;
  constexpr int ldp = G::ldp;
  constexpr int TX = Tpl<NX>::v, TY = Tpl<NY>::v;
  const int iz = blockIdx.x, s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + NX;
  C* plane = ty + NY;
  int* xp = reinterpret_cast<int*>(plane + G::plane);
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tx[i] = to_c<C>(twx[i]);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) ty[i] = to_c<C>(twy[i]);
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  for (int i = threadIdx.x; i < G::plane; i += blockDim.x) plane[i] = mk<C>(R(0), R(0));
  __syncthreads();
  const typename io<R>::cx* src = b1 + ((size_t)s * Nz + iz) * ncp;
  for (int col = threadIdx.x; col < nc; col += blockDim.x)
    plane[col_xy[2 * col + 1] * ldp + col_xy[2 * col]] = to_c<C>(src[col]);
  __syncthreads();
  {
    const int slots = blockDim.x / TY, slot = threadIdx.x / TY, t = threadIdx.x % TY;
    const int rounds = (nxa + slots - 1) / slots;
    for (int r = 0; r < rounds; ++r) {
      const int l = r * slots + slot;
      const bool ok = l < nxa;
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) line_fft<C, NY, true>(plane + xp[l], ldp, ty, t, mask);
    }
  }
  __syncthreads();
  {
    const int slots = blockDim.x / TX, slot = threadIdx.x / TX, t = threadIdx.x % TX;
    const int rounds = (NY + slots - 1) / slots;
    for (int r = 0; r < rounds; ++r) {
      const int iy = r * slots + slot;
      const bool ok = iy < NY;
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) line_fft<C, NX, true>(plane + iy * ldp, 1, tx, t, mask);
    }
  }
  __syncthreads();
  typename io<R>::cx* dst = out + ((size_t)s * Nz + iz) * NY * NX;
  for (int e = threadIdx.x; e < NY * NX; e += blockDim.x) {
    const int iy = e / NX, ix = e - iy * NX;
    dst[e] = from_c(plane[iy * ldp + ix]);
  }
}

// Density accumulation with compile-time line lengths (same result as
// k_density in fft.cu, which it replaces for the supported grids):
//   part[g][iz][iy][ix] = sum_{s in group g} a_s Re(conj(psi_s) dpsi_s) + b_s |psi_s|^2,
// psi_s the cached real-space orbital planes, dpsi_s synthesised here from the
// z-transformed responses b1d (y-lines of the active x positions, then x-lines),
// PL systems at a time; accumulation in FP64 registers.
template <typename R, int NX, int NY>
__global__ void __launch_bounds__(256) k_density_t(const typename io<R>::cx* __restrict__ b1d, int nc, int ncp,
                                                   const int* __restrict__ col_xy, const int* __restrict__ xpos,
                                                   int nxa, int Nz, const typename io<R>::cx* __restrict__ twx,
                                                   const typename io<R>::cx* __restrict__ twy,
                                                   const typename io<R>::cx* __restrict__ psir,
                                                   const double* __restrict__ coef_a,
                                                   const double* __restrict__ coef_b, int nsys, int ngroups,
                                                   double* __restrict__ part) {
  using C = C_t<R>;
  using G = PlaneGeom<C, NX, NY>;
  constexpr int ldp = G::ldp, PL = G::PL;
  constexpr int TX = Tpl<NX>::v, TY = Tpl<NY>::v;
  constexpr int NE = (NX * NY + 255) / 256;
  const int iz = blockIdx.x, g = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + NX;
  C* planes = ty + NY;
  int* xp = reinterpret_cast<int*>(planes + PL * G::plane);
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tx[i] = to_c<C>(twx[i]);
  for (int i = threadIdx.x; i < NY; i += blockDim.x) ty[i] = to_c<C>(twy[i]);
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  // double-float and FP32: the sums in double-float on the FP32 pipe (FP64 runs at a small
  // fraction of the FP32 rate); FP64 otherwise.  Double-float reads the orbitals from their
  // (hi, lo) copy and forms the products in double-float; FP32 forms each system's
  // contribution in FP32 (its inputs carry FP32 rounding already) and adds it exactly.
  using A = typename std::conditional<std::is_same<R, double>::value, double, dfloat>::type;
  A acc[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) acc[i] = A(0.0);
  const int s0 = (int)((long long)g * nsys / ngroups), s1 = (int)((long long)(g + 1) * nsys / ngroups);
  for (int sb = s0; sb < s1; sb += PL) {
    const int npl = min(PL, s1 - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < npl * G::plane; i += blockDim.x) planes[i] = mk<C>(0, 0);
    __syncthreads();
    for (int e = threadIdx.x; e < npl * nc; e += blockDim.x) {
      const int p = e / nc, col = e - p * nc;
      planes[p * G::plane + col_xy[2 * col + 1] * ldp + col_xy[2 * col]] =
          to_c<C>(b1d[((size_t)(sb + p) * Nz + iz) * ncp + col]);
    }
    __syncthreads();
    {
      const int slots = blockDim.x / TY, slot = threadIdx.x / TY, t = threadIdx.x % TY;
      const int items = npl * nxa;
      const int rounds = (items + slots - 1) / slots;
      for (int r = 0; r < rounds; ++r) {
        const int it = r * slots + slot;
        const bool ok = it < items;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int p = it / nxa, l = it - p * nxa;
          line_fft<C, NY, true>(planes + p * G::plane + xp[l], ldp, ty, t, mask);
        }
      }
    }
    __syncthreads();
    {
      const int slots = blockDim.x / TX, slot = threadIdx.x / TX, t = threadIdx.x % TX;
      const int items = npl * NY;
      const int rounds = (items + slots - 1) / slots;
      for (int r = 0; r < rounds; ++r) {
        const int it = r * slots + slot;
        const bool ok = it < items;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int p = it / NY, iy = it - p * NY;
          line_fft<C, NX, true>(planes + p * G::plane + iy * ldp, 1, tx, t, mask);
        }
      }
    }
    __syncthreads();
    for (int p = 0; p < npl; ++p) {
      const int s = sb + p;
      if constexpr (std::is_same<R, dfloat>::value) {
        const dfloat a = to_r<dfloat>(coef_a[s]), b = to_r<dfloat>(coef_b[s]);
        const float4* ps = reinterpret_cast<const float4*>(psir) + ((size_t)s * Nz + iz) * NX * NY;
#pragma unroll
        for (int i = 0; i < NE; ++i) {
          const int e = threadIdx.x + 256 * i;
          if (e < NX * NY) {
            const int iy = e / NX, ix = e - iy * NX;
            const dfloat2 d = planes[p * G::plane + iy * ldp + ix];
            const float4 q = ps[e];
            const dfloat px(q.x, q.y), py(q.z, q.w);
            acc[i] += a * (px * d.x + py * d.y) + b * (px * px + py * py);
          }
        }
      } else if constexpr (std::is_same<R, float>::value) {
        const float a = (float)coef_a[s], b = (float)coef_b[s];
        const float2* ps = psir + ((size_t)s * Nz + iz) * NX * NY;
#pragma unroll
        for (int i = 0; i < NE; ++i) {
          const int e = threadIdx.x + 256 * i;
          if (e < NX * NY) {
            const int iy = e / NX, ix = e - iy * NX;
            const float2 d = planes[p * G::plane + iy * ldp + ix];
            const float2 q = ps[e];
            const float t = fmaf(a, fmaf(q.x, d.x, q.y * d.y), b * fmaf(q.x, q.x, q.y * q.y));
            acc[i] += dfloat(t, 0.f);
          }
        }
      } else {
        const double a = coef_a[s], b = coef_b[s];
        const typename io<R>::cx* ps = psir + ((size_t)s * Nz + iz) * NX * NY;
#pragma unroll
        for (int i = 0; i < NE; ++i) {
          const int e = threadIdx.x + 256 * i;
          if (e < NX * NY) {
            const int iy = e / NX, ix = e - iy * NX;
            const auto d = from_c(planes[p * G::plane + iy * ldp + ix]);
            const typename io<R>::cx q = ps[e];
            const double px = (double)q.x, py = (double)q.y;
            acc[i] += a * (px * (double)d.x + py * (double)d.y) + b * (px * px + py * py);
          }
        }
      }
    }
  }
  double* dst = part + ((size_t)g * Nz + iz) * NX * NY;
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int e = threadIdx.x + 256 * i;
    if (e < NX * NY) dst[e] = to_d(acc[i]);
  }
}

namespace {

template <typename R> const typename io<R>::cx* twp(ikr_ctx* c, int axis);
template <> const double2* twp<double>(ikr_ctx* c, int axis) { return c->d_tw[axis].p; }
template <> const double2* twp<dfloat>(ikr_ctx* c, int axis) { return c->d_tw[axis].p; }
template <> const float2* twp<float>(ikr_ctx* c, int axis) { return c->d_tw32[axis].p; }

template <typename R, int NX, int NY>
bool try_launch(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, const typename io<R>::real* pot,
                const double* pot_scale, const int* active, typename io<R>::cx* b4,
                const typename io<R>::cx* real_in) {
  if (c->N[0] != NX || c->N[1] != NY) return false;
  using G = PlaneGeom<C_t<R>, NX, NY>;
  const size_t smem = sizeof(C_t<R>) * (NX + NY + (size_t)G::PL * G::plane) + sizeof(int) * c->nxa;
  if (smem > 227 * 1024) return false;
  IKR_CUDA(cudaFuncSetAttribute(k_plane_t<R, NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int Nz = c->N[2];
  dim3 grid((Nz + G::PL - 1) / G::PL, nsys);
  // double-float: 48 line groups of 4 lanes, so the x-lines of a 48-row plane
  // take one round and three blocks fit an SM
  const int nth = std::is_same<R, dfloat>::value ? 192 : 256;
  k_plane_t<R, NX, NY><<<grid, nth, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa, Nz,
                                                        twp<R>(c, 0), twp<R>(c, 1), pot, pot_scale, active, b4,
                                                        real_in);
  IKR_CUDA(cudaGetLastError());
  return true;
}

template <typename R, int NX, int NY>
bool try_density(ikr_ctx* c, int nsys, const typename io<R>::cx* b1d, const typename io<R>::cx* psir,
                 const double* ca, const double* cb, int* ngroups_out) {
  if (c->N[0] != NX || c->N[1] != NY) return false;
  using G = PlaneGeom<C_t<R>, NX, NY>;
  const size_t smem = sizeof(C_t<R>) * (NX + NY + (size_t)G::PL * G::plane) + sizeof(int) * c->nxa;
  if (smem > 227 * 1024) return false;
  IKR_CUDA(cudaFuncSetAttribute(k_density_t<R, NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  IKR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_density_t<R, NX, NY>, 256, smem));
  const int ngroups = density_groups(c, nsys, per_sm);
  c->ws.dens_part.reserve((size_t)ngroups * c->Ng);
  double* part = c->ws.dens_part.p;
  *ngroups_out = ngroups;
  dim3 grid(c->N[2], ngroups);
  k_density_t<R, NX, NY><<<grid, 256, smem, c->stream>>>(b1d, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                                          c->N[2], twp<R>(c, 0), twp<R>(c, 1), psir, ca, cb,
                                                          nsys, ngroups, part);
  IKR_CUDA(cudaGetLastError());
  return true;
}

template <typename R, int NX, int NY>
bool try_synth(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, typename io<R>::cx* out) {
  if (c->N[0] != NX || c->N[1] != NY) return false;
  using G = PlaneGeom<C_t<R>, NX, NY>;
  const size_t smem = sizeof(C_t<R>) * (NX + NY + (size_t)G::plane) + sizeof(int) * c->nxa;
  if (smem > 227 * 1024) return false;
  IKR_CUDA(cudaFuncSetAttribute(k_synth_t<R, NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(c->N[2], nsys);
  k_synth_t<R, NX, NY><<<grid, 256, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                                        c->N[2], twp<R>(c, 0), twp<R>(c, 1), out);
  IKR_CUDA(cudaGetLastError());
  return true;
}

}  // namespace

template <typename R>
bool launch_synth_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, typename io<R>::cx* out) {
  return try_synth<R, 48, 48>(c, nsys, b1, out) || try_synth<R, 32, 32>(c, nsys, b1, out) ||
         try_synth<R, 40, 40>(c, nsys, b1, out) || try_synth<R, 96, 96>(c, nsys, b1, out) ||
         try_synth<R, 12, 12>(c, nsys, b1, out) || try_synth<R, 10, 12>(c, nsys, b1, out) ||
         try_synth<R, 24, 24>(c, nsys, b1, out);
}
template bool launch_synth_fast<float>(ikr_ctx*, int, const float2*, float2*);
template bool launch_synth_fast<double>(ikr_ctx*, int, const double2*, double2*);

template <typename R>
bool launch_density_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1d, const typename io<R>::cx* psir,
                         const double* ca, const double* cb, int* ngroups) {
  return try_density<R, 48, 48>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 32, 32>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 40, 40>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 96, 96>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 12, 12>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 10, 12>(c, nsys, b1d, psir, ca, cb, ngroups) ||
         try_density<R, 24, 24>(c, nsys, b1d, psir, ca, cb, ngroups);
}
template bool launch_density_fast<float>(ikr_ctx*, int, const float2*, const float2*, const double*,
                                         const double*, int*);
template bool launch_density_fast<double>(ikr_ctx*, int, const double2*, const double2*, const double*,
                                          const double*, int*);
template bool launch_density_fast<dfloat>(ikr_ctx*, int, const double2*, const double2*, const double*,
                                          const double*, int*);

// The swizzled double-float plane pass for 48 x 48 planes; false: another kernel.
bool launch_plane_sw(ikr_ctx* c, int nsys, const double2* b1, const double* pot, const double* pot_scale,
                     const int* active, double2* b4, const double2* real_in) {
  if (!c->plane_sw || c->N[0] != 48 || c->N[1] != 48) return false;
  constexpr int NX = 48, NY = 48;
  const size_t smem = sizeof(dfloat2) * (NX + NY + (size_t)NX * NY) + sizeof(int) * c->nxa;
  if (smem > 227 * 1024) return false;
  IKR_CUDA(cudaFuncSetAttribute(k_plane_sw<NX, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(c->N[2], nsys);
  k_plane_sw<NX, NY><<<grid, 192, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                                     c->N[2], c->d_tw[0].p, c->d_tw[1].p, pot, pot_scale, active,
                                                     b4, real_in);
  IKR_CUDA(cudaGetLastError());
  return true;
}

// Compile-time plane shapes of the supported grids; false: use the generic kernel.
template <typename R>
bool launch_plane_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, const typename io<R>::real* pot,
                       const double* pot_scale, const int* active, typename io<R>::cx* b4,
                       const typename io<R>::cx* real_in) {
  return try_launch<R, 48, 48>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 32, 32>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 40, 40>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 96, 96>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 12, 12>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 10, 12>(c, nsys, b1, pot, pot_scale, active, b4, real_in) ||
         try_launch<R, 24, 24>(c, nsys, b1, pot, pot_scale, active, b4, real_in);
}

template bool launch_plane_fast<double>(ikr_ctx*, int, const double2*, const double*, const double*, const int*,
                                        double2*, const double2*);
template bool launch_plane_fast<dfloat>(ikr_ctx*, int, const double2*, const double*, const double*, const int*,
                                        double2*, const double2*);
template bool launch_plane_fast<float>(ikr_ctx*, int, const float2*, const float*, const double*, const int*,
                                       float2*, const float2*);

}  // namespace ikr
