// Common device types and the shared-memory line FFT used by every transform
// of the library (F, F^-1 of eq. fft_ifft and the full-grid transforms of the
// Hartree and Kerker kernels).
//
// The line FFT is a mixed-radix (2, 3, 4, 5) Stockham autosort transform:
// at a stage of radix r with Ns outputs already combined, butterfly j of a
// line of length n reads the r inputs j + i n/r, multiplies input i by the
// twiddle e^{-+2 pi i (j mod Ns) i / (Ns r)}, takes the length-r DFT and
// writes the results to (j / Ns) Ns r + (j mod Ns) + i Ns, so that the output
// comes out in natural order after the last stage (Govindaraju et al., SC'08).
// Stages alternate between two shared-memory buffers.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace ikr {

// Double-float ("df64") real: an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32 units.
// Arithmetic from the error-free transformations: TwoSum (Knuth) for a + b,
// the FMA residual a*b - fl(a*b) for products (Dekker's product with a fused
// multiply-add), renormalised by a fast two-sum; additions drop the O(2^-48)
// second-order terms, so each operation has an error of a few 2^-48 relative
// to its operands.  Used where the mixed-precision path needs FP64 accuracy.
struct dfloat {
  float hi, lo;
  __host__ __device__ constexpr dfloat() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dfloat(int i) : hi((float)i), lo(0.f) {}
};

__device__ __forceinline__ dfloat df_fast2sum(float a, float b) {
  const float s = a + b;
  return dfloat(s, b - (s - a));
}
__device__ __forceinline__ dfloat df_2sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfloat(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = df_2sum(a.hi, b.hi);
  return df_fast2sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast2sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfloat df_from_double(double d) {
  const float h = __double2float_rn(d);
  return dfloat(h, __double2float_rn(d - (double)h));
}

// 16-byte aligned, so that a complex element moves as one 128-bit access
// (four 32-bit ones otherwise, which collide in shared memory: 4-way bank
// conflicts on the line layouts of the plane pass)
struct __align__(16) dfloat2 {
  dfloat x, y;
};

template <typename R> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<dfloat> { using type = dfloat2; };
template <typename R> using C_t = typename cplx<R>::type;

// conversions between the storage types and the arithmetic types
template <typename C> __device__ __forceinline__ C to_c(double2 v);
template <> __device__ __forceinline__ double2 to_c<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ dfloat2 to_c<dfloat2>(double2 v) {
  dfloat2 r;
  r.x = df_from_double(v.x);
  r.y = df_from_double(v.y);
  return r;
}
template <typename C> __device__ __forceinline__ C to_c(float2 v);
template <> __device__ __forceinline__ float2 to_c<float2>(float2 v) { return v; }
__device__ __forceinline__ double2 from_c(double2 v) { return v; }
__device__ __forceinline__ float2 from_c(float2 v) { return v; }
__device__ __forceinline__ double2 from_c(dfloat2 v) { return make_double2(df_to_double(v.x), df_to_double(v.y)); }
template <typename R> __device__ __forceinline__ R to_r(double v) { return (R)v; }
template <> __device__ __forceinline__ dfloat to_r<dfloat>(double v) { return df_from_double(v); }
template <typename R> __device__ __forceinline__ R to_r(float v) { return (R)v; }
template <> __device__ __forceinline__ dfloat to_r<dfloat>(float v) { return dfloat(v, 0.f); }

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(dfloat v) { return df_to_double(v); }

// storage type of the arithmetic type R (what global buffers hold)
template <typename R> struct io;
template <> struct io<float> { using real = float; using cx = float2; };
template <> struct io<double> { using real = double; using cx = double2; };
template <> struct io<dfloat> { using real = double; using cx = double2; };

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }

// Double-float complex arithmetic of the FFT butterflies, without the final
// renormalisation: a sum keeps TwoSum(a.hi, b.hi) exact and adds the low parts
// (8 operations instead of 11), a product keeps the FMA residual (4 instead of
// 7).  The low part then may exceed ulp(hi)/2 by the few roundings of the
// transform's O(log N) levels, a relative error of order 1e-13 after a whole
// plane pass; hi + lo stays the value, and every conversion to double sums
// both.  Long accumulations use the normalised scalar operators above.
__device__ __forceinline__ dfloat df_add_lazy(dfloat a, dfloat b) {
  const dfloat s = df_2sum(a.hi, b.hi);
  return dfloat(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfloat df_mul_lazy(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dfloat(p, e);
}
template <> __device__ __forceinline__ dfloat2 cadd<dfloat2>(dfloat2 a, dfloat2 b) {
  return dfloat2{df_add_lazy(a.x, b.x), df_add_lazy(a.y, b.y)};
}
template <> __device__ __forceinline__ dfloat2 csub<dfloat2>(dfloat2 a, dfloat2 b) {
  return dfloat2{df_add_lazy(a.x, -b.x), df_add_lazy(a.y, -b.y)};
}
template <> __device__ __forceinline__ dfloat2 cmul<dfloat2>(dfloat2 a, dfloat2 b) {
  return dfloat2{df_add_lazy(df_mul_lazy(a.x, b.x), -df_mul_lazy(a.y, b.y)),
                 df_add_lazy(df_mul_lazy(a.x, b.y), df_mul_lazy(a.y, b.x))};
}
template <> __device__ __forceinline__ dfloat2 cscale<dfloat2>(dfloat2 a, dfloat s) {
  return dfloat2{df_mul_lazy(a.x, s), df_mul_lazy(a.y, s)};
}
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C rot(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

constexpr int kMaxStages = 12;

// Factorisation of a line length into radices (4 first, then 2, 3, 5).
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
};

// ---- length-r DFTs in registers, X_k = sum_j x_j e^{-+2 pi i jk/r} ----------

template <typename C, int RAD, bool INV> struct Dft;

template <typename C, bool INV> struct Dft<C, 2, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C, bool INV> struct Dft<C, 4, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C s13 = cadd(v[1], v[3]), d13 = rot<C, INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <typename C, bool INV> struct Dft<C, 3, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R h = R(0.86602540378443864676);   // sin(2 pi/3) = sqrt(3)/2
    C t = cadd(v[1], v[2]);
    C m = cadd(v[0], cscale(t, R(-0.5)));
    C d = rot<C, INV>(cscale(csub(v[1], v[2]), h));   // -+ i sqrt(3)/2 (x1 - x2)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, d);
    v[2] = csub(m, d);
  }
};

template <typename C, bool INV> struct Dft<C, 5, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = decltype(C::x);
    const R c1 = R(0.30901699437494742410);    // cos(2 pi/5)
    const R c2 = R(-0.80901699437494742410);   // cos(4 pi/5)
    const R s1 = R(0.95105651629515357212);    // sin(2 pi/5)
    const R s2 = R(0.58778525229247312917);    // sin(4 pi/5)
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
    C a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
    C b1 = rot<C, INV>(cadd(cscale(t3, s1), cscale(t4, s2)));
    C b2 = rot<C, INV>(csub(cscale(t3, s2), cscale(t4, s1)));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

// One Stockham stage of radix RAD on `nlines` lines.  Element e of line l is
// at  base(l) + e * estride,  base(l) = btab ? btab[l] : l * lstride.
// tw[t] = e^{-2 pi i t / n} (conjugated on the fly for the inverse).
template <typename C, int RAD, bool INV>
__device__ __forceinline__ void fft_stage(const C* __restrict__ in, C* __restrict__ out, int n, int Ns,
                                          int nlines, int lstride, const int* __restrict__ btab,
                                          int estride, const C* __restrict__ tw) {
  const int nb = n / RAD;
  const int total = nlines * nb;
  const int twmul = n / (Ns * RAD);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int l = b / nb;
    const int j = b - l * nb;
    const int base = btab ? btab[l] : l * lstride;
    C v[RAD];
#pragma unroll
    for (int i = 0; i < RAD; ++i) v[i] = in[base + (j + i * nb) * estride];
    const int k = j % Ns;
    if (k) {
      const int step = k * twmul;   // i * step < n for i < RAD
#pragma unroll
      for (int i = 1; i < RAD; ++i) {
        C w = tw[i * step];
        if (INV) w.y = -w.y;
        v[i] = cmul(v[i], w);
      }
    }
    Dft<C, RAD, INV>::run(v);
    const int o = base + ((j / Ns) * Ns * RAD + k) * estride;
#pragma unroll
    for (int i = 0; i < RAD; ++i) out[o + i * Ns * estride] = v[i];
  }
}

// Full line FFT (unnormalised; forward e^{-iGr}, inverse e^{+iGr}) on lines
// held in buffer a; b is scratch of the same layout.  Returns the buffer that
// holds the result.  The caller must __syncthreads() before the call (data in
// a complete); the function ends with a __syncthreads().
template <typename C, bool INV>
__device__ C* fft_lines(C* a, C* b, const FftPlan& p, int nlines, int lstride, const int* btab,
                        int estride, const C* tw) {
  int Ns = 1;
  C* in = a;
  C* out = b;
  for (int s = 0; s < p.nstages; ++s) {
    const int r = p.radix[s];
    if (r == 4) fft_stage<C, 4, INV>(in, out, p.n, Ns, nlines, lstride, btab, estride, tw);
    else if (r == 2) fft_stage<C, 2, INV>(in, out, p.n, Ns, nlines, lstride, btab, estride, tw);
    else if (r == 3) fft_stage<C, 3, INV>(in, out, p.n, Ns, nlines, lstride, btab, estride, tw);
    else fft_stage<C, 5, INV>(in, out, p.n, Ns, nlines, lstride, btab, estride, tw);
    __syncthreads();
    Ns *= r;
    C* t = in; in = out; out = t;
  }
  return in;
}

// Asynchronous global -> shared copies (cp.async, cached in L1): a thread issues
// all of its copies of a staging phase back to back and waits once.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 8 bytes, or zeros when !valid (the source is not read then)
__device__ __forceinline__ void cp_async8_zfill(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned n = valid ? 8u : 0u;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

// ---- block reductions (deterministic: fixed tree, fixed order) --------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in thread 0.  `sh` needs blockDim/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

}  // namespace ikr
