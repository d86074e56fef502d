// Arithmetic throughput of the GPU, for the ALU rooflines of the plane passes.
//
// The plane passes of the H_k application keep the grid on chip and are bound
// by the rate at which the SMs issue arithmetic, not by HBM.  Their roofline
// peak is derived from unit counts and clocks (SMs x 128 FP32 lanes x 2 flops
// per FMA x SM clock); the kernels here measure what the SMs sustain on the
// same instruction mixes, so that the derivation is checked on the device:
//   - FP32 FMA chains and FP64 FMA chains (2 flops per FMA);
//   - radix-4 butterflies with twiddle products, in FP32 and in the
//     double-float arithmetic of the FP64-accurate plane pass (3 complex
//     products and 8 complex sums per butterfly: 34 real flops, each
//     double-float operation counted as one FP64 flop).
// Every thread runs 8 independent chains so that the FMA pipes stay full; the
// results are stored so that nothing is optimised away.  Timing: CUDA events
// on the caller's stream around one launch after a warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "ops.hpp"

namespace ikr {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(int iters, T m, T a, T* __restrict__ out) {
  T v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = T(threadIdx.x + j) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) v[j] = v[j] * m + a;     // one FMA
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one radix-4 butterfly on four complex values with twiddles w1..w3, as the
// Stockham stages of the plane pass run it (Dft<C, 4>); every 8 butterflies the
// values are scaled by 2^-8 (their growth: the length-4 DFT doubles the norm)
template <typename C>
__device__ __forceinline__ void butterfly4(C* x, const C* w) {
  x[1] = cmul(x[1], w[0]);
  x[2] = cmul(x[2], w[1]);
  x[3] = cmul(x[3], w[2]);
  Dft<C, 4, false>::run(x);
}

constexpr float kShrink = 0.00390625f;        // 2^-8, exact
__device__ __forceinline__ void shrink(float2& c) { c.x *= kShrink; c.y *= kShrink; }
__device__ __forceinline__ void shrink(dfloat2& c) {
  c.x.hi *= kShrink; c.x.lo *= kShrink; c.y.hi *= kShrink; c.y.lo *= kShrink;
}

template <typename C>
__global__ void __launch_bounds__(kThreads) k_butterflies(int iters, C w0, C w1, C w2, C* __restrict__ out) {
  constexpr int kB = 2;                       // independent butterflies per thread
  C x[kB][4];
  const C w[3] = {w0, w1, w2};
#pragma unroll
  for (int b = 0; b < kB; ++b)
#pragma unroll
    for (int i = 0; i < 4; ++i) x[b][i] = mk<C>(decltype(C::x)(0.25f * (i + 1)), decltype(C::x)(0.125f * b));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int b = 0; b < kB; ++b) butterfly4(x[b], w);
#pragma unroll
    for (int b = 0; b < kB; ++b)
#pragma unroll
      for (int i = 0; i < 4; ++i) shrink(x[b][i]);
  }
  C s = x[0][0];
#pragma unroll
  for (int b = 0; b < kB; ++b)
#pragma unroll
    for (int i = 0; i < 4; ++i) s = cadd(s, x[b][i]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
double time_launch(cudaStream_t st, F&& launch) {
  cudaEvent_t e0, e1;
  IKR_CUDA(cudaEventCreate(&e0));
  IKR_CUDA(cudaEventCreate(&e1));
  launch();                                   // warm-up
  IKR_CUDA(cudaGetLastError());
  IKR_CUDA(cudaEventRecord(e0, st));
  launch();
  IKR_CUDA(cudaEventRecord(e1, st));
  IKR_CUDA(cudaEventSynchronize(e1));
  IKR_CUDA(cudaGetLastError());
  float ms = 0.f;
  IKR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  IKR_CUDA(cudaEventDestroy(e0));
  IKR_CUDA(cudaEventDestroy(e1));
  return ms * 1e-3;
}

}  // namespace

void device_peaks(double* out, cudaStream_t st) {
  int dev = 0, sms = 0, clock_khz = 0;
  IKR_CUDA(cudaGetDevice(&dev));
  IKR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    clock_khz = 0;
  }
  const int blocks = sms * 8;
  const size_t nthr = (size_t)blocks * kThreads;
  DBuf<double2> buf;
  buf.reserve(nthr * 2);                      // room for the largest element type (dfloat2 = 16 bytes)
  const double thr = (double)nthr;
  // FMA chains: iters x 16 x kChains FMAs per thread, 2 flops each
  const int it32 = 4096, it64 = 256;
  const double t32 = time_launch(st, [&] {
    k_fma_chain<float><<<blocks, kThreads, 0, st>>>(it32, 0.999999f, 1e-7f, reinterpret_cast<float*>(buf.p));
  });
  const double t64 = time_launch(st, [&] {
    k_fma_chain<double><<<blocks, kThreads, 0, st>>>(it64, 0.999999999, 1e-12, reinterpret_cast<double*>(buf.p));
  });
  // butterflies: iters x 8 x 2 butterflies of 34 real flops per thread
  const float c = 0.70710678f;
  const int itb32 = 512, itbdf = 128;
  const double tb32 = time_launch(st, [&] {
    k_butterflies<float2><<<blocks, kThreads, 0, st>>>(itb32, make_float2(c, -c), make_float2(0.f, -1.f),
                                                        make_float2(-c, -c), reinterpret_cast<float2*>(buf.p));
  });
  const dfloat2 w0{dfloat(c, 0.f), dfloat(-c, 0.f)}, w1{dfloat(0.f, 0.f), dfloat(-1.f, 0.f)},
      w2{dfloat(-c, 0.f), dfloat(-c, 0.f)};
  const double tbdf = time_launch(st, [&] {
    k_butterflies<dfloat2><<<blocks, kThreads, 0, st>>>(itbdf, w0, w1, w2, reinterpret_cast<dfloat2*>(buf.p));
  });
  out[0] = sms;
  out[1] = thr * it32 * 16.0 * kChains * 2.0 / t32 / 1e12;
  out[2] = thr * it64 * 16.0 * kChains * 2.0 / t64 / 1e12;
  out[3] = thr * itb32 * 8.0 * 2.0 * 34.0 / tb32 / 1e12;
  out[4] = thr * itbdf * 8.0 * 2.0 * 34.0 / tbdf / 1e12;
  out[5] = clock_khz * 1e-3;
}

}  // namespace ikr
