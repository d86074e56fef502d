// Tensor-core projection coefficients (5th-generation tensor cores: tcgen05.mma
// kind::tf32, accumulators in tensor memory):
//   C[s][m] = <v_m, y_s> = sum_G conj(V_k[m][G]) y_s[G]
// for the systems s of each k-point and the vectors v_m of an orbital set
// (Phi_k, or [Phi_k Psi_k] for the Schur-complement solves): the M = Phi^H Y of
// eq. discretised_sternheimer and the Q-projection of the CG, in FP32.
//
// Real form.  With y and v stored as interleaved (re, im) floats, a complex
// inner product is two real ones over 2 Nb_k reals:
//   Re C = <v_il, y_il>,   Im C = <v'_il, y_il>,   v' = (-Im v, Re v),
// so D = A B^T with A = [v_0; v'_0; v_1; v'_1; ...] (2 n_k rows) and B = the
// systems' vectors (K-major both): C[s][m] = D[2m][s] + i D[2m+1][s].  A is
// never stored: each stage forms its rows from the FP32 orbitals in registers.
//
// Precision.  kind::tf32 multiplies the upper 19 bits of each float.  Each
// operand is split on the fly x = hi + lo with hi = x with its low 13
// mantissa bits cleared (exact) and lo = x - hi (exact), and D accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi: products to about 2^-20 relative, FP32
// accumulation, as the CUDA-core kernels.  Global traffic is that of the
// FP32 operands themselves.
//
// Tiling.  One CTA (one warpgroup) owns 128 rows of A, NT systems and a
// split-K chunk of kTC reals; stages of kTK = 32 reals are written to shared
// memory in the canonical no-swizzle K-major layout (8 x 16-byte core
// matrices, 128 bytes apart along K, 8-row groups 1024 bytes apart), one
// thread issues 4 x 3 MMAs (M = 128, N = NT, K = 8 each) and commits them to
// an mbarrier that all threads wait on (bounded) before the next stage.  The
// 128 x NT FP32 partial tile is read back with tcgen05.ld (warp w: lanes
// 32w..32w+31), even/odd rows paired into (re, im), and written as per-chunk
// partials that a second kernel adds in fixed chunk order (deterministic).
#include <cstdint>

#include "ops.hpp"

namespace ikr {

namespace {

constexpr int kTM = 128;     // A rows per tile (64 vectors: re and im rows)
constexpr int kTK = 32;      // reals of K per stage (16 plane waves)
constexpr int kTC = 1024;    // reals of K per split-K chunk (512 plane waves)
constexpr int kTileBytes = kTM * kTK * 4;   // one A tile (16 KB)
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz: bound of every mbarrier wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of the 16-byte group c4 (reals 4 c4 .. 4 c4 + 3) of row r in a
// kTK-wide tile: canonical K-major layout without swizzle
__device__ __forceinline__ int core_off(int r, int c4) { return (r >> 3) * 1024 + c4 * 128 + (r & 7) * 16; }

// shared-memory matrix descriptor: start address, leading (K) byte offset 128,
// stride (8-row group) byte offset 1024, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: D F32, A and B TF32, both K-major, N = n, M = 128
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// waits for the phase with the given parity; false after ~1 s
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate ncols tensor-memory columns, address to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 consecutive columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Work item e of a tile fill -> (row, 16-byte group c4 along K).  In the canonical
// K-major layout the 16-byte bank slot of an element is row mod 8, so a quarter-warp
// (8 threads, one 128-byte wavefront) must write 8 different rows: lanes 0-7 of a warp
// take rows 8 b .. 8 b + 7 at one group, lanes 8-15 the next group, ...; every row then
// gets 4 consecutive groups (64 contiguous bytes of its global vector) from one warp.
__device__ __forceinline__ void tile_item(int e, int& row, int& c4) {
  const int q = e & 31, w = e >> 5;
  row = (q & 7) + 8 * (w >> 1);
  c4 = (q >> 3) + 4 * (w & 1);
}

}  // namespace

// Partial sums of D = A B^T over one split-K chunk: part[(s * maxcnt + m) * nch + chunk] = (Re, Im) C[s][m].
// grid: (chunks, k-points, A-tiles x system tiles); NT systems per tile.
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_coef(const float2* __restrict__ phi, const int* __restrict__ set_off,
              const int* __restrict__ set_cnt, const int* __restrict__ nb_k, const int* __restrict__ kstart,
              const int* __restrict__ kcount, const int* __restrict__ slist, const int* __restrict__ scount,
              const float2* __restrict__ Y, int ldy, int ld, int nmt, int nch,
              int maxcnt, const int* __restrict__ active, double2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sAhi = sm;
  unsigned char* sAlo = sm + kTileBytes;
  unsigned char* sBhi = sm + 2 * kTileBytes;
  unsigned char* sBlo = sBhi + NT * kTK * 4;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sBlo + NT * kTK * 4);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int k = blockIdx.y, chunk = blockIdx.x;
  const int tm = blockIdx.z % nmt, tn = blockIdx.z / nmt;
  const int cnt = set_cnt[k], nb = nb_k[k], ns = scount ? scount[k] : kcount[k];
  // system of tile row j: the k-point's j-th active system (compacted list) or its j-th system
  auto sys_at = [&](int j) { return slist ? slist[kstart[k] + j] : kstart[k] + j; };
  const int i0 = tm * kTM, s0 = tn * NT;
  const int k0 = chunk * kTC, k1 = min(k0 + kTC, 2 * nb);
  if (i0 >= 2 * cnt || s0 >= ns || k0 >= k1) return;   // uniform over the block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kCols = NT < 32 ? 32 : NT;
  if (warp == 0) tmem_alloc(slot, kCols);
  if (tid == 0) mbar_init(bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const float* vbase = reinterpret_cast<const float*>(phi + ((size_t)set_off[k] + i0 / 2) * ld);
  const size_t lda = 2 * (size_t)ld;                    // reals per orbital
  bool ok = true;
  uint32_t phase = 0;
  uint32_t acc = 0;
  // each thread's share of a stage, fetched into registers one stage ahead so that the
  // global loads of stage kb + kTK overlap the MMAs of stage kb
  constexpr int kAE = (kTM / 2) * (kTK / 4) / 128;   // A groups per thread (64 orbitals x 8)
  constexpr int kBE = NT * (kTK / 4) / 128;          // B groups per thread
  float4 ra[kAE], rb[kBE];
  auto fetch = [&](int kb) {
#pragma unroll
    for (int j = 0; j < kAE; ++j) {
      int mo, c4;
      tile_item(tid + 128 * j, mo, c4);
      ra[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      // orbitals past cnt are zero; the orbitals are zero past Nb_k, so a group across
      // 2 Nb_k needs no mask
      if (i0 / 2 + mo < cnt && kb + 4 * c4 < k1)
        ra[j] = *reinterpret_cast<const float4*>(vbase + mo * lda + kb + 4 * c4);
    }
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
      int r, c4;
      tile_item(tid + 128 * j, r, c4);
      const int re = kb + 4 * c4;                      // first real of the group (two plane waves)
      rb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s0 + r < ns && re < k1) {
        const int s = sys_at(s0 + r);
        if (!active || active[s]) {
          rb[j] = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(Y + (size_t)s * ldy) + re);
          if (re + 2 >= k1) rb[j].z = rb[j].w = 0.f;    // second plane wave past Nb_k
        }
      }
    }
  };
  fetch(k0);
  for (int kb = k0; kb < k1 && ok; kb += kTK) {
    // A tile: orbital mo gives row 2 mo = (Re, Im) and row 2 mo + 1 = (-Im, Re) of two plane
    // waves per 16-byte group; B tile: the systems' vectors; both split into hi and lo
#pragma unroll
    for (int j = 0; j < kAE; ++j) {
      int mo, c4;
      tile_item(tid + 128 * j, mo, c4);
      const float4 x = ra[j];
      const float4 y = make_float4(-x.y, x.x, -x.w, x.z);
      const float4 xh = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
      const float4 yh = make_float4(tf32_hi(y.x), tf32_hi(y.y), tf32_hi(y.z), tf32_hi(y.w));
      *reinterpret_cast<float4*>(sAhi + core_off(2 * mo, c4)) = xh;
      *reinterpret_cast<float4*>(sAlo + core_off(2 * mo, c4)) =
          make_float4(x.x - xh.x, x.y - xh.y, x.z - xh.z, x.w - xh.w);
      *reinterpret_cast<float4*>(sAhi + core_off(2 * mo + 1, c4)) = yh;
      *reinterpret_cast<float4*>(sAlo + core_off(2 * mo + 1, c4)) =
          make_float4(y.x - yh.x, y.y - yh.y, y.z - yh.z, y.w - yh.w);
    }
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
      int r, c4;
      tile_item(tid + 128 * j, r, c4);
      const float4 x = rb[j];
      const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
      *reinterpret_cast<float4*>(sBhi + core_off(r, c4)) = h;
      *reinterpret_cast<float4*>(sBlo + core_off(r, c4)) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      constexpr uint32_t id = idesc_tf32(NT);
#pragma unroll
      for (int kk = 0; kk < kTK / 8; ++kk) {
        const uint32_t off = kk * 256;                  // two 16-byte groups along K per MMA
        const uint64_t ah = sdesc(saddr(sAhi) + off), al = sdesc(saddr(sAlo) + off);
        const uint64_t bh = sdesc(saddr(sBhi) + off), bl = sdesc(saddr(sBlo) + off);
        mma_tf32(tmem, ah, bh, id, acc);
        mma_tf32(tmem, ah, bl, id, 1);
        mma_tf32(tmem, al, bh, id, 1);
        acc = 1;
      }
      mma_commit(bar);
    }
    if (kb + kTK < k1) fetch(kb + kTK);
    // the MMAs read this stage's shared memory: wait before it is rewritten; the
    // outcome is made uniform so that no thread leaves the loop alone
    ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0) != 0;
    phase ^= 1;
    tc_fence_after();
  }
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    // a second bounded wait for the MMAs still in flight before their tensor memory is freed
    // (the phase was flipped after the failed wait)
    mbar_wait(bar, phase ^ 1);
    __syncthreads();
  } else {
    // epilogue: lanes 32 w .. 32 w + 31 of tensor memory are rows i0 + 32 w + lane of D
    const int r = 32 * warp + lane;
    const int i = i0 + r, m = i >> 1;
    float v[32];
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 32) {
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float im = __shfl_xor_sync(0xffffffffu, v[j], 1);
        const int sl = s0 + c0 + j;
        if (!(lane & 1) && i < 2 * cnt && sl < ns) {
          const int s = sys_at(sl);
          if (!active || active[s]) part[((size_t)s * maxcnt + m) * nch + chunk] = make_double2((double)v[j], (double)im);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
}

// out[s][g] = alpha in[s][g] + beta sum_m v_m[g] coef[s][m] for the plane waves of one 128-real
// tile (64 plane waves) and NT systems; with dv, dpart[s * nparts + tile] = sum Re(conj(dv) out)
// over the tile (the chunking of the CUDA-core apply: 64 plane waves).
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_apply(const float2* __restrict__ phi, const int* __restrict__ set_off, const int* __restrict__ set_cnt,
               const int* __restrict__ nb_k, const int* __restrict__ kstart, const int* __restrict__ kcount,
               const int* __restrict__ slist, const int* __restrict__ scount,
               const double2* __restrict__ coef, int maxcnt, const float2* in, float alpha, float beta,
               float2* out, int ldy, int ld, const float2* __restrict__ dv, double* __restrict__ dpart, int nparts,
               const int* __restrict__ active, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sAhi = sm;
  unsigned char* sAlo = sm + kTileBytes;
  unsigned char* sBhi = sm + 2 * kTileBytes;
  unsigned char* sBlo = sBhi + NT * kTK * 4;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sBlo + NT * kTK * 4);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  double* red = reinterpret_cast<double*>(slot + 2);              // [4 warps][NT] dot partials
  const int k = blockIdx.y, tile = blockIdx.x, tn = blockIdx.z;
  const int cnt = set_cnt[k], nb = nb_k[k], ns = scount ? scount[k] : kcount[k];
  // system of tile row j: the k-point's j-th active system (compacted list) or its j-th system
  auto sys_at = [&](int j) { return slist ? slist[kstart[k] + j] : kstart[k] + j; };
  const int r0 = tile * kTM, s0 = tn * NT;                        // first real row (2 g + c), first system
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (s0 >= ns) return;                                           // uniform
  if (r0 >= 2 * nb) {                                             // tile past Nb_k: define the dot partials
    if (dpart)
      for (int j = tid; j < NT; j += 128) {
        if (s0 + j >= ns) continue;
        const int s = sys_at(s0 + j);
        if (!active || active[s]) dpart[(size_t)s * nparts + tile] = 0.0;
      }
    return;
  }
  constexpr uint32_t kCols = NT < 32 ? 32 : NT;
  if (warp == 0) tmem_alloc(slot, kCols);
  if (tid == 0) mbar_init(bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int g0 = r0 / 2;                                          // first plane wave of the tile
  const float2* vk = phi + (size_t)set_off[k] * ld;
  const int kend = 2 * cnt;
  bool ok = true;
  uint32_t phase = 0, acc = 0;
  for (int kb = 0; kb < kend && ok; kb += kTK) {
    // A tile = AT[2g + c][2m + q] from the orbitals: (c, q) = (0, 0) Re v_m[g], (0, 1) -Im,
    // (1, 0) Im, (1, 1) Re; an item is one plane wave and one 16-byte group (orbitals 2 c4,
    // 2 c4 + 1), written as one 16-byte store per row; consecutive threads take consecutive
    // plane waves (coalesced loads; rows 2 g and 2 g + 1 of a quarter-warp fall 2 per bank
    // slot); orbitals past cnt are zero (g0 + 63 < ld: the orbitals are zero past Nb_k)
    for (int e = tid; e < (kTM / 2) * (kTK / 4); e += 128) {
      const int gl = e & 63, c4 = e >> 6;
      const int m0 = kb / 2 + 2 * c4;
      const float2 z = make_float2(0.f, 0.f);
      const float2 p0 = m0 < cnt ? vk[(size_t)m0 * ld + g0 + gl] : z;
      const float2 p1 = m0 + 1 < cnt ? vk[(size_t)(m0 + 1) * ld + g0 + gl] : z;
      const float4 r0 = make_float4(p0.x, -p0.y, p1.x, -p1.y), r1 = make_float4(p0.y, p0.x, p1.y, p1.x);
      const float4 h0 = make_float4(tf32_hi(r0.x), tf32_hi(r0.y), tf32_hi(r0.z), tf32_hi(r0.w));
      const float4 h1 = make_float4(tf32_hi(r1.x), tf32_hi(r1.y), tf32_hi(r1.z), tf32_hi(r1.w));
      *reinterpret_cast<float4*>(sAhi + core_off(2 * gl, c4)) = h0;
      *reinterpret_cast<float4*>(sAlo + core_off(2 * gl, c4)) =
          make_float4(r0.x - h0.x, r0.y - h0.y, r0.z - h0.z, r0.w - h0.w);
      *reinterpret_cast<float4*>(sAhi + core_off(2 * gl + 1, c4)) = h1;
      *reinterpret_cast<float4*>(sAlo + core_off(2 * gl + 1, c4)) =
          make_float4(r1.x - h1.x, r1.y - h1.y, r1.z - h1.z, r1.w - h1.w);
    }
    for (int e = tid; e < NT * (kTK / 4); e += 128) {
      int r, c4;
      tile_item(e, r, c4);
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      const int s = s0 + r < ns ? sys_at(s0 + r) : -1;
      if (s >= 0 && (!active || active[s]))
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int i = kb + 4 * c4 + 2 * q;                      // real index 2 m (+1 below)
          if (i < kend) {
            const double2 cc = coef[(size_t)s * maxcnt + (i >> 1)];
            x[2 * q] = (float)cc.x;
            x[2 * q + 1] = (float)cc.y;
          }
        }
      const float4 h = make_float4(tf32_hi(x[0]), tf32_hi(x[1]), tf32_hi(x[2]), tf32_hi(x[3]));
      *reinterpret_cast<float4*>(sBhi + core_off(r, c4)) = h;
      *reinterpret_cast<float4*>(sBlo + core_off(r, c4)) =
          make_float4(x[0] - h.x, x[1] - h.y, x[2] - h.z, x[3] - h.w);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      constexpr uint32_t id = idesc_tf32(NT);
#pragma unroll
      for (int kk = 0; kk < kTK / 8; ++kk) {
        const uint32_t off = kk * 256;
        const uint64_t ah = sdesc(saddr(sAhi) + off), al = sdesc(saddr(sAlo) + off);
        const uint64_t bh = sdesc(saddr(sBhi) + off), bl = sdesc(saddr(sBlo) + off);
        mma_tf32(tmem, ah, bh, id, acc);
        mma_tf32(tmem, ah, bl, id, 1);
        mma_tf32(tmem, al, bh, id, 1);
        acc = 1;
      }
      mma_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0) != 0;
    phase ^= 1;
    tc_fence_after();
  }
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    // a second bounded wait for the MMAs still in flight before their tensor memory is freed
    // (the phase was flipped after the failed wait)
    mbar_wait(bar, phase ^ 1);
    __syncthreads();
  } else {
    const int row = r0 + 32 * warp + lane;                         // 2 g + c
    const int g = row >> 1;
    float v[32];
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 32) {
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float im = __shfl_xor_sync(0xffffffffu, v[j], 1);
        const int sl = s0 + c0 + j;
        const int s = sl < ns ? sys_at(sl) : -1;
        const bool on = !(lane & 1) && g < nb && s >= 0 && (!active || active[s]);
        double d = 0.0;
        if (on) {
          const size_t o = (size_t)s * ldy + g;
          float2 y = make_float2(beta * v[j], beta * im);
          if (alpha != 0.f) {
            const float2 xi = in[o];
            y.x += alpha * xi.x;
            y.y += alpha * xi.y;
          }
          out[o] = y;
          if (dv) {
            const float2 w = dv[o];
            d = (double)w.x * y.x + (double)w.y * y.y;
          }
        }
        if (dpart) {
          d = warp_sum(d);
          if (lane == 0) red[warp * NT + c0 + j] = d;
        }
      }
    }
    if (dpart) {
      __syncthreads();
      for (int j = tid; j < NT; j += 128) {
        if (s0 + j >= ns) continue;
        const int s = sys_at(s0 + j);
        if (!active || active[s])
          dpart[(size_t)s * nparts + tile] = ((red[j] + red[NT + j]) + red[2 * NT + j]) + red[3 * NT + j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
}

// coef[s][m] = sum of the chunk partials in chunk order: a warp per coefficient
__global__ void k_tc_reduce(const double2* __restrict__ part, int nsys, int maxcnt, int nch,
                            const int* __restrict__ sys_k, const int* __restrict__ set_cnt,
                            const int* __restrict__ nb_k, const int* __restrict__ active, double2* __restrict__ coef) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nsys * maxcnt) return;
  const int s = (int)(w / maxcnt), m = (int)(w - (long long)s * maxcnt);
  if (active && !active[s]) return;
  const int k = sys_k[s];
  if (m >= set_cnt[k]) return;
  const int nc = (2 * nb_k[k] + kTC - 1) / kTC;
  const double2* p = part + ((size_t)s * maxcnt + m) * nch;
  double ax = 0.0, ay = 0.0;
  for (int cc = lane; cc < nc; cc += 32) {
    const double2 v = p[cc];
    ax += v.x;
    ay += v.y;
  }
  ax = warp_sum(ax);
  ay = warp_sum(ay);
  if (lane == 0) coef[w] = make_double2(ax, ay);
}

// The active systems of every k-point, in order, at the k-point's offset kstart[k]
// (slist), and their number (scount): the tensor-core kernels tile over these, so
// systems whose CG has finished cost nothing.  One warp per k-point: ballot and
// population count over chunks of 32 systems.
__global__ void k_tc_compact(const int* __restrict__ active, const int* __restrict__ kstart,
                             const int* __restrict__ kcount, int nk, int* __restrict__ slist,
                             int* __restrict__ scount) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= nk) return;
  const int s0 = kstart[k], n = kcount[k];
  int pos = 0;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    const bool a = j < n && active[s0 + j] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (a) slist[s0 + pos + __popc(m & ((1u << lane) - 1u))] = s0 + j;
    pos += __popc(m);
  }
  if (lane == 0) scount[k] = pos;
}

// ----------------------------------------------------------------- host --

namespace {
// compacted active lists for a masked launch (nullptr, nullptr without a mask)
void tc_active_lists(ikr_ctx* c, const SysList& L, const int* active, const int** slist, const int** scount) {
  *slist = nullptr;
  *scount = nullptr;
  if (!active || L.n == 0) return;
  const int nk = (int)c->k.size();
  c->ws.tc_list.reserve(L.n);
  c->ws.tc_cnt.reserve(nk);
  k_tc_compact<<<(nk + 3) / 4, 128, 0, c->stream>>>(active, L.d_kstart.p, L.d_kcount.p, nk, c->ws.tc_list.p,
                                                     c->ws.tc_cnt.p);
  IKR_CUDA(cudaGetLastError());
  *slist = c->ws.tc_list.p;
  *scount = c->ws.tc_cnt.p;
}
}  // namespace

// the error flag of the tensor-core kernels: set by any launch whose wait ran out,
// cleared only when it is created and by tc_check, so no later launch hides it
static void tc_flag_ready(ikr_ctx* c) {
  if (c->tc_err.p) return;
  c->tc_err.reserve(1);
  IKR_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
}

bool tc_proj_ok(ikr_ctx* c, const OrbSet& set) {
  return c->tc_proj && set.maxcnt >= 1 && (c->ld % 2) == 0;
}

void proj_coef_tc(ikr_ctx* c, const SysList& L, const float2* Y, int ldy, const int* active, double2* coef,
                  const OrbSet& set) {
  IKR_REQUIRE(ldy % 2 == 0, IKR_ERR_ARG, "tensor-core projections need an even vector stride");
  int maxns = 0, maxnb = 0;
  for (int v : L.kcount) maxns = std::max(maxns, v);
  for (auto& K : c->k) maxnb = std::max(maxnb, K.nb);
  const int nch = (2 * maxnb + kTC - 1) / kTC;
  const int nmt = (2 * set.maxcnt + kTM - 1) / kTM;
  const int nt = maxns <= 32 ? 32 : (maxns <= 64 ? 64 : 128);
  const int nnt = (maxns + nt - 1) / nt;
  c->ws.cpart.reserve((size_t)nch * L.n * set.maxcnt * 2);
  double2* part = reinterpret_cast<double2*>(c->ws.cpart.p);
  tc_flag_ready(c);
  dim3 grid(nch, (unsigned)c->k.size(), (unsigned)(nmt * std::max(nnt, 1)));
  const size_t smem = 2 * kTileBytes + 2 * (size_t)nt * kTK * 4 + 64;
  const int *slist, *scount;
  tc_active_lists(c, L, active, &slist, &scount);
  auto launch = [&](auto kern) {
    IKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 128, smem, c->stream>>>(set.phi32, set.off, set.cnt, c->d_nb.p, L.d_kstart.p, L.d_kcount.p, slist,
                                         scount, Y, ldy, c->ld, nmt, nch, set.maxcnt, active, part, c->tc_err.p);
  };
  if (nt == 32) launch(k_tc_coef<32>);
  else if (nt == 64) launch(k_tc_coef<64>);
  else launch(k_tc_coef<128>);
  IKR_CUDA(cudaGetLastError());
  const long long threads = 32LL * L.n * set.maxcnt;
  k_tc_reduce<<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(part, L.n, set.maxcnt, nch, L.d_k.p,
                                                                         set.cnt, c->d_nb.p, active, coef);
  IKR_CUDA(cudaGetLastError());
}

void proj_apply_tc(ikr_ctx* c, const SysList& L, const double2* coef, const float2* in, float alpha, float beta,
                   float2* out, int ldy, const float2* dv, double* dpart, const int* active, const OrbSet& set) {
  int maxns = 0;
  for (int v : L.kcount) maxns = std::max(maxns, v);
  const int nparts = (c->ld + 63) / 64;                           // 64 plane waves per tile and dot partial
  const int nt = maxns <= 32 ? 32 : (maxns <= 64 ? 64 : 128);
  const int nnt = std::max(1, (maxns + nt - 1) / nt);
  tc_flag_ready(c);
  dim3 grid(nparts, (unsigned)c->k.size(), (unsigned)nnt);
  const size_t smem = 2 * kTileBytes + 2 * (size_t)nt * kTK * 4 + 16 + 32 * (size_t)nt;
  const int *slist, *scount;
  tc_active_lists(c, L, active, &slist, &scount);
  auto launch = [&](auto kern) {
    IKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 128, smem, c->stream>>>(set.phi32, set.off, set.cnt, c->d_nb.p, L.d_kstart.p, L.d_kcount.p, slist,
                                         scount, coef, set.maxcnt, in, alpha, beta, out, ldy, c->ld, dv, dpart, nparts,
                                         active, c->tc_err.p);
  };
  if (nt == 32) launch(k_tc_apply<32>);
  else if (nt == 64) launch(k_tc_apply<64>);
  else launch(k_tc_apply<128>);
  IKR_CUDA(cudaGetLastError());
}

void tc_check(ikr_ctx* c) {
  if (!c->tc_err.p) return;
  int e = 0;
  IKR_CUDA(cudaMemcpyAsync(&e, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  IKR_CUDA(cudaStreamSynchronize(c->stream));
  if (e != 0) IKR_CUDA(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
  IKR_REQUIRE(e == 0, IKR_ERR_TIMEOUT, "tensor-core projection: an mbarrier wait ran out");
}

}  // namespace ikr
