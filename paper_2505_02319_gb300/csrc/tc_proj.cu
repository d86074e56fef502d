// Tensor-core projection products (5th-generation tensor cores: tcgen05.mma
// kind::f16 with bf16 operands, accumulators in tensor memory):
//   C[s][m] = <v_m, y_s> = sum_G conj(V_k[m][G]) y_s[G]            (k_tc_coef + k_tc_reduce)
//   out_s   = alpha in_s + beta sum_m v_m C[s][m]                    (k_tc_apply)
// for the systems s of each k-point and the vectors v_m of an orbital set
// (Phi_k, [Phi_k Psi_k] for the Schur-complement solves, or the
// Kleinman-Bylander projectors): the M = Phi^H Y of eq.
// discretised_sternheimer, the Q-projection of the CG and B D B^H, in FP32.
//
// Real form.  With y and v stored as interleaved (re, im) floats, a complex
// inner product is two real ones over 2 Nb_k reals:
//   Re C = <v_il, y_il>,   Im C = <v'_il, y_il>,   v' = (-Im v, Re v),
// so C = A B^T with A = [v_0; v'_0; v_1; v'_1; ...] (2 n_k rows) and B = the
// systems' vectors; V C has the rows (Re v, -Im v) and (Im v, Re v) of every
// plane wave against the interleaved coefficients.  The rotated rows are
// never stored: the kernels form them from the FP32 data in registers.
//
// Precision.  Every FP32 operand is split exactly into three bf16 numbers,
//   x = b0 + b1 + b2,  b0 = RN(x), b1 = RN(x - b0), b2 = x - b0 - b1
// (x has 24 significant bits; b0 and b1 take 8 each with round-to-nearest,
// which leaves at most 8 for b2), and D accumulates the six products
// a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0, each exact in FP32.  The
// omitted terms are below 2^-23 of |a b|: the products are as accurate as
// FP32 multiplications.  The leading products a0 b0 and the five corrections
// go to two accumulators (added in the epilogue), so the long FP32 sum of a
// chunk sees one accumulation per K step instead of six, and V^H Y sums at
// most 512 reals per chunk in FP32 before the FP64 reduction.  (A split into
// TF32 halves leaves 2^-20 per product, which stalls the CG at the smallest
// tolerances of the solve.)  Global traffic is that of the FP32 operands
// themselves.
//
// Pipeline.  One CTA (8 warps) owns a 128-row tile of D and NT systems; K runs
// in stages of kTK = 32 reals through a ring of two shared-memory buffers
// holding the three pieces of both operands, K-major, in 8-row x 64-byte atoms
// (64-byte swizzle, or the canonical layout of 8 x 16-byte core matrices:
// ikr_set_tensor_cores mode 1 or 2).  For stage st every thread waits (bounded)
// for the MMAs of stage st - 2, which read the same buffer, splits its
// registers into that buffer, issues the global loads of stage st + 2 into
// the registers it just freed, and meets the others at one barrier; thread 0
// then issues the stage's 2 x 6 MMAs (M = 128, N = NT, K = 16) and commits
// them to the buffer's mbarrier.  So the MMAs of one stage run while the next
// is filled, and every load has two stages to arrive.  The systems of the
// tile (the k-point's active systems, compacted in order) are listed once per
// CTA in shared memory: finished systems cost nothing, and inside the CG the
// tile width follows the number of systems still active.  The accumulator
// tile is read back with tcgen05.ld (warp w: lanes 32 (w mod 4) + 0..31,
// column half w / 4), even/odd rows paired into (re, im).  V^H Y runs split-K
// with the chunks sized for about two CTAs per SM, and a second kernel adds the
// FP32 chunk partials in FP64 in chunk order (deterministic).
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include "ops.hpp"

namespace ikr {

namespace {

constexpr int kTM = 128;                  // D rows per tile (coef: 64 vectors; apply: 64 plane waves)
constexpr int kTK = 32;                   // reals of K per stage
constexpr int kRowB = 2 * kTK;            // bytes of one row of one bf16 piece in a stage
constexpr int kSBO = 8 * kRowB;           // bytes between 8-row groups
constexpr int kAPiece = kTM * kRowB;      // one piece of the A tile (8 KB)
constexpr int kThreads = 256;
constexpr int kMaxChunk = 512;            // reals of V^H Y summed in FP32 before the FP64 reduction
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz: bound of every mbarrier wait

template <int NT> struct TcLayout {
  static constexpr int kBPiece = NT * kRowB;
  static constexpr int kStage = 3 * kAPiece + 3 * kBPiece;      // A0 A1 A2 B0 B1 B2
  static constexpr int kBar = 2 * kStage;                       // two mbarriers
  static constexpr int kSlot = kBar + 16;                       // tensor-memory address
  static constexpr int kSys = kSlot + 16;                       // [NT] systems of the tile
  static constexpr int kWcnt = kSys + 4 * NT;                   // [8] active systems per warp (scan)
  static constexpr int kRed = (kWcnt + 4 * 8 + 15) / 16 * 16;   // apply: [NT][2] dot partials
  static constexpr int kCoef = kRed;
  static constexpr int kApply = kRed + 2 * NT * 8;
  // apply: after the MMAs the ring holds D as [NT systems][128 rows] floats
  static_assert(NT * kTM * 4 <= 2 * kStage, "the D tile fits the ring");
  // two accumulators of NT columns: the leading products a0 b0, and the five corrections
  static constexpr uint32_t kCols = 2 * NT < 32 ? 32 : 2 * NT;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of the 16-byte chunk c (reals 8 c .. 8 c + 7) of row r in one piece:
// 64-byte swizzle (row r of its atom at 64 (r mod 8), chunk c at c xor ((r / 2) mod 4)),
// or the canonical layout (core matrices of 8 rows x 16 bytes, 128 bytes apart along K)
template <bool SWZ>
__device__ __forceinline__ int chunk_off(int r, int c) {
  return SWZ ? (r >> 3) * kSBO + (r & 7) * kRowB + ((c ^ ((r >> 1) & 3)) << 4)
             : (r >> 3) * kSBO + c * 128 + (r & 7) * 16;
}

// shared-memory matrix descriptor: start address, leading byte offset (K-adjacent core
// matrices, 128 bytes; not used by the swizzled layout), stride byte offset 512 (8-row
// groups), descriptor version 1, layout (4: 64-byte swizzle, 0: none)
template <bool SWZ>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = SWZ ? 1 : (128 >> 4);
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (lbo << 16) | ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46) |
         ((SWZ ? 4ull : 0ull) << 61);
}
// start offset of K step kk (16 bf16 = 32 bytes of every row)
template <bool SWZ> __device__ __forceinline__ uint32_t kstep_off(int kk) { return SWZ ? 32u * kk : 256u * kk; }

// instruction descriptor: D F32, A and B BF16, both K-major, N = n, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
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
// 16 consecutive columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// ------------------------------------------------------------ bf16 split --
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);        // .x (lower address) = lo
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
// the pair (a, b) split into three bf16 pairs: a = a0 + a1 + a2, b likewise, exactly
__device__ __forceinline__ void split2(float a, float b, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  w0 = pack_bf16(a, b);
  const float ra = a - bf_lo(w0), rb = b - bf_hi(w0);
  w1 = pack_bf16(ra, rb);
  w2 = pack_bf16(ra - bf_lo(w1), rb - bf_hi(w1));
}
// on a bf16 pair (lo, hi), exactly: (-hi, lo), (lo, -hi), (hi, lo)
__device__ __forceinline__ uint32_t rot_pair(uint32_t w) { return __byte_perm(w, 0, 0x1032) ^ 0x00008000u; }
__device__ __forceinline__ uint32_t conj_pair(uint32_t w) { return w ^ 0x80000000u; }
__device__ __forceinline__ uint32_t swap_pair(uint32_t w) { return __byte_perm(w, 0, 0x1032); }

// Eight reals (four interleaved complex numbers) in three bf16 pieces.
struct Pieces {
  uint4 p[3];
};
__device__ __forceinline__ Pieces split8(float4 u, float4 v) {
  Pieces q;
  split2(u.x, u.y, q.p[0].x, q.p[1].x, q.p[2].x);
  split2(u.z, u.w, q.p[0].y, q.p[1].y, q.p[2].y);
  split2(v.x, v.y, q.p[0].z, q.p[1].z, q.p[2].z);
  split2(v.z, v.w, q.p[0].w, q.p[1].w, q.p[2].w);
  return q;
}
template <typename F>
__device__ __forceinline__ Pieces map_pairs(const Pieces& q, F f) {
  Pieces r;
#pragma unroll
  for (int i = 0; i < 3; ++i) r.p[i] = make_uint4(f(q.p[i].x), f(q.p[i].y), f(q.p[i].z), f(q.p[i].w));
  return r;
}
// the three pieces of row r, chunk c into the piece tiles at t, t + pb, t + 2 pb
template <bool SWZ>
__device__ __forceinline__ void put_pieces(unsigned char* t, int pb, int r, int c, const Pieces& q) {
  const int off = chunk_off<SWZ>(r, c);
#pragma unroll
  for (int i = 0; i < 3; ++i) *reinterpret_cast<uint4*>(t + i * pb + off) = q.p[i];
}
// Rows 2 p and 2 p + 1 of a row pair, written by a quarter-warp of consecutive p: the
// lanes with p mod 8 >= 4 write row 2 p + 1 first, so that each store covers 8 different
// row slots of the atom (in both layouts the bank slot depends on the row mod 8).
template <bool SWZ>
__device__ __forceinline__ void put_pair(unsigned char* t, int pb, int p, int c, const Pieces& even,
                                         const Pieces& odd) {
  const bool swap = (p >> 2) & 1;
  put_pieces<SWZ>(t, pb, 2 * p + (swap ? 1 : 0), c, swap ? odd : even);
  put_pieces<SWZ>(t, pb, 2 * p + (swap ? 0 : 1), c, swap ? even : odd);
}

// Work item e of a tile fill -> (row, chunk c).  A quarter-warp (8 threads) writes 8
// consecutive rows at one chunk; a warp covers 8 rows x the 4 chunks of a stage (the
// 128 contiguous bytes of each row's FP32 data).
__device__ __forceinline__ void tile_item(int e, int& row, int& c) {
  row = (e & 7) + 8 * (e >> 5);
  c = (e >> 3) & 3;
}

// The systems of tile rows [s0, s0 + NT) of k-point k: the k-point's active
// systems in order (all of them without a mask), -1 past the last.  Returns the
// number of active systems of the k-point.  One pass of the whole block per 256
// systems (a ballot per warp, the warps' counts through shared memory), so a
// launch waits for one load of the flags.  Contains barriers (whole block).
template <int NT>
__device__ int tile_systems(int* sys_s, int* wcnt, int sk, int n, const int* __restrict__ active, int s0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = threadIdx.x; j < NT; j += blockDim.x) sys_s[j] = -1;
  int base = 0;
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const bool a = j < n && (!active || active[sk + j] != 0);
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wcnt[warp] = __popc(m);
    __syncthreads();
    int before = base, total = base;
    for (int w = 0; w < nw; ++w) {
      before += w < warp ? wcnt[w] : 0;
      total += wcnt[w];
    }
    const int idx = before + __popc(m & ((1u << lane) - 1u));
    if (a && idx >= s0 && idx < s0 + NT) sys_s[idx - s0] = sk + j;
    __syncthreads();                                               // wcnt is rewritten by the next pass
    base = total;
  }
  __syncthreads();
  return base;
}

// The two-buffer stage loop shared by both kernels.  fetch(R, kb) loads the
// registers of the stage at K offset kb, store(R, buffer) splits them into a
// buffer; the loads of stage st + 2 are issued when stage st has been stored.
// Stages are numbered globally from gbase on (a CTA that runs several tiles
// continues the numbering, so that buffers and mbarrier phases stay in step);
// last holds the global index of the last stage whose MMAs were committed (-1
// if none) and is updated.  Returns whether every wait ended in time.
template <int NT, bool SWZ, typename Regs, typename Fetch, typename Store>
__device__ __forceinline__ bool stage_loop(unsigned char* sm, uint64_t* bar, uint32_t tmem, int nst, int kbase,
                                           int gbase, Fetch&& fetch, Store&& store, int& last) {
  using Lay = TcLayout<NT>;
  const int tid = threadIdx.x;
  Regs R0, R1;
  if (nst > 0) fetch(R0, kbase);
  if (nst > 1) fetch(R1, kbase + kTK);
  auto step = [&](Regs& r, int st) -> bool {
    const int g = gbase + st, b = g & 1;
    unsigned char* buf = sm + b * Lay::kStage;
    bool mine = true;
    if (g >= 2) mine = mbar_wait(&bar[b], ((g - 2) >> 1) & 1);     // MMAs of stage g - 2 (same buffer)
    tc_fence_after();
    store(r, buf);
    if (st + 2 < nst) fetch(r, kbase + (st + 2) * kTK);
    fence_async_smem();
    tc_fence_before();
    if (!__syncthreads_and(mine ? 1 : 0)) return false;            // uniform: no thread leaves alone
    if (tid == 0) {
      tc_fence_after();
      constexpr uint32_t id = idesc_bf16(NT);
      const uint32_t a = saddr(buf), bb = a + 3 * kAPiece;
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        const uint32_t off = kstep_off<SWZ>(kk);
        const uint64_t a0 = sdesc<SWZ>(a + off), a1 = sdesc<SWZ>(a + kAPiece + off),
                       a2 = sdesc<SWZ>(a + 2 * kAPiece + off);
        const uint64_t b0 = sdesc<SWZ>(bb + off), b1 = sdesc<SWZ>(bb + Lay::kBPiece + off),
                       b2 = sdesc<SWZ>(bb + 2 * Lay::kBPiece + off);
        const uint32_t first = (st | kk) ? 1u : 0u, corr = tmem + NT;
        mma_bf16(tmem, a0, b0, id, first);
        mma_bf16(corr, a0, b1, id, first);
        mma_bf16(corr, a1, b0, id, 1u);
        mma_bf16(corr, a0, b2, id, 1u);
        mma_bf16(corr, a1, b1, id, 1u);
        mma_bf16(corr, a2, b0, id, 1u);
      }
      mma_commit(&bar[b]);
    }
    last = g;
    return true;
  };
  bool ok = true;
  for (int st = 0; st < nst && ok; st += 2) {
    ok = step(R0, st);
    if (ok && st + 1 < nst) ok = step(R1, st + 1);
  }
  // the commit of the last stage completes after all earlier MMAs
  if (ok && nst > 0) ok = __syncthreads_and(mbar_wait(&bar[last & 1], (last >> 1) & 1) ? 1 : 0) != 0;
  return ok;
}

// a hint to bring the 128-byte line at p into L2 (the loads of a later stage then hit L2)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
constexpr int kPrefetch = 4;              // stages between an L2 prefetch and the loads of its stage

// common prologue: tensor-memory allocation and the two mbarriers
template <int NT>
__device__ __forceinline__ uint32_t tc_prologue(uint64_t* bar, uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, TcLayout<NT>::kCols);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}

// common end: on a failed wait, flag it and wait (bounded) for the MMAs in
// flight; then free the tensor memory
template <int NT>
__device__ __forceinline__ void tc_end(bool ok, int last, uint64_t* bar, uint32_t tmem, int* err) {
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    if (last >= 0) mbar_wait(&bar[last & 1], (last >> 1) & 1);
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TcLayout<NT>::kCols);
  }
}

// columns [c0, c0 + 16) of D for this thread's lane (row quarter w mod 4): the leading
// accumulator plus the correction accumulator NT columns further
template <int NT>
__device__ __forceinline__ void acc_cols16(uint32_t tmem, int c0, float* v) {
  const uint32_t a = tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)c0;
  float w[16];
  tmem_ld16(a, v);
  tmem_ld16(a + NT, w);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] += w[j];
}

}  // namespace

// Partial sums of C = V^H Y over one split-K chunk of `chunk` reals:
// part[(chunk index * nsys + s) * maxcnt + m] = (Re, Im) C[s][m] (the FP32 accumulator).
// grid: (A tiles, chunks, k-points x system tiles).
template <int NT, bool SWZ>
__global__ void __launch_bounds__(kThreads, 2)
    k_tc_coef(const float2* __restrict__ phi, const int* __restrict__ set_off, const int* __restrict__ set_cnt,
              const int* __restrict__ nb_k, const int* __restrict__ kstart, const int* __restrict__ kcount,
              const float2* __restrict__ Y, int ldy, int ld, int nnt, int chunk, int nsys, int maxcnt,
              const int* __restrict__ active, float2* __restrict__ part, int* __restrict__ err) {
  using Lay = TcLayout<NT>;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Lay::kBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + Lay::kSlot);
  int* sys_s = reinterpret_cast<int*>(sm + Lay::kSys);
  int* wcnt = reinterpret_cast<int*>(sm + Lay::kWcnt);
  const int tm = blockIdx.x, ch = blockIdx.y, k = blockIdx.z / nnt, tn = blockIdx.z - k * nnt;
  const int cnt = set_cnt[k], nb = nb_k[k];
  const int i0 = tm * kTM, s0 = tn * NT;
  const int k0 = ch * chunk, k1 = min(k0 + chunk, 2 * nb);
  if (i0 >= 2 * cnt || k0 >= k1) return;                         // uniform over the block
  const int nact = tile_systems<NT>(sys_s, wcnt, kstart[k], kcount[k], active, s0);
  if (nact <= s0) return;                                          // uniform
  const int nrow = min(NT, nact - s0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tmem = tc_prologue<NT>(bar, slot);

  // this thread's items: A (a vector, a chunk of 8 reals) and B (a system, a chunk);
  // with NT = 32 only the first 128 threads have a B item
  constexpr int kBN = NT * 4 / kThreads > 0 ? NT * 4 / kThreads : 1;
  int mo, ca;
  tile_item(tid, mo, ca);
  const float* vbase = reinterpret_cast<const float*>(phi + ((size_t)set_off[k] + i0 / 2) * ld);
  const float* pa = i0 / 2 + mo < cnt ? vbase + (size_t)mo * 2 * ld + 8 * ca : nullptr;
  const float* pb[kBN];
  int rb[kBN], cb[kBN];
#pragma unroll
  for (int j = 0; j < kBN; ++j) {
    tile_item(tid + kThreads * j, rb[j], cb[j]);
    const int s = rb[j] < NT ? sys_s[rb[j]] : -1;
    pb[j] = s >= 0 ? reinterpret_cast<const float*>(Y + (size_t)s * ldy) + 8 * cb[j] : nullptr;
  }
  struct Regs {
    float4 a[2], b[kBN][2];
  };
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fetch = [&](Regs& R, int kb) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {   // the vectors are zero past Nb_k: a group across 2 Nb_k needs no mask
      const int q = kb + 8 * ca + 4 * h;
      R.a[h] = pa && q < k1 ? *reinterpret_cast<const float4*>(pa + kb + 4 * h) : z4;
    }
#pragma unroll
    for (int j = 0; j < kBN; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = kb + 8 * cb[j] + 4 * h;
        R.b[j][h] = pb[j] && q < k1 ? *reinterpret_cast<const float4*>(pb[j] + kb + 4 * h) : z4;
        if (q + 2 >= k1) R.b[j][h].z = R.b[j][h].w = 0.f;          // second plane wave past Nb_k
      }
    // the rows' lines kPrefetch stages on (chunk 0 of a row starts its 128-byte line)
    const int kp = kb + kPrefetch * kTK;
    if (kp < k1) {
      if (pa && ca == 0) prefetch_l2(pa + kp);
#pragma unroll
      for (int j = 0; j < kBN; ++j)
        if (pb[j] && cb[j] == 0) prefetch_l2(pb[j] + kp);
    }
  };
  auto store = [&](Regs& R, unsigned char* buf) {
    // vector mo: row 2 mo = (Re, Im), row 2 mo + 1 = (-Im, Re) of the chunk's four plane waves
    const Pieces x = split8(R.a[0], R.a[1]);
    put_pair<SWZ>(buf, kAPiece, mo, ca, x, map_pairs(x, rot_pair));
#pragma unroll
    for (int j = 0; j < kBN; ++j)
      if (rb[j] < NT) put_pieces<SWZ>(buf + 3 * kAPiece, Lay::kBPiece, rb[j], cb[j], split8(R.b[j][0], R.b[j][1]));
  };
  int last = -1;
  const int nst = (k1 - k0 + kTK - 1) / kTK;
  const bool ok = stage_loop<NT, SWZ, Regs>(sm, bar, tmem, nst, k0, 0, fetch, store, last);
  if (ok) {
    tc_fence_after();
    // lanes 32 q .. 32 q + 31 of tensor memory are rows i0 + 32 q + lane of C^T; the two
    // warps of a quarter take the two halves of the columns
    const int q = warp & 3, half = warp >> 2;
    const int i = i0 + 32 * q + lane, m = i >> 1;
    const bool rowok = !(lane & 1) && i < 2 * cnt;
    float v[16];
#pragma unroll 1
    for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2) && c0 < nrow; c0 += 16) {   // uniform per warp
      acc_cols16<NT>(tmem, c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float im = __shfl_xor_sync(0xffffffffu, v[j], 1);
        if (rowok && c0 + j < nrow)
          part[((size_t)ch * nsys + sys_s[c0 + j]) * maxcnt + m] = make_float2(v[j], im);
      }
    }
  }
  tc_end<NT>(ok, last, bar, tmem, err);
}

// out[s][g] = alpha in[s][g] + beta sum_m v_m[g] coef32[s][m] (coef32: the FP32 coefficients at
// row stride ldc, even, zero past N_k), one work item = the plane waves
// of one 128-real tile (64 plane waves) of one k-point and NT systems; with dv,
// dpart[s * nparts + tile] = sum Re(conj(dv) out) over the tile (the chunking of the
// CUDA-core apply: 64 plane waves).  Persistent: a CTA keeps its tensor memory, mbarriers
// and system list and takes the items blockIdx.x, blockIdx.x + gridDim.x, ... (tile fastest,
// then k-point, then system tile), continuing the stage numbering from item to item.
template <int NT, bool SWZ>
__global__ void __launch_bounds__(kThreads, 2)
    k_tc_apply(const float2* __restrict__ phi, const int* __restrict__ set_off, const int* __restrict__ set_cnt,
               const int* __restrict__ nb_k, const int* __restrict__ kstart, const int* __restrict__ kcount,
               const float2* __restrict__ coef32, int ldc, const float2* in, float alpha, float beta,
               float2* out, int ldy, int ld, const float2* __restrict__ dv, double* __restrict__ dpart, int nparts,
               int nk, int nitems, const int* __restrict__ active, int* __restrict__ err) {
  using Lay = TcLayout<NT>;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Lay::kBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + Lay::kSlot);
  int* sys_s = reinterpret_cast<int*>(sm + Lay::kSys);
  int* wcnt = reinterpret_cast<int*>(sm + Lay::kWcnt);
  double* red = reinterpret_cast<double*>(sm + Lay::kRed);       // [NT][2] dot partials
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tmem = tc_prologue<NT>(bar, slot);
  constexpr int kBN = NT * 4 / kThreads > 0 ? NT * 4 / kThreads : 1;
  const int gla = tid & 63, ca = tid >> 6;
  const float2 z2 = make_float2(0.f, 0.f);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  int last = -1, gbase = 0, cur = -1, nact = 0;
  bool ok = true;
  for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
    const int tile = item % nparts, rest = item / nparts;
    const int k = rest % nk, tn = rest / nk;
    const int cnt = set_cnt[k], nb = nb_k[k];
    const int r0 = tile * kTM, s0 = tn * NT, g0 = r0 / 2;
    if (rest != cur) {                                             // uniform: the item's system list
      nact = tile_systems<NT>(sys_s, wcnt, kstart[k], kcount[k], active, s0);
      cur = rest;
    }
    if (nact <= s0) continue;                                      // uniform
    const int nrow = min(NT, nact - s0);
    if (r0 >= 2 * nb) {                                            // tile past Nb_k: define the dot partials
      if (dpart)
        for (int j = tid; j < nrow; j += kThreads) dpart[(size_t)sys_s[j] * nparts + tile] = 0.0;
      __syncthreads();                                             // sys_s may be rewritten by the next item
      continue;
    }
    // A item: plane wave gl of the tile and chunk ca (vectors 4 ca .. 4 ca + 3 of the stage);
    // consecutive threads take consecutive plane waves (coalesced loads).  B item: a system
    // and a chunk (its coefficients of the same four vectors).
    const float2* vk = phi + (size_t)set_off[k] * ld + g0;        // g0 + 63 < ld: ld is a multiple of 64
    struct Regs {
      float2 a[4];
      float4 b[kBN][2];
    };
    // (the B items' rows and chunks are recomputed where used: fewer live registers)
    auto fetch = [&](Regs& R, int kb) {
      const int mb = kb / 2;                                       // first vector of the stage
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = mb + 4 * ca + u;
        R.a[u] = m < cnt ? vk[(size_t)m * ld + gla] : z2;
      }
#pragma unroll
      for (int j = 0; j < kBN; ++j) {
        int r, c;
        tile_item(tid + kThreads * j, r, c);
        const int sj = r < NT ? sys_s[r] : -1;
        // coefficients m, m + 1 per 16 bytes (the copy is zero from N_k to its even stride)
        const float2* pc = coef32 + (size_t)(sj < 0 ? 0 : sj) * ldc + mb + 4 * c;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          R.b[j][h] = sj >= 0 && mb + 4 * c + 2 * h < ldc ? *reinterpret_cast<const float4*>(pc + 2 * h) : z4;
      }
      // the vectors' lines of a later stage (16 plane waves of 8 bytes per 128-byte line)
      const int mp = mb + kPrefetch * (kTK / 2);
      if ((gla & 15) == 0)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (mp + 4 * ca + u < cnt) prefetch_l2(vk + (size_t)(mp + 4 * ca + u) * ld + gla);
    };
    auto store = [&](Regs& R, unsigned char* buf) {
      // plane wave gl: row 2 gl = (Re v, -Im v), row 2 gl + 1 = (Im v, Re v) of the chunk's four vectors
      const Pieces x = split8(make_float4(R.a[0].x, R.a[0].y, R.a[1].x, R.a[1].y),
                              make_float4(R.a[2].x, R.a[2].y, R.a[3].x, R.a[3].y));
      put_pair<SWZ>(buf, kAPiece, gla, ca, map_pairs(x, conj_pair), map_pairs(x, swap_pair));
#pragma unroll
      for (int j = 0; j < kBN; ++j) {
        int r, cc;
        tile_item(tid + kThreads * j, r, cc);
        if (r >= NT) continue;
        put_pieces<SWZ>(buf + 3 * kAPiece, Lay::kBPiece, r, cc, split8(R.b[j][0], R.b[j][1]));
      }
    };
    const int nst = (2 * cnt + kTK - 1) / kTK;
    ok = stage_loop<NT, SWZ, Regs>(sm, bar, tmem, nst, 0, gbase, fetch, store, last);
    gbase += nst;
    if (!ok) break;                                                // uniform
    tc_fence_after();
    // D through shared memory (the ring is free now): Ds[j][r] for system column j and
    // tile row r = 2 g + c, so that every thread then takes whole plane waves of one system
    float* Ds = reinterpret_cast<float*>(sm);
    {
      const int q = warp & 3, half = warp >> 2;
      const int r = 32 * q + lane;
      float v[16];
#pragma unroll 1
      for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2) && c0 < nrow; c0 += 16) {   // uniform per warp
        if (nst > 0) {
          acc_cols16<NT>(tmem, c0, v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;                 // an empty set: V C = 0
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) Ds[(c0 + j) * kTM + r] = v[j];
      }
    }
    tc_fence_before();
    __syncthreads();
    // thread t: plane wave g0 + (t mod 64) of the systems t / 64, t / 64 + 4, ...; the loads of
    // 8 systems first (each element is read and written by this thread only)
    const int g = g0 + gla, j0 = tid >> 6;
    const bool gok = g < nb;
#pragma unroll 1
    for (int jb = j0; jb < NT; jb += 32) {
      float2 xin[8], w[8];
      int sv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = jb + 4 * u;
        sv[u] = gok && j < nrow ? sys_s[j] : -1;
        const size_t o = (size_t)(sv[u] < 0 ? 0 : sv[u]) * ldy + g;
        xin[u] = sv[u] >= 0 && alpha != 0.f ? in[o] : z2;
        w[u] = sv[u] >= 0 && dv ? dv[o] : z2;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = jb + 4 * u;
        const float2 dd = *reinterpret_cast<const float2*>(Ds + j * kTM + 2 * gla);
        float2 y = make_float2(beta * dd.x, beta * dd.y);
        if (alpha != 0.f) {
          y.x += alpha * xin[u].x;
          y.y += alpha * xin[u].y;
        }
        double d = 0.0;
        if (sv[u] >= 0) {
          out[(size_t)sv[u] * ldy + g] = y;
          d = (double)w[u].x * y.x + (double)w[u].y * y.y;
        }
        if (dpart) {                                               // the 64 plane waves of system j: 2 warps
          d = warp_sum(d);
          if (lane == 0) red[2 * j + ((tid >> 5) & 1)] = d;
        }
      }
    }
    if (dpart) {
      __syncthreads();
      for (int j = tid; j < nrow; j += kThreads) dpart[(size_t)sys_s[j] * nparts + tile] = red[2 * j] + red[2 * j + 1];
    }
    __syncthreads();                                               // Ds, red and sys_s are reused by the next item
  }
  tc_end<NT>(ok, last, bar, tmem, err);
}

// coef[s][m] = sum of the chunk partials, and its FP32 copy coef32[s][m] (row stride ldc,
// even; zero from N_k on) for the V C product.  Block (32, 8): threadIdx.x picks one of 32
// consecutive coefficients (coalesced loads of a chunk's partials), threadIdx.y = q sums the
// chunks q, q + 8, q + 16, ...; the eight sums are added in a fixed tree through shared
// memory, so the order is the same on every run.
__global__ void __launch_bounds__(256) k_tc_reduce(const float2* __restrict__ part, int nsys, int maxcnt, int chunk,
                                                   const int* __restrict__ sys_k, const int* __restrict__ set_cnt,
                                                   const int* __restrict__ nb_k, const int* __restrict__ active,
                                                   double2* __restrict__ coef, float2* __restrict__ coef32, int ldc) {
  __shared__ double2 sh[8][32];
  const long long t = (long long)blockIdx.x * 32 + threadIdx.x;
  const int q = threadIdx.y;
  bool sys_on = t < (long long)nsys * maxcnt, on = false;
  int s = 0, m = 0, nc = 0;
  if (sys_on) {
    s = (int)(t / maxcnt);
    m = (int)(t - (long long)s * maxcnt);
    sys_on = !active || active[s];
    on = sys_on && m < set_cnt[sys_k[s]];
    nc = (2 * nb_k[sys_k[s]] + chunk - 1) / chunk;
  }
  double ax = 0.0, ay = 0.0;
  if (on) {
    const size_t stride = (size_t)nsys * maxcnt;
    const float2* p = part + (size_t)s * maxcnt + m;
    int c = q;
    for (; c + 8 < nc; c += 16) {                                  // two loads in flight
      const float2 v0 = p[(size_t)c * stride], v1 = p[(size_t)(c + 8) * stride];
      ax += (double)v0.x;
      ay += (double)v0.y;
      ax += (double)v1.x;
      ay += (double)v1.y;
    }
    if (c < nc) {
      const float2 v = p[(size_t)c * stride];
      ax += (double)v.x;
      ay += (double)v.y;
    }
  }
  sh[q][threadIdx.x] = make_double2(ax, ay);
  __syncthreads();
  if (q == 0 && sys_on) {
    double sx = 0.0, sy = 0.0;
    if (on) {
      double2 r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = sh[u][threadIdx.x];
      sx = ((r[0].x + r[1].x) + (r[2].x + r[3].x)) + ((r[4].x + r[5].x) + (r[6].x + r[7].x));
      sy = ((r[0].y + r[1].y) + (r[2].y + r[3].y)) + ((r[4].y + r[5].y) + (r[6].y + r[7].y));
      coef[t] = make_double2(sx, sy);
    }
    coef32[(size_t)s * ldc + m] = make_float2((float)sx, (float)sy);
    if (m == maxcnt - 1 && ldc > maxcnt) coef32[(size_t)s * ldc + maxcnt] = make_float2(0.f, 0.f);
  }
}

// coef32[s][m] = (float) coef[s][m] for m < N_k of the system's k-point, 0 up to the even stride
// ldc (two coefficients per 16-byte load in k_tc_apply)
__global__ void k_tc_coef32(const double2* __restrict__ coef, int nsys, int maxcnt, int ldc,
                            const int* __restrict__ sys_k, const int* __restrict__ set_cnt,
                            const int* __restrict__ active, float2* __restrict__ coef32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nsys * ldc) return;
  const int s = (int)(t / ldc), m = (int)(t - (long long)s * ldc);
  if (active && !active[s]) return;
  const double2 v = m < set_cnt[sys_k[s]] ? coef[(size_t)s * maxcnt + m] : make_double2(0.0, 0.0);
  coef32[t] = make_float2((float)v.x, (float)v.y);
}

// ----------------------------------------------------------------- host --

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

namespace {

// system tile width: the most systems of one k-point a launch can find active
int tile_nt(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : 128); }

int sm_count() {
  int dev = 0;
  IKR_CUDA(cudaGetDevice(&dev));
  static int cached[64] = {};                                      // per device, read once
  if (dev < 64 && cached[dev] > 0) return cached[dev];
  int sms = 0;
  IKR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  sms = std::max(sms, 1);
  if (dev < 64) cached[dev] = sms;
  return sms;
}

// The kernel's shared memory, with the whole carveout for shared memory (two or three CTAs
// per SM; the L1 cache is not used by these kernels' operand traffic).  Every instance has a
// fixed size, so the attributes are set once per kernel and device.
template <typename K>
void smem_attrs(K kern, size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  IKR_CUDA(cudaGetDevice(&dev));
  const void* f = reinterpret_cast<const void*>(kern);
  {
    std::lock_guard<std::mutex> g(mu);
    for (const auto& e : done)
      if (e.first == f && e.second == dev) return;
  }
  IKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  IKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  std::lock_guard<std::mutex> g(mu);
  done.push_back({f, dev});
}

// the most systems of one k-point that a launch can find active: all of them without
// a mask, else also at most the bound the CG keeps (its count of active systems)
int active_bound(ikr_ctx* c, const SysList& L, const int* active) {
  int maxns = 0;
  for (int v : L.kcount) maxns = std::max(maxns, v);
  if (active && c->mask_bound > 0) maxns = std::min(maxns, c->mask_bound);
  return maxns;
}

}  // namespace

void proj_coef_tc(ikr_ctx* c, const SysList& L, const float2* Y, int ldy, const int* active, double2* coef,
                  const OrbSet& set) {
  IKR_REQUIRE(ldy % 2 == 0, IKR_ERR_ARG, "tensor-core projections need an even vector stride");
  int maxnb = 0;
  for (auto& K : c->k) maxnb = std::max(maxnb, K.nb);
  const int maxns = active_bound(c, L, active);
  if (maxns == 0 || L.n == 0) return;
  const int nk = (int)c->k.size();
  const int nmt = (2 * set.maxcnt + kTM - 1) / kTM;
  const int nt = tile_nt(maxns);
  const int nnt = (maxns + nt - 1) / nt;
  tc_flag_ready(c);
  auto launch = [&](auto kern, size_t smem) {
    smem_attrs(kern, smem);
    // split-K: chunks (multiples of a stage) of at most kMaxChunk reals (the length of the
    // FP32 sums).  Among the chunk counts that fill w = 1, 2, ... waves of two CTAs per SM, take
    // the one with the least time: waves x (stages per CTA + the CTA's fixed cost, about three
    // stages: the system scan, the first loads, the epilogue)
    const int slots = 2 * sm_count(), tiles = std::max(1, nk * nmt * nnt), K = 2 * maxnb;
    int chunk = 0;
    double best = 1e300;
    for (int w = 1; w <= 16; ++w) {
      const int want = std::max(1, w * slots / tiles);
      const int ch = std::max(kTK, ((K + want - 1) / want + kTK - 1) / kTK * kTK);
      if (ch > kMaxChunk && w < 16) continue;
      const int n = (K + ch - 1) / ch;
      const int waves = (n * tiles + slots - 1) / slots;
      const double cost = waves * (ch / (double)kTK + 3.0);
      if (cost < best) {
        best = cost;
        chunk = ch;
      }
    }
    const int nch = (K + chunk - 1) / chunk;
    c->ws.cpart.reserve((size_t)nch * L.n * set.maxcnt);            // doubles: room for float2 partials
    float2* part = reinterpret_cast<float2*>(c->ws.cpart.p);
    dim3 grid((unsigned)nmt, (unsigned)nch, (unsigned)(nk * nnt));
    kern<<<grid, kThreads, smem, c->stream>>>(set.phi32, set.off, set.cnt, c->d_nb.p, L.d_kstart.p, L.d_kcount.p,
                                              Y, ldy, c->ld, nnt, chunk, L.n, set.maxcnt, active, part, c->tc_err.p);
    IKR_CUDA(cudaGetLastError());
    const long long ncoef = (long long)L.n * set.maxcnt;
    const int ldc = (set.maxcnt + 1) & ~1;
    c->tc_coef32.reserve((size_t)L.n * ldc);
    k_tc_reduce<<<(unsigned)((ncoef + 31) / 32), dim3(32, 8), 0, c->stream>>>(part, L.n, set.maxcnt, chunk, L.d_k.p,
                                                                             set.cnt, c->d_nb.p, active, coef,
                                                                             c->tc_coef32.p, ldc);
    IKR_CUDA(cudaGetLastError());
    c->tc_coef32_of = coef;                                        // the FP32 copy is current
    c->tc_coef32_mask = active;
    c->tc_coef32_ldc = ldc;
    c->tc_coef32_n = L.n;
  };
  const bool swz = c->tc_swizzle;
  if (nt == 32) {
    if (swz) launch(k_tc_coef<32, true>, TcLayout<32>::kCoef);
    else launch(k_tc_coef<32, false>, TcLayout<32>::kCoef);
  } else if (nt == 64) {
    if (swz) launch(k_tc_coef<64, true>, TcLayout<64>::kCoef);
    else launch(k_tc_coef<64, false>, TcLayout<64>::kCoef);
  } else {
    if (swz) launch(k_tc_coef<128, true>, TcLayout<128>::kCoef);
    else launch(k_tc_coef<128, false>, TcLayout<128>::kCoef);
  }
}

void proj_apply_tc(ikr_ctx* c, const SysList& L, const double2* coef, const float2* in, float alpha, float beta,
                   float2* out, int ldy, const float2* dv, double* dpart, const int* active, const OrbSet& set) {
  const int maxns = active_bound(c, L, active);
  if (maxns == 0 || L.n == 0) return;
  const int nparts = (c->ld + 63) / 64;                           // 64 plane waves per tile and dot partial
  const int nt = tile_nt(maxns);
  const int nnt = (maxns + nt - 1) / nt;
  const int nk = (int)c->k.size();
  const int nitems = nparts * nk * nnt;
  tc_flag_ready(c);
  const int ldc = (set.maxcnt + 1) & ~1;
  // the FP32 copy of the coefficients: from the tensor-core V^H Y that produced them, else made here
  if (!(coef == c->tc_coef32_of && active == c->tc_coef32_mask && ldc == c->tc_coef32_ldc &&
        L.n == c->tc_coef32_n)) {
    c->tc_coef32.reserve((size_t)L.n * ldc);
    const long long n = (long long)L.n * ldc;
    k_tc_coef32<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(coef, L.n, set.maxcnt, ldc, L.d_k.p, set.cnt,
                                                                      active, c->tc_coef32.p);
    IKR_CUDA(cudaGetLastError());
    c->tc_coef32_of = nullptr;
  }
  // persistent: two CTAs per SM (or one per item)
  const dim3 grid((unsigned)std::min(nitems, 2 * sm_count()));
  auto launch = [&](auto kern, size_t smem) {
    smem_attrs(kern, smem);
    kern<<<grid, kThreads, smem, c->stream>>>(set.phi32, set.off, set.cnt, c->d_nb.p, L.d_kstart.p, L.d_kcount.p,
                                              c->tc_coef32.p, ldc, in, alpha, beta, out, ldy, c->ld, dv, dpart,
                                              nparts, nk, nitems, active, c->tc_err.p);
    IKR_CUDA(cudaGetLastError());
  };
  const bool swz = c->tc_swizzle;
  if (nt == 32) {
    if (swz) launch(k_tc_apply<32, true>, TcLayout<32>::kApply);
    else launch(k_tc_apply<32, false>, TcLayout<32>::kApply);
  } else if (nt == 64) {
    if (swz) launch(k_tc_apply<64, true>, TcLayout<64>::kApply);
    else launch(k_tc_apply<64, false>, TcLayout<64>::kApply);
  } else {
    if (swz) launch(k_tc_apply<128, true>, TcLayout<128>::kApply);
    else launch(k_tc_apply<128, false>, TcLayout<128>::kApply);
  }
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
