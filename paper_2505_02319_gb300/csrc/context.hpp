// Host-side context of the library and the internal entry points shared by
// the translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ikr.h"
#include "common.cuh"

namespace ikr {

struct Error : std::runtime_error {
  ikr_status status;
  Error(ikr_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define IKR_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      throw ::ikr::Error(e_ == cudaErrorMemoryAllocation ? IKR_ERR_OOM : IKR_ERR_CUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));            \
    }                                                                                    \
  } while (0)

#define IKR_REQUIRE(cond, status, msg)                  \
  do {                                                  \
    if (!(cond)) throw ::ikr::Error((status), (msg));  \
  } while (0)

// Device buffer owned by the context.
template <typename T> struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // ensure capacity >= count elements (contents are not preserved)
  void reserve(size_t count) {
    if (count <= n) return;
    release();
    IKR_CUDA(cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 16));
    n = count;
  }
};

// Per-k-point data.
struct KPoint {
  int nb = 0;                   // basis size Nb_k
  double kfrac[3] = {0, 0, 0};
  double weight = 0.0;
  std::vector<int> miller;      // nb x 3 signed Miller triples (lexicographic)
  std::vector<double> kin;      // |k+G|^2 / 2
  std::vector<int> colinfo;     // per union column: {sphere offset, count, z start position}
  // ground state
  int nbands = 0, nocc = 0;
  std::vector<double> eps, f, fp;  // nbands each
  double rownorm = 0.0;         // ||F_k^-1 Phi_k||_{2,inf}
  double rownorm_re = 0.0;      // ||Re F_k^-1 Phi_k||_{2,inf}
};

// One batch of Sternheimer-type systems (k-point, band), grouped by k.
struct SysList {
  int n = 0;
  std::vector<int> k, band;     // host
  std::vector<int> kstart, kcount;  // per k-point: first system and count
  DBuf<int> d_k, d_band, d_kstart, d_kcount;
};

struct Workspace {
  // FFT intermediates [s][iz][column] (complex, FP64 sized; the FP32 path reuses them)
  DBuf<double2> b1, b4, b1b;
  // CG state and chi0 vectors (complex, stride ld), FP64
  DBuf<double2> X, R, P, Z, W, B, Y;
  // FP32 CG state
  DBuf<float2> X32, R32, P32, Z32, W32, B32;
  // projection coefficients (n x noccmax complex, stored as 2 doubles)
  DBuf<double> cpart;           // per-chunk partial sums of Phi^H Y
  DBuf<double> coef, coefM, coefP;
  DBuf<double> coefX;           // Psi^H b of the Schur-complement solves (n x xmax complex)
  DBuf<double> xshift;          // per-system shifts eps_s of the Schur-complement solves
  DBuf<double> dpart;           // per-system partial dot products
  DBuf<double> sys;             // per-system CG scalars (see SysField)
  DBuf<double> val;             // per-system reduced dot products
  DBuf<int> active;
  DBuf<int> alist;              // compacted indices of the active CG systems
  DBuf<double2> kbc;            // B^H x of the nonlocal products
  DBuf<double> deps, ca, cb;    // deps_s and the density coefficients
  DBuf<double> rn;              // per-system residual norms (mixed precision)
  DBuf<double> grid1, grid2, grid3, grid4, grid5, grid6;   // Ng-sized real scratch
  DBuf<double2> cgrid;          // Ng complex scratch (full-grid FFTs)
  DBuf<double> dens_part;       // density partial planes
  DBuf<double> scal;            // a few device scalars
  DBuf<double> gm_V;            // GMRES basis (m+1) x Ng
  DBuf<double> gm_h;            // Arnoldi coefficients and partials
  // lockstep right-hand sides (batch.cu): per item the potential, density and
  // norms, the right-hand sides and solutions of its systems, Phi^H Y, the
  // dphi^P coefficients and deps; per right-hand side the Krylov basis and three vectors
  DBuf<double> bu, bdrho, bnrm, bM, bCP, bdeps, bgm;
  DBuf<double2> bB, bX;
  // tensor-core projections: the active systems of every k-point in order, and their counts
  DBuf<int> tc_list, tc_cnt;
};

// offsets into the per-system scalar block (nsys doubles each)
enum SysField {
  kSysShift = 0,    // eps_n (the Sternheimer shift)
  kSysKappa,        // preconditioner constant
  kSysTol2,         // tolerance squared
  kSysRz,           // <r, z>
  kSysAlpha,
  kSysBeta,
  kSysRr,           // ||r||^2
  kSysPap,          // <p, A p>
  kSysIters,
  kSysStatus,       // 0 running, 1 converged, 2 numeric failure, 3 cap
  kSysFields
};

// Kernel classes for launch counting and optional CUDA-event timing.
enum KernelClass {
  kKidZInv = 0,     // k_z_inverse: sphere scatter + inverse z-FFT
  kKidPlane,        // k_plane: y/x FFTs, potential product, x/y FFTs
  kKidZFwd,         // k_z_forward: forward z-FFT + sphere gather (+ kinetic)
  kKidProjCoef,     // Phi^H Y (partials + fixed-order reduction)
  kKidProjApply,    // Y -/+ Phi C (+ fused dot partials)
  kKidCgVec,        // CG vector updates
  kKidDensity,      // density accumulation + transpose
  kKidGridFFT,      // full-grid FFT passes (K^H, Kerker)
  kKidGridOps,      // grid-sized elementwise / reductions / Arnoldi
  kKidScalar,       // per-system scalar kernels
  kNumKid
};

struct Profiler {
  unsigned mask = 0;                    // bit i: time class i with CUDA events
  long long launches[kNumKid] = {};
  long long units32[kNumKid] = {};      // work units (systems) launched in FP32
  long long units64[kNumKid] = {};      // ... and in FP64
  std::vector<cudaEvent_t> ev[2 * kNumKid];   // [class] FP32 calls, [kNumKid + class] FP64 calls
  size_t used[2 * kNumKid] = {};
};

}  // namespace ikr

namespace ikr {
}  // namespace ikr

struct ikr_ctx {
  std::string err;
  int N[3] = {0, 0, 0};
  int nsm = 152;                // streaming multiprocessors of the device
  double vmax = 0.0;            // largest value of the local potential V(r)
  size_t Ng = 0;
  double lattice[9];            // columns are cell vectors
  double recip[9];              // columns are b_i
  double volume = 0.0;
  double Ecut = 0.0;
  double T = 0.0;
  int nel = 0;
  std::vector<ikr::KPoint> k;
  int ld = 0;                   // padded stride of orbital-sized vectors
  // union of the sphere columns (j1, j2) over all k-points
  int nc = 0, ncp = 0;
  std::vector<int> col_ix, col_iy;
  ikr::DBuf<int> d_col_xy;      // 2 per column: grid positions ix, iy
  int nxa = 0;
  std::vector<int> xpos;        // active x positions
  ikr::DBuf<int> d_xpos;
  // one-thread-per-line plane pass: 3 per active x position, ordered by
  // (x + N0/2) mod N0: that shifted position, the first y of the column's
  // cyclic y-interval and the interval length - 1; bit x of xmask = x active
  ikr::DBuf<int> d_xr;
  unsigned long long xmask = 0;
  bool reg_plane_ok = false;    // every active column's y-set is one cyclic interval
  bool xr_contig = false;       // the shifted active x positions are pxlo, pxlo + 1, ..., pxlo + nxa - 1
  int pxlo = 0;
  bool plane_sw = true;         // swizzled double-float plane pass of 48 x 48 planes (IKR_PLANE_SW=0: off)
  int plane_rc = 5;             // compact FP32 plane kernel at 5 (or 4) blocks per SM; 0: the full-plane one
  // one-thread-per-column z-pass: per k, nc + 1 prefix sums of the column
  // counts (= the sphere offsets of the columns); zspan = the largest sphere
  // slice of kZC consecutive columns
  ikr::DBuf<int> d_colpre;
  int zspan = 0;
  bool zreg_ok = false;
  // launch plan of the fused FP32 CG update (cg_fused.cu), for cgf_nsmax systems per k-point
  int cgf_nsmax = -1, cgf_maxcnt = -1, cgf_cs = 0, cgf_sl = 0, cgf_lds = 0;
  int cgf_force = 0;            // cluster size chosen by the autotuner (0: the planner's choice)
  int cgf_planned_force = -1;   // cgf_force of the cached plan
  size_t cgf_smem = 0;
  bool cgf_ok = false;
  ikr::FftPlan plan[3];
  ikr::DBuf<double2> d_tw[3];
  ikr::DBuf<float2> d_tw32[3];
  ikr::DBuf<double> d_V;        // potential, C order
  ikr::DBuf<double> d_Vt;       // potential / Ng in plane layout [i3][i2][i1]
  ikr::DBuf<float> d_Vt32;
  ikr::DBuf<int> k_colinfo;     // nk x nc x 3: sphere offset, count, z start of every column
  ikr::DBuf<double> d_kin_all;  // nk x ld kinetic energies |k+G|^2/2
  ikr::DBuf<float> d_kin_all32;
  ikr::DBuf<int> d_nb;          // nk basis sizes
  ikr::DBuf<double> d_coul;     // 4 pi/|G|^2 / Ng (G = 0 -> 0), C order
  ikr::DBuf<double> d_G2;       // |G|^2 of every grid frequency, C order
  double knorm = 0.0;           // ||K|| = max_G 4 pi/|G|^2 + max_r |K^xc(r)| (bound, set with the ground state)
  // ground state
  bool have_gs = false;
  double eF = 0.0;
  ikr::DBuf<double> d_rho, d_kxc;
  ikr::DBuf<double2> d_b1phi;   // z-transformed occupied orbitals [s][iz][c]
  ikr::DBuf<float2> d_b1phi32;
  ikr::DBuf<double2> d_psir;    // real-space planes of the occupied orbitals [s][iz][iy][ix] (unnormalised)
  ikr::DBuf<float2> d_psir32;
  ikr::SysList occ;             // all occupied (k, n) in k-major order
  int noccmax = 0;
  // Kleinman-Bylander nonlocal part (kb.cu): nproj projectors per k-point,
  // block k at k * nproj * ld (projector j at j * ld within it), and the couplings
  int nproj = 0;
  double kb_dmax = 0.0;         // the largest coupling D_j
  ikr::DBuf<double2> d_kb;
  ikr::DBuf<float2> d_kb32;
  ikr::DBuf<double> d_kbD;
  ikr::DBuf<int> d_kboff, d_kbcnt;   // the projectors as a vector set: row k nproj + j, nproj per k
  ikr::DBuf<float4> d_psir_df; // the real-space orbital planes as double-float (x.hi, x.lo, y.hi, y.lo)
  ikr::DBuf<double2> d_phi_all; // occupied orbitals, vector s of occ at s * ld (complex128)
  ikr::DBuf<float2> d_phi_all32;
  ikr::DBuf<int> d_phi_off;     // nk: index of the first occupied orbital of k
  ikr::DBuf<int> d_nocc;        // nk
  ikr::DBuf<int> d_occ_kstart;  // == d_phi_off
  ikr::DBuf<double> d_eps_occ, d_f_occ, d_fp_occ, d_w_occ, d_kappa_occ;  // per occupied system
  // Schur-complement Sternheimer solves (ikr_set_schur): per k-point the occupied
  // orbitals followed by the extra computed bands Psi_k (nbands - N_occ,k of them),
  // vector j of k at (roff[k] + j) * ld; Psi_k starts at xoff[k] = roff[k] + N_occ,k.
  // reps holds the eigenvalue of every stored vector (same index).
  bool schur = false;
  // system list of the batched CG over `batch_items` E applications (batch.cu),
  // and the position of each of its systems in the per-item blocks
  int batch_items = -1;
  // tensor-core projection coefficients (tc_proj.cu; ikr_set_tensor_cores)
  bool tc_proj = false;
  bool tc_swizzle = true;       // 64-byte swizzled operand tiles (false: the canonical layout)
  int mask_bound = 0;           // > 0: at most this many systems are active in masked FP32 projections (CG)
  ikr::DBuf<int> tc_err;
  ikr::DBuf<float2> tc_coef32;  // FP32 copy of the coefficients of a tensor-core V C product
  // the coefficient buffer (and mask, stride) whose FP32 copy tc_coef32 holds: written by the
  // tensor-core V^H Y together with the FP64 result, cleared by every other writer
  const double2* tc_coef32_of = nullptr;
  const int* tc_coef32_mask = nullptr;
  int tc_coef32_ldc = 0, tc_coef32_n = 0;
  ikr::SysList batch_list;
  ikr::DBuf<int> d_batch_map;
  int rmax = 0, xmax = 0;
  ikr::DBuf<double2> d_rset;
  ikr::DBuf<float2> d_rset32;
  ikr::DBuf<int> d_roff, d_rcnt, d_xoff, d_xcnt;
  ikr::DBuf<double> d_reps;
  std::vector<double> h_kappa_occ;
  int* h_pinned = nullptr;      // pinned host scratch: 64 ints, then doubles
  double* h_pinned_d = nullptr;
  size_t pinned_bytes = 0;
  ikr::Profiler prof;
  int active_hint = 0;          // systems active in the next masked launch (for accounting)
  bool emulate_fp64 = false;    // FP64 plane passes in double-float on the FP32 units (mixed path)
  ~ikr_ctx() {
    if (h_pinned) cudaFreeHost(h_pinned);
    for (auto& v : prof.ev)
      for (auto e : v) cudaEventDestroy(e);
  }
  ikr::Workspace ws;
  cudaStream_t stream = 0;
};

namespace ikr {

// Counts the launches of a wrapper and, if its class is selected, brackets
// them with CUDA events on the context's stream.
struct ProfScope {
  ikr_ctx* c;
  int id;
  bool timed;
  ProfScope(ikr_ctx* c_, int id_, int nlaunch, long long units = 0, int fp_bytes = 8) : c(c_), id(id_) {
    c->prof.launches[id] += nlaunch;
    if (fp_bytes == 4) c->prof.units32[id] += units;
    else c->prof.units64[id] += units;
    timed = (c->prof.mask >> id) & 1u;
    if (fp_bytes != 4) id += kNumKid;
    if (timed) record();
  }
  ~ProfScope() {
    if (timed) record();
  }
  void record() {
    auto& v = c->prof.ev[id];
    size_t& u = c->prof.used[id];
    if (u == v.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        timed = false;
        return;
      }
      v.push_back(e);
    }
    cudaEventRecord(v[u++], c->stream);
  }
};

// setup.cu
void setup_system(ikr_ctx* c, const ikr_system* sys);
void set_eigenpairs(ikr_ctx* c, const ikr_eigenpairs* eig);
void make_syslist(ikr_ctx* c, SysList& L, int nsys, const int* kof, const int* band);
}  // namespace ikr
