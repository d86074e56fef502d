// Declarations of the kernel wrappers in fft.cu and ops.cu.
#pragma once

#include "context.hpp"

namespace ikr {

template <typename T> struct CgVecs {
  C_t<T>* X;
  C_t<T>* R;
  C_t<T>* P;
  C_t<T>* Z;
  C_t<T>* W;
  const C_t<T>* B;
};

// fft.cu
template <typename R>
void launch_z_inverse(ikr_ctx* c, const SysList& L, const C_t<R>* sphere, int ld, const int* active,
                      C_t<R>* b1, const int* list = nullptr, int nlist = 0);
template <typename R>
void launch_plane(ikr_ctx* c, const SysList& L, const C_t<R>* b1, const R* pot, const double* pot_scale,
                  const int* active, C_t<R>* b4, const C_t<R>* real_in = nullptr, const int* list = nullptr,
                  int nlist = 0);
template <typename R> void launch_synth_planes(ikr_ctx* c, int nsys, const C_t<R>* b1, C_t<R>* out);
// the swizzled double-float plane pass of 48 x 48 planes (fft_plane.cu); false when
// the grid has another plane shape or the context turned it off
bool launch_plane_sw(ikr_ctx* c, int nsys, const double2* b1, const double* pot, const double* pot_scale,
                     const int* active, double2* b4, const double2* real_in);
template <typename R>
bool launch_plane_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, const typename io<R>::real* pot,
                       const double* pot_scale, const int* active, typename io<R>::cx* b4,
                       const typename io<R>::cx* real_in);
constexpr int kZC = 32;        // columns per block of the one-thread-per-column z-pass
// FP32 z-pass with one thread per column (fft_reg.cu); false: not covered
bool z_reg_ok(ikr_ctx* c);
int z_reg_chunks(ikr_ctx* c);
bool launch_z_inverse_reg(ikr_ctx* c, int nsys, const int* d_k, const float2* sphere, int ld, const int* active,
                          const int* list, float2* b1);
bool launch_z_forward_reg(ikr_ctx* c, int nsys, const int* d_k, const float2* b4, float2* out, int ld,
                          const float2* psi, const double* shift, const float* kin, const int* active,
                          const int* list, double* dpart);
// FP32 plane pass with one thread per line (fft_reg.cu); false: shape not covered
// list: the nlist systems to process (a compacted active set), else all nsys under `active`
bool launch_plane_reg(ikr_ctx* c, int nsys, const float2* b1, const float* pot, const double* pot_scale,
                      const int* active, float2* b4, const float2* real_in, const int* list, int nlist);
template <typename R>
void launch_z_forward(ikr_ctx* c, const SysList& L, const C_t<R>* b4, C_t<R>* out, int ld,
                      const C_t<R>* psi, const double* shift, bool kinetic, const int* active,
                      double* dpart = nullptr, const int* list = nullptr, int nlist = 0);
int zf_chunks(ikr_ctx* c);    // dot partials per system written by launch_z_forward (largest)
int zf_chunks(ikr_ctx* c, int fp_bytes);   // ... by the launch of that precision
// Real-space planes of sphere vectors by the compile-time kernel (fft_plane.cu); false: not covered
template <typename R>
bool launch_synth_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1, typename io<R>::cx* out);
// Density partial planes by the compile-time kernel (fft_plane.cu) into
// c->ws.dens_part; *ngroups = the number of partial planes.  false: shape not covered.
template <typename R>
bool launch_density_fast(ikr_ctx* c, int nsys, const typename io<R>::cx* b1d, const typename io<R>::cx* psir,
                         const double* ca, const double* cb, int* ngroups);
int density_groups(ikr_ctx* c, int nsys, int per_sm);
template <typename R>
void launch_density(ikr_ctx* c, int nsys, const C_t<R>* b1phi, const C_t<R>* b1d,
                    const double* coef_a, const double* coef_b, double* out, double scale,
                    const C_t<R>* psi_real = nullptr);
template <typename R>
void to_plane_layout(ikr_ctx* c, const double* in, R* out, double scale, const double* dscale);
void full_fft(ikr_ctx* c, double2* data, bool inverse);
// |psi_s|^2 and (Re e^{-i theta_s} psi_s)^2 summed over the orbitals, theta_s of
// the most-real gauge (rot: nsys scratch entries, receives (cos, sin) theta_s)
void orbital_sq_sums(ikr_ctx* c, const double2* psir, int nsys, double* abs2, double* re2, double2* rot);

template <typename R> const R* kin_all_ptr(ikr_ctx* c);
template <> inline const double* kin_all_ptr<double>(ikr_ctx* c) { return c->d_kin_all.p; }
template <> inline const float* kin_all_ptr<float>(ikr_ctx* c) { return c->d_kin_all32.p; }

// A set of orthonormal vectors per k-point for the projections, stored like the
// occupied orbitals: vector j of k-point k at (off[k] + j) * ld, cnt[k] of them.
// The projections use the occupied orbitals Phi_k unless another set is given.
struct OrbSet {
  const double2* phi = nullptr;
  const float2* phi32 = nullptr;
  const int* off = nullptr;     // device, one per k-point
  const int* cnt = nullptr;     // device, one per k-point
  int maxcnt = 0;
};
OrbSet occ_set(ikr_ctx* c);     // Phi_k
OrbSet schur_set(ikr_ctx* c);   // [Phi_k Psi_k]: the occupied and the extra computed bands
OrbSet extra_set(ikr_ctx* c);   // Psi_k
OrbSet kb_set(ikr_ctx* c);      // the Kleinman-Bylander projectors B_k (kb.cu)

// ops.cu
// Fused FP32 CG update after the H_k application (cg_fused.cu): false when the
// shape does not fit a thread-block cluster per k-point (then nothing is launched)
// set: project z on the complement of this orbital set (default: Phi_k)
bool launch_cg_fused(ikr_ctx* c, const SysList& L, float2* X, float2* Rv, float2* P, const float2* W, double* sys,
                     int maxit, int* active, int* counter, int* list, const double* zpart, int nzf,
                     const OrbSet* set = nullptr);
// the cluster size the fused update would launch with for sets of up to maxcnt vectors (0: none)
int cg_fused_cluster(ikr_ctx* c, const SysList& L, int maxcnt);
// FP32 projections (proj32.cu)
int proj_chunks32();
void proj_coef32(ikr_ctx* c, const SysList& L, const float2* Y, int ldy, const int* active, double2* coef,
                 const OrbSet& set);
void proj_apply32(ikr_ctx* c, const SysList& L, const double2* coef, const float2* in, float alpha, float beta,
                  float2* out, int ldy, const float2* dv, double* dpart, const int* active, const OrbSet& set);
// Tensor-core projection products (tc_proj.cu): the FP32 V^H Y of proj_coef32
// and Y - V C of proj_apply32 by tcgen05 MMAs
bool tc_proj_ok(ikr_ctx* c, const OrbSet& set);
void proj_coef_tc(ikr_ctx* c, const SysList& L, const float2* Y, int ldy, const int* active, double2* coef,
                  const OrbSet& set);
void proj_apply_tc(ikr_ctx* c, const SysList& L, const double2* coef, const float2* in, float alpha, float beta,
                   float2* out, int ldy, const float2* dv, double* dpart, const int* active, const OrbSet& set);
void tc_check(ikr_ctx* c);    // IKR_ERR_TIMEOUT if a tensor-core launch gave up on a wait
int proj_chunks(ikr_ctx* c);                  // the largest count (workspace sizing)
int proj_chunks(ikr_ctx* c, int fp_bytes);    // dot partials per system written by proj_apply
int cg_chunks(ikr_ctx* c);
// coef[s][m] = <v_m, y_s> for the vectors v of `set` (default: Phi_k), stride set->maxcnt
template <typename R>
void proj_coef(ikr_ctx* c, const SysList& L, const C_t<R>* Y, int ldy, const int* active, double2* coef,
               const OrbSet* set = nullptr);
// out = alpha in + beta sum_m v_m coef[s][m] (and the dot partials with dv)
template <typename R>
void proj_apply(ikr_ctx* c, const SysList& L, const double2* coef, const C_t<R>* in, R alpha, R beta,
                C_t<R>* out, int ldy, const C_t<R>* dv, double* dpart, const int* active,
                const OrbSet* set = nullptr);
void sys_reduce(ikr_ctx* c, const double* part, int nparts, int nsys, const int* active, double* out);
template <typename R>
void cg_xr(ikr_ctx* c, const SysList& L, int mode, CgVecs<R>& v, const double* sys, const int* active,
           double* dpart);
template <typename R>
void cg_p(ikr_ctx* c, const SysList& L, int mode, CgVecs<R>& v, const double* sys, const int* active);
void cg_scalars(ikr_ctx* c, int stage, double* sys, const double* part, int nparts, int nsys, int maxit,
                int* active, int* counter, int* list = nullptr);
void count_active(ikr_ctx* c, const int* active, int n, int* dout);
void chi0_sys(ikr_ctx* c, const SysList& L, const double2* M, double* deps, double2* coefP);
// a[s][j] /= lambda_j - shift[s] for the extra bands j of k_s (stride c->xmax)
void deflate_coef(ikr_ctx* c, const SysList& L, double2* a, const double* shift);
void occupation_response(ikr_ctx* c, const double* deps, double* coef_a, double* coef_b, double* deF);
void apply_K(ikr_ctx* c, const double* v, double* Kv, double* d_norm);
void apply_kerker(ikr_ctx* c, const double* v, double* Tv, double alpha);
void norm2(ikr_ctx* c, const double* x, double* d_out3);
void axpy(ikr_ctx* c, const double* x, const double* y, double sa, const double* da, double* out);
void scale_by(ikr_ctx* c, const double* w, const double* dinv, double* out);
void multidot(ikr_ctx* c, const double* V, int nv, const double* w, double* h, int accumulate);
void sub_combination(ikr_ctx* c, const double* V, int nv, const double* h, double* w);
void add_combination(ikr_ctx* c, const double* V, int nv, const double* y, const double* x0, double* x);
void exchange_kernel(ikr_ctx* c);
void grid_max(ikr_ctx* c, const double* v, size_t n, double* dout);
void to_fp32(ikr_ctx* c, const double2* in, size_t n, float2* out);
void to_fp64(ikr_ctx* c, const float2* in, size_t n, double2* out);

// measured arithmetic throughput of the current device (peaks.cu): out[0] SMs,
// [1] FP32 FMA TFLOP/s, [2] FP64 FMA TFLOP/s, [3] FP32 and [4] double-float radix-4
// butterfly TFLOP/s, [5] the device's reported maximum SM clock in MHz
void device_peaks(double* out, cudaStream_t st);

}  // namespace ikr
