// Batched transforms between the orbital spheres G_k and the real-space grid
// X (eq. fft_ifft):
//   F^{-1} c (r) = |Omega|^{-1/2} sum_{G in G_k} c_G e^{iG.r},
//   F x (G)      = |Omega|^{1/2} / Ng sum_r x_r e^{-iG.r}.
// A product F(v . F^{-1} c) therefore carries the factor 1/Ng, which the
// callers fold into the potential.
//
// Layout of one batch of systems s (each with its own k-point and sphere):
//   z-pass   (k_z_inverse / k_z_forward): one line per sphere column (j1, j2)
//            of the union of all spheres; the ball meets each column in one
//            contiguous z-interval, so the scatter/gather is a contiguous
//            copy.  Output/input buffer b1/b4[s][iz][c].
//   plane    (k_plane): one CTA per (s, iz) keeps the whole Ny x Nx plane in
//            shared memory: y-lines of the active x positions, x-lines of all
//            rows, the pointwise product with the potential, and back.
// Only the columns and x positions that the spheres touch are transformed
// (pruned FFT); the grid never goes through global memory.
#include "ops.hpp"

namespace ikr {

// shared memory a block may use on sm_103a, and the error for a plane of a grid
// with no compiled shape that does not fit (the runtime-size plane kernel keeps
// the whole Ny x Nx plane twice)
constexpr size_t kMaxPlaneSmem = 227 * 1024;
static std::string plane_smem_message(const ikr_ctx* c, size_t smem) {
  return "the " + std::to_string(c->N[0]) + " x " + std::to_string(c->N[1]) +
         " grid plane has no compiled kernel shape and needs " + std::to_string(smem) +
         " bytes of shared memory, more than the " + std::to_string(kMaxPlaneSmem) + " a block may use";
}


namespace {

template <typename R> const C_t<R>* tw_ptr(ikr_ctx* c, int axis);
template <> const double2* tw_ptr<double>(ikr_ctx* c, int axis) { return c->d_tw[axis].p; }
template <> const float2* tw_ptr<float>(ikr_ctx* c, int axis) { return c->d_tw32[axis].p; }

template <typename F> void set_smem(F* f, size_t bytes) {
  IKR_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

inline int lines_per_cta(int n) { return n <= 64 ? 16 : (n <= 128 ? 8 : 4); }

}  // namespace

// ------------------------------------------------------------------ z-pass --

// R is the arithmetic type; global arrays hold its storage type io<R>
// (double2 for the double-float passes of the mixed path), converted on load
// and store.
template <typename R>
__global__ void __launch_bounds__(256) k_z_inverse(const typename io<R>::cx* __restrict__ sphere, int ld,
                                                   const int* __restrict__ sys_k,
                                                   const int* __restrict__ colinfo, int nc, int ncp,
                                                   FftPlan pz, const typename io<R>::cx* __restrict__ twz,
                                                   const int* __restrict__ active, int LZ,
                                                   typename io<R>::cx* __restrict__ b1) {
  using C = C_t<R>;
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nz = pz.n, lds = Nz + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* A = tw + Nz;
  C* B = A + LZ * lds;
  const int k = sys_k[s];
  const int c0 = blockIdx.x * LZ;
  for (int i = threadIdx.x; i < Nz; i += blockDim.x) tw[i] = to_c<C>(twz[i]);
  const typename io<R>::cx* src = sphere + (size_t)s * ld;
  for (int idx = threadIdx.x; idx < LZ * Nz; idx += blockDim.x) {
    const int l = idx / Nz, z = idx - l * Nz;
    const int col = c0 + l;
    C v = mk<C>(R(0), R(0));
    if (col < nc) {
      const int* inf = colinfo + ((size_t)k * nc + col) * 3;
      int t = z - inf[2];
      if (t < 0) t += Nz;
      if (t < inf[1]) v = to_c<C>(src[inf[0] + t]);
    }
    A[l * lds + z] = v;
  }
  __syncthreads();
  C* res = fft_lines<C, true>(A, B, pz, LZ, lds, nullptr, 1, tw);
  typename io<R>::cx* dst = b1 + (size_t)s * Nz * ncp;
  for (int idx = threadIdx.x; idx < LZ * Nz; idx += blockDim.x) {
    const int iz = idx / LZ, l = idx - iz * LZ;
    const int col = c0 + l;
    if (col < nc) dst[(size_t)iz * ncp + col] = from_c(res[l * lds + iz]);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_z_forward(const typename io<R>::cx* __restrict__ b4, int nc, int ncp,
                                                   const int* __restrict__ sys_k,
                                                   const int* __restrict__ colinfo, FftPlan pz,
                                                   const typename io<R>::cx* __restrict__ twz, int LZ,
                                                   typename io<R>::cx* __restrict__ out, int ld, int ldk,
                                                   const typename io<R>::cx* __restrict__ psi,
                                                   const double* __restrict__ shift,
                                                   const typename io<R>::real* __restrict__ kin_all,
                                                   const int* __restrict__ active,
                                                   double* __restrict__ dpart) {
  using C = C_t<R>;
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int Nz = pz.n, lds = Nz + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* A = tw + Nz;
  C* B = A + LZ * lds;
  const int k = sys_k[s];
  const int c0 = blockIdx.x * LZ;
  for (int i = threadIdx.x; i < Nz; i += blockDim.x) tw[i] = to_c<C>(twz[i]);
  const typename io<R>::cx* src = b4 + (size_t)s * Nz * ncp;
  for (int idx = threadIdx.x; idx < LZ * Nz; idx += blockDim.x) {
    const int iz = idx / LZ, l = idx - iz * LZ;
    const int col = c0 + l;
    A[l * lds + iz] = (col < nc) ? to_c<C>(src[(size_t)iz * ncp + col]) : mk<C>(R(0), R(0));
  }
  __syncthreads();
  C* res = fft_lines<C, false>(A, B, pz, LZ, lds, nullptr, 1, tw);
  typename io<R>::cx* dst = out + (size_t)s * ld;
  const typename io<R>::cx* ps = psi ? psi + (size_t)s * ld : nullptr;
  const R sh = shift ? to_r<R>(shift[s]) : R(0);
  const typename io<R>::real* kin = kin_all ? kin_all + (size_t)k * ldk : nullptr;
  double dot = 0.0;
  for (int idx = threadIdx.x; idx < LZ * Nz; idx += blockDim.x) {
    const int l = idx / Nz, z = idx - l * Nz;
    const int col = c0 + l;
    if (col >= nc) continue;
    const int* inf = colinfo + ((size_t)k * nc + col) * 3;
    int t = z - inf[2];
    if (t < 0) t += Nz;
    if (t >= inf[1]) continue;
    const int i = inf[0] + t;
    C v = res[l * lds + z];
    if (ps) {
      const R d = (kin ? to_r<R>(kin[i]) : R(0)) - sh;
      const C p = to_c<C>(ps[i]);
      v.x += d * p.x;
      v.y += d * p.y;
      dot += to_d(p.x) * to_d(v.x) + to_d(p.y) * to_d(v.y);
    }
    dst[i] = from_c(v);
  }
  if (dpart) {
    // Re <psi, out> over this CTA's plane waves (fixed-order block reduction)
    dot = block_sum(dot, red);
    if (threadIdx.x == 0) dpart[(size_t)s * gridDim.x + blockIdx.x] = dot;
  }
}

// ----------------------------------------------------------------- planes --

template <typename R>
__global__ void __launch_bounds__(256) k_plane(const C_t<R>* __restrict__ b1, int nc, int ncp,
                                               const int* __restrict__ col_xy,
                                               const int* __restrict__ xpos, int nxa, FftPlan px,
                                               FftPlan py, int Nz, const C_t<R>* __restrict__ twx,
                                               const C_t<R>* __restrict__ twy,
                                               const R* __restrict__ pot,
                                               const double* __restrict__ pot_scale,
                                               const int* __restrict__ active,
                                               C_t<R>* __restrict__ b4,
                                               const C_t<R>* __restrict__ real_in) {
  using C = C_t<R>;
  const int s = blockIdx.y, iz = blockIdx.x;
  if (active && !active[s]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nx = px.n, Ny = py.n, ldp = Nx + 1;
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + Nx;
  C* A = ty + Ny;
  C* B = A + Ny * ldp;
  int* xp = reinterpret_cast<int*>(B + Ny * ldp);
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  C* P;
  C* Q;
  if (real_in) {
    // the synthesis sum_G c_G e^{iG.r} of this plane is given
    const C* rp = real_in + ((size_t)s * Nz + iz) * Ny * Nx;
    for (int e = threadIdx.x; e < Ny * Nx; e += blockDim.x) {
      const int iy = e / Nx, ix = e - iy * Nx;
      A[iy * ldp + ix] = rp[e];
    }
    __syncthreads();
    P = A;
    Q = B;
  } else {
    for (int i = threadIdx.x; i < 2 * Ny * ldp; i += blockDim.x) A[i] = mk<C>(0, 0);
    __syncthreads();
    const C* src = b1 + ((size_t)s * Nz + iz) * ncp;
    for (int col = threadIdx.x; col < nc; col += blockDim.x)
      A[col_xy[2 * col + 1] * ldp + col_xy[2 * col]] = src[col];
    __syncthreads();
    P = fft_lines<C, true>(A, B, py, nxa, 0, xp, ldp, ty);          // y-lines, active x
    Q = (P == A) ? B : A;
    P = fft_lines<C, true>(P, Q, px, Ny, ldp, nullptr, 1, tx);     // x-lines, all rows
    Q = (P == A) ? B : A;
  }
  const R sc = pot_scale ? (R)(*pot_scale) : R(1);
  const R* pp = pot + (size_t)iz * Ny * Nx;
  for (int e = threadIdx.x; e < Ny * Nx; e += blockDim.x) {
    const int iy = e / Nx, ix = e - iy * Nx;
    P[iy * ldp + ix] = cscale(P[iy * ldp + ix], pp[e] * sc);
  }
  __syncthreads();
  P = fft_lines<C, false>(P, Q, px, Ny, ldp, nullptr, 1, tx);
  Q = (P == A) ? B : A;
  P = fft_lines<C, false>(P, Q, py, nxa, 0, xp, ldp, ty);
  C* dst = b4 + ((size_t)s * Nz + iz) * ncp;
  for (int col = threadIdx.x; col < nc; col += blockDim.x)
    dst[col] = P[col_xy[2 * col + 1] * ldp + col_xy[2 * col]];
}

// Density-type accumulation over a group of systems for one z-plane:
//   part[g][iz][iy][ix] = sum_{s in g} a_s Re(conj(psi_s) dpsi_s) + b_s |psi_s|^2
// with psi_s, dpsi_s the unnormalised syntheses sum_G c_G e^{iG.r} of the
// z-transformed inputs b1phi, b1d (b1d may be null: only the b_s term).
constexpr int kDensThreads = 512;
constexpr int kDensMaxPerThread = 20;

template <typename R>
__global__ void __launch_bounds__(kDensThreads) k_density(
    const C_t<R>* __restrict__ b1phi, const C_t<R>* __restrict__ b1d, int nc, int ncp,
    const int* __restrict__ col_xy, const int* __restrict__ xpos, int nxa, FftPlan px, FftPlan py,
    int Nz, const C_t<R>* __restrict__ twx, const C_t<R>* __restrict__ twy,
    const double* __restrict__ coef_a, const double* __restrict__ coef_b, int nsys, int ngroups,
    double* __restrict__ part, const C_t<R>* __restrict__ psi_real) {
  using C = C_t<R>;
  const int iz = blockIdx.x, g = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nx = px.n, Ny = py.n, ldp = Nx + 1, np = Ny * ldp;
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + Nx;
  C* buf[3] = {ty + Ny, ty + Ny + np, ty + Ny + 2 * np};
  int* xp = reinterpret_cast<int*>(buf[2] + np);
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  double acc[kDensMaxPerThread];
#pragma unroll
  for (int i = 0; i < kDensMaxPerThread; ++i) acc[i] = 0.0;
  const int s0 = (int)((long long)g * nsys / ngroups), s1 = (int)((long long)(g + 1) * nsys / ngroups);
  for (int s = s0; s < s1; ++s) {
    // psi plane in buf[0]/buf[1]
    C* psi;
    if (psi_real) {
      const C* rp = psi_real + ((size_t)s * Nz + iz) * Ny * Nx;
      for (int e = threadIdx.x; e < Ny * Nx; e += blockDim.x) {
        const int iy = e / Nx, ix = e - iy * Nx;
        buf[0][iy * ldp + ix] = rp[e];
      }
      __syncthreads();
      psi = buf[0];
    } else {
      for (int i = threadIdx.x; i < 2 * np; i += blockDim.x) buf[0][i] = mk<C>(0, 0);
      __syncthreads();
      const C* src = b1phi + ((size_t)s * Nz + iz) * ncp;
      for (int col = threadIdx.x; col < nc; col += blockDim.x)
        buf[0][col_xy[2 * col + 1] * ldp + col_xy[2 * col]] = src[col];
      __syncthreads();
      C* P = fft_lines<C, true>(buf[0], buf[1], py, nxa, 0, xp, ldp, ty);
      C* Q = (P == buf[0]) ? buf[1] : buf[0];
      psi = fft_lines<C, true>(P, Q, px, Ny, ldp, nullptr, 1, tx);
    }
    C* D = nullptr;
    if (b1d) {
      C* f0 = buf[2];
      C* f1 = (psi == buf[0]) ? buf[1] : buf[0];
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        f0[i] = mk<C>(0, 0);
        f1[i] = mk<C>(0, 0);
      }
      __syncthreads();
      const C* sd = b1d + ((size_t)s * Nz + iz) * ncp;
      for (int col = threadIdx.x; col < nc; col += blockDim.x)
        f0[col_xy[2 * col + 1] * ldp + col_xy[2 * col]] = sd[col];
      __syncthreads();
      C* P2 = fft_lines<C, true>(f0, f1, py, nxa, 0, xp, ldp, ty);
      C* Q2 = (P2 == f0) ? f1 : f0;
      D = fft_lines<C, true>(P2, Q2, px, Ny, ldp, nullptr, 1, tx);
    }
    const double a = coef_a ? coef_a[s] : 0.0, b = coef_b ? coef_b[s] : 0.0;
#pragma unroll
    for (int i = 0; i < kDensMaxPerThread; ++i) {
      const int e = threadIdx.x + i * kDensThreads;
      if (e < Ny * Nx) {
        const int iy = e / Nx, ix = e - iy * Nx;
        const C p = psi[iy * ldp + ix];
        double v = b * ((double)p.x * p.x + (double)p.y * p.y);
        if (D) {
          const C d = D[iy * ldp + ix];
          v += a * ((double)p.x * d.x + (double)p.y * d.y);
        }
        acc[i] += v;
      }
    }
    __syncthreads();
  }
  double* dst = part + ((size_t)g * Nz + iz) * Ny * Nx;
#pragma unroll
  for (int i = 0; i < kDensMaxPerThread; ++i) {
    const int e = threadIdx.x + i * kDensThreads;
    if (e < Ny * Nx) dst[e] = acc[i];
  }
}

// Unnormalised syntheses sum_G c_G e^{iG.r} of the z-transformed vectors b1,
// written plane by plane: out[s][iz][iy][ix].
template <typename R>
__global__ void __launch_bounds__(256) k_synth_planes(const C_t<R>* __restrict__ b1, int nc, int ncp,
                                                      const int* __restrict__ col_xy,
                                                      const int* __restrict__ xpos, int nxa, FftPlan px,
                                                      FftPlan py, int Nz, const C_t<R>* __restrict__ twx,
                                                      const C_t<R>* __restrict__ twy,
                                                      C_t<R>* __restrict__ out) {
  using C = C_t<R>;
  const int s = blockIdx.y, iz = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nx = px.n, Ny = py.n, ldp = Nx + 1;
  C* tx = reinterpret_cast<C*>(smem_raw);
  C* ty = tx + Nx;
  C* A = ty + Ny;
  C* B = A + Ny * ldp;
  int* xp = reinterpret_cast<int*>(B + Ny * ldp);
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) tx[i] = twx[i];
  for (int i = threadIdx.x; i < Ny; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < nxa; i += blockDim.x) xp[i] = xpos[i];
  for (int i = threadIdx.x; i < 2 * Ny * ldp; i += blockDim.x) A[i] = mk<C>(0, 0);
  __syncthreads();
  const C* src = b1 + ((size_t)s * Nz + iz) * ncp;
  for (int col = threadIdx.x; col < nc; col += blockDim.x)
    A[col_xy[2 * col + 1] * ldp + col_xy[2 * col]] = src[col];
  __syncthreads();
  C* P = fft_lines<C, true>(A, B, py, nxa, 0, xp, ldp, ty);
  C* Q = (P == A) ? B : A;
  P = fft_lines<C, true>(P, Q, px, Ny, ldp, nullptr, 1, tx);
  C* dst = out + ((size_t)s * Nz + iz) * Ny * Nx;
  for (int e = threadIdx.x; e < Ny * Nx; e += blockDim.x) {
    const int iy = e / Nx, ix = e - iy * Nx;
    dst[e] = P[iy * ldp + ix];
  }
}

// Phase of the most-real gauge of every orbital: with S_s = sum_r psi_s(r)^2,
// e^{-i theta_s} psi_s, theta_s = arg(S_s)/2, has the largest sum_r (Re)^2
// (sum_r (Re e^{-i theta} psi)^2 = (sum |psi|^2 + Re(e^{-2i theta} S))/2), so its
// real part loses nothing where the orbital has a real representation (Sec.
// "Dropping the imaginary part of the orbitals").  One block per orbital,
// fixed-order reduction; rot[s] = (cos theta_s, sin theta_s).
__global__ void __launch_bounds__(256) k_orbital_phase(const double2* __restrict__ psir, size_t ng,
                                                       double2* __restrict__ rot) {
  __shared__ double sh[8];
  const double2* p = psir + (size_t)blockIdx.x * ng;
  double a = 0.0, b = 0.0;
  for (size_t r = threadIdx.x; r < ng; r += blockDim.x) {
    const double2 v = p[r];
    a += v.x * v.x - v.y * v.y;
    b += 2.0 * v.x * v.y;
  }
  a = block_sum(a, sh);
  __syncthreads();
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    const double th = 0.5 * atan2(b, a);
    rot[blockIdx.x] = make_double2(cos(th), sin(th));
  }
}

// sum over n systems of |psi_s(r)|^2 and (Re e^{-i theta_s} psi_s(r))^2 at every
// grid point (planes of the cached real-space orbitals; the order of r does not matter)
__global__ void k_orbital_sq_sums(const double2* __restrict__ psir, const double2* __restrict__ rot, int nsys,
                                  size_t ng, double* __restrict__ abs2, double* __restrict__ re2) {
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < ng; r += (size_t)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int s = 0; s < nsys; ++s) {
      const double2 v = psir[(size_t)s * ng + r];
      const double2 q = rot[s];
      const double re = v.x * q.x + v.y * q.y;
      a += v.x * v.x + v.y * v.y;
      b += re * re;
    }
    abs2[r] = a;
    re2[r] = b;
  }
}

void orbital_sq_sums(ikr_ctx* c, const double2* psir, int nsys, double* abs2, double* re2, double2* rot) {
  ProfScope ps(c, kKidGridOps, 2);
  k_orbital_phase<<<nsys, 256, 0, c->stream>>>(psir, c->Ng, rot);
  IKR_CUDA(cudaGetLastError());
  k_orbital_sq_sums<<<152 * 8, 256, 0, c->stream>>>(psir, rot, nsys, c->Ng, abs2, re2);
  IKR_CUDA(cudaGetLastError());
}

// plane layout [iz][iy][ix] (summed over ngroups partial planes) -> C order
// [ix][iy][iz]; tiles of 32 (ix) x 32 (iz) per fixed iy.
__global__ void k_planes_to_c(const double* __restrict__ part, int ngroups, int Nx, int Ny, int Nz,
                              double scale, double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int iy = blockIdx.z;
  const int ix0 = blockIdx.x * 32, iz0 = blockIdx.y * 32;
  const size_t plane = (size_t)Ny * Nx, vol = plane * Nz;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int iz = iz0 + j, ix = ix0 + threadIdx.x;
    double v = 0.0;
    if (iz < Nz && ix < Nx) {
      const size_t o = (size_t)iz * plane + (size_t)iy * Nx + ix;
      for (int g = 0; g < ngroups; ++g) v += part[g * vol + o];
    }
    tile[j][threadIdx.x] = v;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int ix = ix0 + j, iz = iz0 + threadIdx.x;
    if (ix < Nx && iz < Nz) out[((size_t)ix * Ny + iy) * Nz + iz] = scale * tile[threadIdx.x][j];
  }
}

// C order [ix][iy][iz] -> plane layout [iz][iy][ix], times scale (and an
// optional device scalar factor).
template <typename R>
__global__ void k_c_to_planes(const double* __restrict__ in, int Nx, int Ny, int Nz, double scale,
                              const double* __restrict__ dscale, R* __restrict__ out) {
  __shared__ double tile[32][33];
  const int iy = blockIdx.z;
  const int iz0 = blockIdx.x * 32, ix0 = blockIdx.y * 32;
  const double sc = scale * (dscale ? *dscale : 1.0);
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int ix = ix0 + j, iz = iz0 + threadIdx.x;
    tile[j][threadIdx.x] = (ix < Nx && iz < Nz) ? in[((size_t)ix * Ny + iy) * Nz + iz] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int iz = iz0 + j, ix = ix0 + threadIdx.x;
    if (ix < Nx && iz < Nz) out[((size_t)iz * Ny + iy) * Nx + ix] = (R)(sc * tile[threadIdx.x][j]);
  }
}

// ------------------------------------------------------- full-grid lines --
// In-place FFT of every line along one axis of a C-order complex grid.  Line
// q = (o, t), o < n_outer, t < n_inner, starts at o*ostride + t*istride and
// its elements are estride apart.
template <bool INV>
__global__ void __launch_bounds__(256) k_fft_axis(double2* __restrict__ data, FftPlan p,
                                                  const double2* __restrict__ tw, int nlines,
                                                  int n_inner, int istride, int ostride, int estride,
                                                  int L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, lds = n + 1;
  double2* t = reinterpret_cast<double2*>(smem_raw);
  double2* A = t + n;
  double2* B = A + L * lds;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = tw[i];
  const int q0 = blockIdx.x * L;
  const bool efast = (estride == 1);
  for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
    int l, e;
    if (efast) { l = idx / n; e = idx - l * n; } else { e = idx / L; l = idx - e * L; }
    const int q = q0 + l;
    double2 v = make_double2(0, 0);
    if (q < nlines) {
      const int o = q / n_inner, tt = q - o * n_inner;
      v = data[(size_t)o * ostride + (size_t)tt * istride + (size_t)e * estride];
    }
    A[l * lds + e] = v;
  }
  __syncthreads();
  double2* res = fft_lines<double2, INV>(A, B, p, L, lds, nullptr, 1, t);
  for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
    int l, e;
    if (efast) { l = idx / n; e = idx - l * n; } else { e = idx / L; l = idx - e * L; }
    const int q = q0 + l;
    if (q < nlines) {
      const int o = q / n_inner, tt = q - o * n_inner;
      data[(size_t)o * ostride + (size_t)tt * istride + (size_t)e * estride] = res[l * lds + e];
    }
  }
}

// ---------------------------------------------------------------- launches --

template <typename R>
void launch_z_inverse(ikr_ctx* c, const SysList& L, const C_t<R>* sphere, int ld, const int* active,
                      C_t<R>* b1, const int* list, int nlist) {
  if (L.n == 0) return;
  ProfScope ps(c, kKidZInv, 1, active ? c->active_hint : L.n, (int)sizeof(R));
  if constexpr (sizeof(R) == 4) {
    if (list && nlist <= 0 && z_reg_ok(c)) return;   // no active system
    if (launch_z_inverse_reg(c, list ? nlist : L.n, L.d_k.p, sphere, ld, active, list, b1)) return;
  }
  const int Nz = c->N[2];
  const int LZ = lines_per_cta(Nz);
  const size_t smem = sizeof(C_t<R>) * (Nz + 2 * LZ * (Nz + 1));
  dim3 grid((c->nc + LZ - 1) / LZ, L.n);
  if (sizeof(R) == 8 && c->emulate_fp64) {
    // FP64-accurate pass of the mixed path on the FP32 pipe (double-float:
    // 3.7 -> 3.0 ms per cfg2 solve against the FP64 pipe)
    set_smem(k_z_inverse<dfloat>, smem);
    k_z_inverse<dfloat><<<grid, 256, smem, c->stream>>>(
        reinterpret_cast<const double2*>(sphere), ld, L.d_k.p, c->k_colinfo.p, c->nc, c->ncp, c->plan[2],
        c->d_tw[2].p, active, LZ, reinterpret_cast<double2*>(b1));
    IKR_CUDA(cudaGetLastError());
    return;
  }
  set_smem(k_z_inverse<R>, smem);
  k_z_inverse<R><<<grid, 256, smem, c->stream>>>(sphere, ld, L.d_k.p, c->k_colinfo.p, c->nc, c->ncp,
                                                  c->plan[2], tw_ptr<R>(c, 2), active, LZ, b1);
  IKR_CUDA(cudaGetLastError());
}

template <typename R>
void launch_plane(ikr_ctx* c, const SysList& L, const C_t<R>* b1, const R* pot, const double* pot_scale,
                  const int* active, C_t<R>* b4, const C_t<R>* real_in, const int* list, int nlist) {
  if (L.n == 0) return;
  ProfScope ps(c, kKidPlane, 1, active ? c->active_hint : L.n, (int)sizeof(R));
  if (sizeof(R) == 8 && c->emulate_fp64) {
    // FP64-accurate pass of the mixed path on the FP32 units (double-float)
    if (launch_plane_sw(c, L.n, reinterpret_cast<const double2*>(b1), reinterpret_cast<const double*>(pot),
                        pot_scale, active, reinterpret_cast<double2*>(b4),
                        reinterpret_cast<const double2*>(real_in)))
      return;
    if (launch_plane_fast<dfloat>(c, L.n, reinterpret_cast<const double2*>(b1),
                                  reinterpret_cast<const double*>(pot), pot_scale, active,
                                  reinterpret_cast<double2*>(b4), reinterpret_cast<const double2*>(real_in)))
      return;
  }
  if constexpr (sizeof(R) == 4) {
    if (launch_plane_reg(c, L.n, b1, pot, pot_scale, active, b4, real_in, list, nlist)) return;
  }
  if (launch_plane_fast<R>(c, L.n, b1, pot, pot_scale, active, b4, real_in)) return;
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  const size_t smem = sizeof(C_t<R>) * (Nx + Ny + 2 * (size_t)Ny * (Nx + 1)) + sizeof(int) * c->nxa;
  IKR_REQUIRE(smem <= kMaxPlaneSmem, IKR_ERR_ARG, plane_smem_message(c, smem));
  set_smem(k_plane<R>, smem);
  dim3 grid(Nz, L.n);
  k_plane<R><<<grid, 256, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                              c->plan[0], c->plan[1], Nz, tw_ptr<R>(c, 0),
                                              tw_ptr<R>(c, 1), pot, pot_scale, active, b4, real_in);
  IKR_CUDA(cudaGetLastError());
}

int zf_chunks(ikr_ctx* c, int fp_bytes) {
  if (fp_bytes == 4 && z_reg_ok(c)) return z_reg_chunks(c);
  const int LZ = lines_per_cta(c->N[2]);
  return (c->nc + LZ - 1) / LZ;
}
int zf_chunks(ikr_ctx* c) { return std::max(zf_chunks(c, 4), zf_chunks(c, 8)); }

template <typename R>
void launch_z_forward(ikr_ctx* c, const SysList& L, const C_t<R>* b4, C_t<R>* out, int ld,
                      const C_t<R>* psi, const double* shift, bool kinetic, const int* active,
                      double* dpart, const int* list, int nlist) {
  if (L.n == 0) return;
  ProfScope ps(c, kKidZFwd, 1, active ? c->active_hint : L.n, (int)sizeof(R));
  if constexpr (sizeof(R) == 4) {
    if (list && nlist <= 0 && z_reg_ok(c)) return;   // no active system
    if (launch_z_forward_reg(c, list ? nlist : L.n, L.d_k.p, b4, out, ld, psi, shift,
                             kinetic ? kin_all_ptr<R>(c) : nullptr, active, list, dpart))
      return;
  }
  const int Nz = c->N[2];
  const int LZ = lines_per_cta(Nz);
  const size_t smem = sizeof(C_t<R>) * (Nz + 2 * LZ * (Nz + 1));
  dim3 grid((c->nc + LZ - 1) / LZ, L.n);
  // (the FP64-accurate forward pass stays on the FP64 pipe: in double-float its
  // conversions and the normalised kinetic term cost more than they save)
  set_smem(k_z_forward<R>, smem);
  const R* kin = kinetic ? kin_all_ptr<R>(c) : nullptr;
  k_z_forward<R><<<grid, 256, smem, c->stream>>>(b4, c->nc, c->ncp, L.d_k.p, c->k_colinfo.p,
                                                  c->plan[2], tw_ptr<R>(c, 2), LZ, out, ld, c->ld,
                                                  psi, shift, kin, active, dpart);
  IKR_CUDA(cudaGetLastError());
}

// Number of system groups G of a density launch (grid Nz x G, each block
// walking nsys/G systems): the G that minimises (waves of blocks) x (systems
// per block) for per_sm resident blocks on each SM, the smaller on ties.
int density_groups(ikr_ctx* c, int nsys, int per_sm) {
  const int slots = std::max(1, c->nsm * std::max(per_sm, 1));
  const int Nz = c->N[2];
  const int gmax = std::max(1, std::min(nsys, 64));
  int best = 1;
  long long best_t = -1;
  for (int g = 1; g <= gmax; ++g) {
    const long long t = (long long)((Nz * g + slots - 1) / slots) * ((nsys + g - 1) / g);
    if (best_t < 0 || t < best_t) {
      best_t = t;
      best = g;
    }
  }
  return best;
}

template <typename R>
void launch_density(ikr_ctx* c, int nsys, const C_t<R>* b1phi, const C_t<R>* b1d,
                    const double* coef_a, const double* coef_b, double* out, double scale,
                    const C_t<R>* psi_real) {
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  IKR_REQUIRE(Nx * Ny <= kDensThreads * kDensMaxPerThread, IKR_ERR_ARG,
              "grid plane too large for the density kernel");
  ProfScope ps(c, kKidDensity, 2, nsys, (int)sizeof(R));
  const size_t np = (size_t)Ny * (Nx + 1);
  const size_t smem = sizeof(C_t<R>) * (Nx + Ny + 3 * np) + sizeof(int) * c->nxa;
  bool fast = false;
  int G = 1;
  if (nsys > 0 && psi_real && b1d) {
    if (sizeof(R) == 8 && c->emulate_fp64 && c->d_psir_df.p &&
        reinterpret_cast<const void*>(psi_real) == reinterpret_cast<const void*>(c->d_psir.p))
      // the double-float kernel reads the (hi, lo) copy of the cached orbitals
      fast = launch_density_fast<dfloat>(c, nsys, reinterpret_cast<const double2*>(b1d),
                                         reinterpret_cast<const double2*>(c->d_psir_df.p), coef_a, coef_b, &G);
    if (!fast) fast = launch_density_fast<R>(c, nsys, b1d, psi_real, coef_a, coef_b, &G);
  }
  if (fast) {
  } else if (nsys > 0) {
    set_smem(k_density<R>, smem);
    int per_sm = 1;
    IKR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_density<R>, kDensThreads, smem));
    G = density_groups(c, nsys, per_sm);
    c->ws.dens_part.reserve((size_t)G * c->Ng);
    dim3 grid(Nz, G);
    k_density<R><<<grid, kDensThreads, smem, c->stream>>>(
        b1phi, b1d, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa, c->plan[0], c->plan[1], Nz,
        tw_ptr<R>(c, 0), tw_ptr<R>(c, 1), coef_a, coef_b, nsys, G, c->ws.dens_part.p, psi_real);
    IKR_CUDA(cudaGetLastError());
  } else {
    c->ws.dens_part.reserve(c->Ng);
    IKR_CUDA(cudaMemsetAsync(c->ws.dens_part.p, 0, sizeof(double) * G * c->Ng, c->stream));
  }
  dim3 tgrid((Nx + 31) / 32, (Nz + 31) / 32, Ny);
  k_planes_to_c<<<tgrid, dim3(32, 8), 0, c->stream>>>(c->ws.dens_part.p, G, Nx, Ny, Nz, scale, out);
  IKR_CUDA(cudaGetLastError());
}

template <typename R>
void launch_synth_planes(ikr_ctx* c, int nsys, const C_t<R>* b1, C_t<R>* out) {
  if (nsys == 0) return;
  ProfScope ps(c, kKidPlane, 1, nsys, (int)sizeof(R));
  if (launch_synth_fast<R>(c, nsys, b1, out)) return;
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  const size_t smem = sizeof(C_t<R>) * (Nx + Ny + 2 * (size_t)Ny * (Nx + 1)) + sizeof(int) * c->nxa;
  set_smem(k_synth_planes<R>, smem);
  dim3 grid(Nz, nsys);
  k_synth_planes<R><<<grid, 256, smem, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                                     c->plan[0], c->plan[1], Nz, tw_ptr<R>(c, 0),
                                                     tw_ptr<R>(c, 1), out);
  IKR_CUDA(cudaGetLastError());
}

template <typename R>
void to_plane_layout(ikr_ctx* c, const double* in, R* out, double scale, const double* dscale) {
  ProfScope ps(c, kKidGridOps, 1);
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  dim3 tgrid((Nz + 31) / 32, (Nx + 31) / 32, Ny);
  k_c_to_planes<R><<<tgrid, dim3(32, 8), 0, c->stream>>>(in, Nx, Ny, Nz, scale, dscale, out);
  IKR_CUDA(cudaGetLastError());
}

void full_fft(ikr_ctx* c, double2* data, bool inverse) {
  ProfScope ps(c, kKidGridFFT, 3);
  const int N1 = c->N[0], N2 = c->N[1], N3 = c->N[2];
  // axis 3 (contiguous), axis 2, axis 1
  struct Ax { int axis, nlines, n_inner, istride, ostride, estride; } ax[3] = {
      {2, N1 * N2, 1, 0, N3, 1},
      {1, N1 * N3, N3, 1, N2 * N3, N3},
      {0, N2 * N3, N2 * N3, 1, 0, N2 * N3},
  };
  for (auto& a : ax) {
    const int n = c->plan[a.axis].n;
    const int L = lines_per_cta(n);
    const size_t smem = sizeof(double2) * (n + 2 * L * (n + 1));
    const int blocks = (a.nlines + L - 1) / L;
    if (inverse) {
      set_smem(k_fft_axis<true>, smem);
      k_fft_axis<true><<<blocks, 256, smem, c->stream>>>(data, c->plan[a.axis], c->d_tw[a.axis].p,
                                                          a.nlines, a.n_inner, a.istride, a.ostride,
                                                          a.estride, L);
    } else {
      set_smem(k_fft_axis<false>, smem);
      k_fft_axis<false><<<blocks, 256, smem, c->stream>>>(data, c->plan[a.axis], c->d_tw[a.axis].p,
                                                           a.nlines, a.n_inner, a.istride, a.ostride,
                                                           a.estride, L);
    }
    IKR_CUDA(cudaGetLastError());
  }
}

#define IKR_INST(R)                                                                                 \
  template void launch_z_inverse<R>(ikr_ctx*, const SysList&, const C_t<R>*, int, const int*,     \
                                    C_t<R>*, const int*, int);                                      \
  template void launch_plane<R>(ikr_ctx*, const SysList&, const C_t<R>*, const R*, const double*,  \
                                const int*, C_t<R>*, const C_t<R>*, const int*, int);               \
  template void launch_synth_planes<R>(ikr_ctx*, int, const C_t<R>*, C_t<R>*);                      \
  template void launch_z_forward<R>(ikr_ctx*, const SysList&, const C_t<R>*, C_t<R>*, int,         \
                                    const C_t<R>*, const double*, bool, const int*, double*,        \
                                    const int*, int);                                               \
  template void launch_density<R>(ikr_ctx*, int, const C_t<R>*, const C_t<R>*,                     \
                                  const double*, const double*, double*, double, const C_t<R>*);    \
  template void to_plane_layout<R>(ikr_ctx*, const double*, R*, double, const double*);
IKR_INST(double)
IKR_INST(float)
#undef IKR_INST

// ------------------------------------------- raw-pointer launches (no SysList) --
// Launch the three H_k kernels for n systems whose k-point indices are in the
// device array d_sysk; used by the no-allocation entry point, which keeps its
// scratch (including d_sysk) in a static device array.
void launch_hamiltonian_raw(ikr_ctx* c, int n, const int* d_sysk, const double2* psi, int ld, double2* b1,
                            double2* b4, double2* hpsi) {
  if (n == 0) return;
  const int Nx = c->N[0], Ny = c->N[1], Nz = c->N[2];
  const int LZ = lines_per_cta(Nz);
  const size_t smz = sizeof(double2) * (Nz + 2 * LZ * (Nz + 1));
  const size_t smp = sizeof(double2) * (Nx + Ny + 2 * (size_t)Ny * (Nx + 1)) + sizeof(int) * c->nxa;
  set_smem(k_z_inverse<double>, smz);
  set_smem(k_z_forward<double>, smz);
  dim3 gz((c->nc + LZ - 1) / LZ, n);
  k_z_inverse<double><<<gz, 256, smz, c->stream>>>(psi, ld, d_sysk, c->k_colinfo.p, c->nc, c->ncp, c->plan[2],
                                                   c->d_tw[2].p, nullptr, LZ, b1);
  IKR_CUDA(cudaGetLastError());
  // the compiled plane shape where there is one (what ikr_apply_hamiltonian runs), else the
  // runtime-size kernel, whose whole plane must fit in shared memory
  if (!launch_plane_fast<double>(c, n, b1, c->d_Vt.p, nullptr, nullptr, b4, nullptr)) {
    IKR_REQUIRE(smp <= kMaxPlaneSmem, IKR_ERR_ARG, plane_smem_message(c, smp));
    set_smem(k_plane<double>, smp);
    dim3 gp(Nz, n);
    k_plane<double><<<gp, 256, smp, c->stream>>>(b1, c->nc, c->ncp, c->d_col_xy.p, c->d_xpos.p, c->nxa,
                                                 c->plan[0], c->plan[1], Nz, c->d_tw[0].p, c->d_tw[1].p,
                                                 c->d_Vt.p, nullptr, nullptr, b4, nullptr);
    IKR_CUDA(cudaGetLastError());
  }
  k_z_forward<double><<<gz, 256, smz, c->stream>>>(b4, c->nc, c->ncp, d_sysk, c->k_colinfo.p, c->plan[2],
                                                   c->d_tw[2].p, LZ, hpsi, ld, c->ld, psi, nullptr,
                                                   c->d_kin_all.p, nullptr, nullptr);
  IKR_CUDA(cudaGetLastError());
}

}  // namespace ikr
