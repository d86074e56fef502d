// Context setup: plane-wave spheres (Sec. 2.3.1, k-form of Sec. 4.1.1), the
// pruned FFT geometry, the potential, and the ground state (occupations,
// Fermi level, density rho and exchange kernel K^xc[rho]).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cmath>
#include <map>

#include "ops.hpp"

namespace ikr {

namespace {

void inv3(const double* a, double* inv) {
  // a is row-major 3x3
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  IKR_REQUIRE(std::fabs(det) > 1e-12, IKR_ERR_ARG, "singular lattice");
  inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  auto push = [&](int r) {
    IKR_REQUIRE(p.nstages < kMaxStages, IKR_ERR_ARG, "FFT size has too many factors");
    p.radix[p.nstages++] = r;
    m /= r;
  };
  while (m % 4 == 0) push(4);
  while (m % 2 == 0) push(2);
  while (m % 3 == 0) push(3);
  while (m % 5 == 0) push(5);
  IKR_REQUIRE(m == 1, IKR_ERR_ARG, "FFT grid sizes may only contain the prime factors 2, 3 and 5");
  return p;
}

template <typename T> void upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
  d.reserve(h.size() ? h.size() : 1);
  if (!h.empty()) IKR_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
}

inline int signed_index(int p, int n) { return p < (n + 1) / 2 ? p : p - n; }

// Fermi-Dirac f(x) = 2/(1+e^x) and its derivative, evaluated without overflow.
double fd(double x) { return x > 0 ? 2.0 * std::exp(-x) / (1.0 + std::exp(-x)) : 2.0 / (1.0 + std::exp(x)); }
double fd_prime(double x) {
  const double e = std::exp(-std::fabs(x));
  return -2.0 * e / ((1.0 + e) * (1.0 + e));
}

}  // namespace

void setup_system(ikr_ctx* c, const ikr_system* sys) {
  IKR_REQUIRE(sys, IKR_ERR_ARG, "system is NULL");
  {
    int dev = 0;
    IKR_CUDA(cudaGetDevice(&dev));
    IKR_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  IKR_REQUIRE(sys->nkpt >= 1 && sys->kpoints && sys->kweights && sys->V, IKR_ERR_ARG,
              "k-points, weights and V are required");
  IKR_REQUIRE(sys->Ecut > 0, IKR_ERR_ARG, "Ecut must be positive");
  IKR_REQUIRE(sys->temperature >= 0, IKR_ERR_ARG, "temperature must be >= 0");
  IKR_REQUIRE(sys->n_electrons > 0 && sys->n_electrons % 2 == 0, IKR_ERR_ARG,
              "n_electrons must be positive and even");
  for (int a = 0; a < 3; ++a) {
    IKR_REQUIRE(sys->dims[a] >= 2 && sys->dims[a] <= 4096, IKR_ERR_ARG, "grid size out of range");
    c->N[a] = sys->dims[a];
    c->plan[a] = make_plan(sys->dims[a]);
  }
  c->Ng = (size_t)c->N[0] * c->N[1] * c->N[2];
  c->Ecut = sys->Ecut;
  c->T = sys->temperature;
  c->nel = sys->n_electrons;
  for (int i = 0; i < 9; ++i) c->lattice[i] = sys->lattice[i];
  // B = 2 pi A^{-T}; lattice[3*i+j] = A_ij (columns are cell vectors)
  double inv[9];
  inv3(c->lattice, inv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c->recip[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
  const double* A = c->lattice;
  c->volume = std::fabs(A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                        A[2] * (A[3] * A[7] - A[4] * A[6]));
  const cudaStream_t st = c->stream;

  // twiddles e^{-2 pi i t / n}
  for (int a = 0; a < 3; ++a) {
    const int n = c->N[a];
    std::vector<double2> tw(n);
    std::vector<float2> tw32(n);
    for (int t = 0; t < n; ++t) {
      const long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)n;
      tw[t] = make_double2((double)cosl(ang), (double)-sinl(ang));
      tw32[t] = make_float2((float)tw[t].x, (float)tw[t].y);
    }
    upload(c->d_tw[a], tw, st);
    upload(c->d_tw32[a], tw32, st);
  }

  // spheres G_k = {G : |k+G|^2 <= 2 Ecut}, lexicographic in (j1, j2, j3)
  const double* B = c->recip;
  const double radius = std::sqrt(2.0 * sys->Ecut);
  int jmax[3];
  for (int i = 0; i < 3; ++i) {
    // |j_i| <= |row_i(B^-1)| (|k+G| + ...) ; B^-1 = A^T / (2 pi)
    const double rn = std::sqrt(A[0 + i] * A[0 + i] + A[3 + i] * A[3 + i] + A[6 + i] * A[6 + i]) / (2.0 * M_PI);
    jmax[i] = (int)std::ceil(radius * rn + 1.0);
  }
  c->k.assign(sys->nkpt, KPoint());
  std::map<std::pair<int, int>, int> cols;
  int nbmax = 0;
  for (int ik = 0; ik < sys->nkpt; ++ik) {
    KPoint& K = c->k[ik];
    for (int i = 0; i < 3; ++i) K.kfrac[i] = sys->kpoints[3 * ik + i];
    K.weight = sys->kweights[ik];
    double kc[3];
    for (int i = 0; i < 3; ++i) kc[i] = B[3 * i] * K.kfrac[0] + B[3 * i + 1] * K.kfrac[1] + B[3 * i + 2] * K.kfrac[2];
    for (int j1 = -jmax[0]; j1 <= jmax[0]; ++j1)
      for (int j2 = -jmax[1]; j2 <= jmax[1]; ++j2)
        for (int j3 = -jmax[2]; j3 <= jmax[2]; ++j3) {
          double q[3];
          for (int i = 0; i < 3; ++i) q[i] = kc[i] + B[3 * i] * j1 + B[3 * i + 1] * j2 + B[3 * i + 2] * j3;
          const double e = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
          if (e <= sys->Ecut) {
            const int jj[3] = {j1, j2, j3};
            for (int a = 0; a < 3; ++a)
              IKR_REQUIRE(jj[a] >= -(c->N[a] / 2) && jj[a] < (c->N[a] + 1) / 2, IKR_ERR_ARG,
                          "plane-wave sphere does not fit inside the FFT grid");
            K.miller.push_back(j1);
            K.miller.push_back(j2);
            K.miller.push_back(j3);
            K.kin.push_back(e);
            cols[{j1, j2}] = 0;
          }
        }
    K.nb = (int)K.kin.size();
    IKR_REQUIRE(K.nb > 0, IKR_ERR_ARG, "empty plane-wave basis");
    nbmax = std::max(nbmax, K.nb);
  }
  c->ld = (nbmax + 63) / 64 * 64;
  // union columns
  c->nc = (int)cols.size();
  c->ncp = (c->nc + 15) / 16 * 16;
  c->col_ix.clear();
  c->col_iy.clear();
  std::vector<int> colxy;
  int ci = 0;
  std::vector<int> xs;
  for (auto& kv : cols) {
    kv.second = ci++;
    const int ix = ((kv.first.first % c->N[0]) + c->N[0]) % c->N[0];
    const int iy = ((kv.first.second % c->N[1]) + c->N[1]) % c->N[1];
    c->col_ix.push_back(ix);
    c->col_iy.push_back(iy);
    colxy.push_back(ix);
    colxy.push_back(iy);
    xs.push_back(ix);
  }
  std::sort(xs.begin(), xs.end());
  xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
  c->xpos = xs;
  c->nxa = (int)xs.size();
  upload(c->d_col_xy, colxy, st);
  upload(c->d_xpos, c->xpos, st);
  {
    const int N0 = c->N[0], N1 = c->N[1];
    std::map<int, std::vector<int>> ys;   // active x -> y of its columns
    for (size_t i = 0; i < c->col_ix.size(); ++i) ys[c->col_ix[i]].push_back(c->col_iy[i]);
    std::vector<std::array<int, 3>> rows;
    bool ok = N0 <= 64;
    unsigned long long mask = 0;
    for (auto& kv : ys) {
      std::vector<char> has(N1, 0);
      for (int y : kv.second) has[y] = 1;
      const int n = (int)kv.second.size();
      int ylo = 0, runs = 0;
      if (n == N1) {
        runs = 1;
      } else {
        for (int y = 0; y < N1; ++y)
          if (has[y] && !has[(y + N1 - 1) % N1]) {
            ylo = y;
            ++runs;
          }
      }
      ok = ok && runs == 1;
      rows.push_back({(kv.first + N0 / 2) % N0, ylo, n - 1});
      if (kv.first < 64) mask |= 1ull << kv.first;
    }
    std::sort(rows.begin(), rows.end());
    std::vector<int> xr;
    for (const auto& r : rows) xr.insert(xr.end(), r.begin(), r.end());
    c->xmask = mask;
    c->reg_plane_ok = ok;
    // the shifted active x positions form one run px_lo, px_lo + 1, ... (a sphere's
    // projection is an interval): the compact plane layout of k_plane_rc needs that
    bool contig = !rows.empty();
    for (size_t l = 0; l < rows.size(); ++l) contig = contig && rows[l][0] == rows[0][0] + (int)l;
    c->xr_contig = contig;
    c->pxlo = rows.empty() ? 0 : rows[0][0];
    // IKR_PLANE_RC=0 selects the full-plane FP32 kernel instead of the compact one,
    // IKR_PLANE_RC=4 the compact one compiled for 4 blocks per SM (read when the
    // context is created)
    // IKR_PLANE_SW=0 selects k_plane_t for the double-float pass of 48 x 48 planes
    if (const char* e = std::getenv("IKR_PLANE_SW")) c->plane_sw = std::atoi(e) != 0;
    if (const char* e = std::getenv("IKR_PLANE_RC")) {
      const int v = std::atoi(e);
      c->plane_rc = (v == 0 || v == 4) ? v : 5;
    }
    upload(c->d_xr, xr, st);
  }
  // per-k column info and kinetic energies
  const int nk = sys->nkpt;
  std::vector<int> colinfo((size_t)nk * c->nc * 3, 0);
  std::vector<double> kin((size_t)nk * c->ld, 0.0);
  std::vector<float> kin32((size_t)nk * c->ld, 0.0f);
  std::vector<int> nbs(nk);
  for (int ik = 0; ik < nk; ++ik) {
    KPoint& K = c->k[ik];
    nbs[ik] = K.nb;
    for (int i = 0; i < K.nb; ++i) {
      kin[(size_t)ik * c->ld + i] = K.kin[i];
      kin32[(size_t)ik * c->ld + i] = (float)K.kin[i];
    }
    int i = 0;
    while (i < K.nb) {
      const int j1 = K.miller[3 * i], j2 = K.miller[3 * i + 1];
      int e = i;
      while (e < K.nb && K.miller[3 * e] == j1 && K.miller[3 * e + 1] == j2) {
        IKR_REQUIRE(K.miller[3 * e + 2] == K.miller[3 * i + 2] + (e - i), IKR_ERR_ARG,
                    "sphere column is not contiguous");
        ++e;
      }
      const int col = cols[{j1, j2}];
      int* inf = &colinfo[((size_t)ik * c->nc + col) * 3];
      inf[0] = i;
      inf[1] = e - i;
      inf[2] = ((K.miller[3 * i + 2] % c->N[2]) + c->N[2]) % c->N[2];
      i = e;
    }
    K.colinfo.assign(colinfo.begin() + (size_t)ik * c->nc * 3, colinfo.begin() + (size_t)(ik + 1) * c->nc * 3);
  }
  upload(c->k_colinfo, colinfo, st);
  {
    // column prefix sums for the one-thread-per-column z-pass; it relies on the
    // runs of consecutive columns being consecutive in the sphere order
    std::vector<int> pre((size_t)nk * (c->nc + 1), 0);
    bool ok = true;
    int span = 0;
    for (int ik = 0; ik < nk; ++ik) {
      int* pk = &pre[(size_t)ik * (c->nc + 1)];
      for (int col = 0; col < c->nc; ++col) {
        const int* inf = &colinfo[((size_t)ik * c->nc + col) * 3];
        if (inf[1] > 0 && inf[0] != pk[col]) ok = false;
        pk[col + 1] = pk[col] + inf[1];
      }
      for (int c0 = 0; c0 < c->nc; c0 += kZC) span = std::max(span, pk[std::min(c0 + kZC, c->nc)] - pk[c0]);
    }
    c->zreg_ok = ok;
    c->zspan = std::max(span, 1);
    upload(c->d_colpre, pre, st);
  }
  upload(c->d_kin_all, kin, st);
  upload(c->d_kin_all32, kin32, st);
  upload(c->d_nb, nbs, st);

  // potential: C order, and plane layout [i3][i2][i1] divided by Ng
  const int N1 = c->N[0], N2 = c->N[1], N3 = c->N[2];
  std::vector<double> V(sys->V, sys->V + c->Ng);
  c->vmax = *std::max_element(V.begin(), V.end());
  std::vector<double> Vt(c->Ng);
  std::vector<float> Vt32(c->Ng);
  for (int i1 = 0; i1 < N1; ++i1)
    for (int i2 = 0; i2 < N2; ++i2)
      for (int i3 = 0; i3 < N3; ++i3) {
        const double v = V[((size_t)i1 * N2 + i2) * N3 + i3] / (double)c->Ng;
        Vt[((size_t)i3 * N2 + i2) * N1 + i1] = v;
        Vt32[((size_t)i3 * N2 + i2) * N1 + i1] = (float)v;
      }
  upload(c->d_V, V, st);
  upload(c->d_Vt, Vt, st);
  upload(c->d_Vt32, Vt32, st);
  // |G|^2 and the Coulomb kernel 4 pi / |G|^2 (G = 0 -> 0), divided by Ng
  std::vector<double> G2(c->Ng), coul(c->Ng);
  for (int p1 = 0; p1 < N1; ++p1)
    for (int p2 = 0; p2 < N2; ++p2)
      for (int p3 = 0; p3 < N3; ++p3) {
        const int j1 = signed_index(p1, N1), j2 = signed_index(p2, N2), j3 = signed_index(p3, N3);
        double g[3];
        for (int i = 0; i < 3; ++i) g[i] = B[3 * i] * j1 + B[3 * i + 1] * j2 + B[3 * i + 2] * j3;
        const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const size_t o = ((size_t)p1 * N2 + p2) * N3 + p3;
        G2[o] = g2;
        coul[o] = (g2 > 0.0) ? 4.0 * M_PI / g2 / (double)c->Ng : 0.0;
      }
  upload(c->d_G2, G2, st);
  upload(c->d_coul, coul, st);
  IKR_CUDA(cudaStreamSynchronize(st));
}

void make_syslist(ikr_ctx* c, SysList& L, int nsys, const int* kof, const int* band) {
  const int nk = (int)c->k.size();
  L.n = nsys;
  L.k.assign(kof, kof + nsys);
  L.band.assign(band, band + nsys);
  L.kstart.assign(nk, 0);
  L.kcount.assign(nk, 0);
  for (int s = 0; s < nsys; ++s) {
    IKR_REQUIRE(kof[s] >= 0 && kof[s] < nk, IKR_ERR_ARG, "k-point index out of range");
    IKR_REQUIRE(s == 0 || kof[s] >= kof[s - 1], IKR_ERR_ARG, "systems must be grouped by nondecreasing k");
    IKR_REQUIRE(band[s] >= 0, IKR_ERR_ARG, "band index out of range");
  }
  for (int s = nsys - 1; s >= 0; --s) {
    L.kstart[kof[s]] = s;
    L.kcount[kof[s]]++;
  }
  upload(L.d_k, L.k, c->stream);
  upload(L.d_band, L.band, c->stream);
  upload(L.d_kstart, L.kstart, c->stream);
  upload(L.d_kcount, L.kcount, c->stream);
}

// (hi, lo) float pairs of complex128 values: hi = fl32(x), lo = fl32(x - hi)
__global__ void k_to_dfloat(const double2* __restrict__ in, size_t n, float4* __restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[e];
    const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
    out[e] = make_float4(xh, __double2float_rn(v.x - (double)xh), yh, __double2float_rn(v.y - (double)yh));
  }
}

// rho[C order] = scale * sum_s wf[s] |psir_s|^2 from the cached real-space
// planes [s][i3][i2][i1] (systems added in order)
__global__ void k_rho_from_planes(const double2* __restrict__ psir, int S, int N1, int N2, int N3,
                                  const double* __restrict__ wf, double scale, double* __restrict__ rho) {
  const size_t ng = (size_t)N1 * N2 * N3;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ng; e += (size_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int s = 0; s < S; ++s) {
      const double2 v = psir[(size_t)s * ng + e];
      a += wf[s] * (v.x * v.x + v.y * v.y);
    }
    const size_t i1 = e % N1, i2 = (e / N1) % N2, i3 = e / ((size_t)N1 * N2);
    rho[(i1 * N2 + i2) * N3 + i3] = scale * a;
  }
}

void set_eigenpairs(ikr_ctx* c, const ikr_eigenpairs* eig) {
  IKR_REQUIRE(eig && eig->eigenvalues && eig->eigenvectors, IKR_ERR_ARG, "eigenpairs are NULL");
  const int nk = (int)c->k.size();
  const int nb = eig->nbands;
  IKR_REQUIRE(nb >= 1, IKR_ERR_ARG, "nbands must be positive");
  const cudaStream_t st = c->stream;
  for (int ik = 0; ik < nk; ++ik) {
    KPoint& K = c->k[ik];
    IKR_REQUIRE(nb <= K.nb, IKR_ERR_ARG, "nbands exceeds the basis size");
    K.nbands = nb;
    K.eps.assign(eig->eigenvalues + (size_t)ik * nb, eig->eigenvalues + (size_t)(ik + 1) * nb);
    for (int n = 1; n < nb; ++n)
      IKR_REQUIRE(K.eps[n] >= K.eps[n - 1], IKR_ERR_ARG, "eigenvalues must be ascending");
    IKR_REQUIRE(eig->eigenvectors[ik], IKR_ERR_ARG, "eigenvector pointer is NULL");
  }
  // occupations (eq. density); Fermi level by bisection for T > 0
  if (c->T == 0.0) {
    const int no = c->nel / 2;
    for (int ik = 0; ik < nk; ++ik) {
      KPoint& K = c->k[ik];
      IKR_REQUIRE(nb >= no + 1, IKR_ERR_ARG, "insulator needs nbands >= N/2 + 1");
      if (!(K.eps[no] - K.eps[no - 1] > 0.0)) throw Error(IKR_ERR_NOGAP, "no gap above band N/2");
      K.nocc = no;
      K.f.assign(nb, 0.0);
      K.fp.assign(nb, 0.0);
      for (int n = 0; n < no; ++n) K.f[n] = 2.0;
    }
    double homo = -1e300, lumo = 1e300;
    for (auto& K : c->k) {
      homo = std::max(homo, K.eps[no - 1]);
      lumo = std::min(lumo, K.eps[no]);
    }
    c->eF = 0.5 * (homo + lumo);
  } else {
    double lo = 1e300, hi = -1e300;
    for (auto& K : c->k) {
      lo = std::min(lo, K.eps.front());
      hi = std::max(hi, K.eps.back());
    }
    lo -= 50 * c->T + 1.0;
    hi += 50 * c->T + 1.0;
    auto count = [&](double eF) {
      double s = 0;
      for (auto& K : c->k)
        for (int n = 0; n < nb; ++n) s += K.weight * fd((K.eps[n] - eF) / c->T);
      return s;
    };
    IKR_REQUIRE(count(hi) >= c->nel, IKR_ERR_ARG, "nbands too small to hold N electrons");
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count(mid) < c->nel) lo = mid; else hi = mid;
    }
    c->eF = 0.5 * (lo + hi);
    for (auto& K : c->k) {
      K.f.resize(nb);
      K.fp.resize(nb);
      K.nocc = 0;
      for (int n = 0; n < nb; ++n) {
        const double x = (K.eps[n] - c->eF) / c->T;
        K.f[n] = fd(x);
        K.fp[n] = fd_prime(x) / c->T;
        if (K.f[n] > 1e-10) K.nocc = n + 1;
      }
      IKR_REQUIRE(K.nocc >= 1, IKR_ERR_ARG, "no occupied band at a k-point");
      IKR_REQUIRE(K.nocc < nb, IKR_ERR_ARG, "nbands must exceed N_occ,k (f > 1e-10)");
      if (!(K.eps[K.nocc] - K.eps[K.nocc - 1] > 0.0)) throw Error(IKR_ERR_NOGAP, "no gap above N_occ,k");
    }
  }
  // occupied system list and per-system data
  std::vector<int> kof, band, off(nk), noccs(nk);
  std::vector<double> eps_o, f_o, fp_o, w_o;
  c->noccmax = 0;
  for (int ik = 0; ik < nk; ++ik) {
    KPoint& K = c->k[ik];
    off[ik] = (int)kof.size();
    noccs[ik] = K.nocc;
    c->noccmax = std::max(c->noccmax, K.nocc);
    for (int n = 0; n < K.nocc; ++n) {
      kof.push_back(ik);
      band.push_back(n);
      eps_o.push_back(K.eps[n]);
      f_o.push_back(K.f[n]);
      fp_o.push_back(K.fp[n]);
      w_o.push_back(K.weight);
    }
  }
  const int S = (int)kof.size();
  make_syslist(c, c->occ, S, kof.data(), band.data());
  upload(c->d_phi_off, off, st);
  upload(c->d_occ_kstart, off, st);
  upload(c->d_nocc, noccs, st);
  upload(c->d_eps_occ, eps_o, st);
  upload(c->d_f_occ, f_o, st);
  upload(c->d_fp_occ, fp_o, st);
  upload(c->d_w_occ, w_o, st);
  // occupied orbitals, zero padded to ld
  const int ld = c->ld;
  c->d_phi_all.reserve((size_t)S * ld);
  c->d_phi_all32.reserve((size_t)S * ld);
  IKR_CUDA(cudaMemsetAsync(c->d_phi_all.p, 0, sizeof(double2) * S * ld, st));
  for (int ik = 0; ik < nk; ++ik) {
    const KPoint& K = c->k[ik];
    IKR_CUDA(cudaMemcpy2DAsync(c->d_phi_all.p + (size_t)off[ik] * ld, sizeof(double2) * ld,
                               eig->eigenvectors[ik], sizeof(double2) * K.nb, sizeof(double2) * K.nb,
                               K.nocc, cudaMemcpyDeviceToDevice, st));
  }
  to_fp32(c, c->d_phi_all.p, (size_t)S * ld, c->d_phi_all32.p);
  // all computed bands per k-point (occupied, then extra) for the Schur-complement solves
  {
    std::vector<int> roff(nk), rcnt(nk), xoff(nk), xcnt(nk);
    std::vector<double> reps;
    int tot = 0;
    c->rmax = c->xmax = 0;
    for (int ik = 0; ik < nk; ++ik) {
      const KPoint& K = c->k[ik];
      roff[ik] = tot;
      rcnt[ik] = nb;
      xoff[ik] = tot + K.nocc;
      xcnt[ik] = nb - K.nocc;
      c->rmax = std::max(c->rmax, nb);
      c->xmax = std::max(c->xmax, nb - K.nocc);
      for (int n = 0; n < nb; ++n) reps.push_back(K.eps[n]);
      tot += nb;
    }
    c->d_rset.reserve((size_t)tot * ld);
    c->d_rset32.reserve((size_t)tot * ld);
    IKR_CUDA(cudaMemsetAsync(c->d_rset.p, 0, sizeof(double2) * tot * ld, st));
    for (int ik = 0; ik < nk; ++ik) {
      const KPoint& K = c->k[ik];
      IKR_CUDA(cudaMemcpy2DAsync(c->d_rset.p + (size_t)roff[ik] * ld, sizeof(double2) * ld,
                                 eig->eigenvectors[ik], sizeof(double2) * K.nb, sizeof(double2) * K.nb, nb,
                                 cudaMemcpyDeviceToDevice, st));
    }
    to_fp32(c, c->d_rset.p, (size_t)tot * ld, c->d_rset32.p);
    upload(c->d_roff, roff, st);
    upload(c->d_rcnt, rcnt, st);
    upload(c->d_xoff, xoff, st);
    upload(c->d_xcnt, xcnt, st);
    upload(c->d_reps, reps, st);
    c->schur = false;
    c->batch_items = -1;
  }
  // preconditioner constants kappa_n = max(1, <phi_n, |k+G|^2/2 phi_n>)
  std::vector<double2> hphi((size_t)S * ld);
  IKR_CUDA(cudaMemcpyAsync(hphi.data(), c->d_phi_all.p, sizeof(double2) * S * ld, cudaMemcpyDeviceToHost, st));
  IKR_CUDA(cudaStreamSynchronize(st));
  c->h_kappa_occ.assign(S, 1.0);
  for (int s = 0; s < S; ++s) {
    const KPoint& K = c->k[kof[s]];
    double e = 0.0;
    for (int i = 0; i < K.nb; ++i) {
      const double2 v = hphi[(size_t)s * ld + i];
      e += K.kin[i] * (v.x * v.x + v.y * v.y);
    }
    c->h_kappa_occ[s] = std::max(1.0, e);
  }
  upload(c->d_kappa_occ, c->h_kappa_occ, st);
  // z-transformed occupied orbitals (reused by every chi0 application)
  const size_t b1n = (size_t)S * c->N[2] * c->ncp;
  c->d_b1phi.reserve(b1n);
  c->d_b1phi32.reserve(b1n);
  IKR_CUDA(cudaMemsetAsync(c->d_b1phi.p, 0, sizeof(double2) * b1n, st));
  launch_z_inverse<double>(c, c->occ, c->d_phi_all.p, ld, nullptr, c->d_b1phi.p);
  to_fp32(c, c->d_b1phi.p, b1n, c->d_b1phi32.p);
  c->d_psir.reserve((size_t)S * c->Ng);
  launch_synth_planes<double>(c, S, c->d_b1phi.p, c->d_psir.p);
  c->d_psir32.reserve((size_t)S * c->Ng);
  to_fp32(c, c->d_psir.p, (size_t)S * c->Ng, c->d_psir32.p);
  {
    const size_t n = (size_t)S * c->Ng;
    c->d_psir_df.reserve(n);
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 32);
    k_to_dfloat<<<blocks, 256, 0, st>>>(c->d_psir.p, n, c->d_psir_df.p);
    IKR_CUDA(cudaGetLastError());
  }
  // density rho = sum_k w_k sum_n f_nk |F^-1 phi_nk|^2 and K^xc[rho]
  std::vector<double> wf(S);
  for (int s = 0; s < S; ++s) wf[s] = w_o[s] * f_o[s];
  DBuf<double> d_wf;
  upload(d_wf, wf, st);
  c->d_rho.reserve(c->Ng);
  c->d_kxc.reserve(c->Ng);
  {
    const int blocks = (int)std::min<size_t>((c->Ng + 255) / 256, 152 * 16);
    k_rho_from_planes<<<blocks, 256, 0, st>>>(c->d_psir.p, S, c->N[0], c->N[1], c->N[2], d_wf.p, 1.0 / c->volume,
                                              c->d_rho.p);
    IKR_CUDA(cudaGetLastError());
  }
  exchange_kernel(c);
  {
    // ||K|| <= max 4 pi/|G|^2 + max |K^xc| (K^H and K^xc symmetric; K^xc <= 0)
    std::vector<double> kx(c->Ng);
    IKR_CUDA(cudaMemcpyAsync(kx.data(), c->d_kxc.p, sizeof(double) * c->Ng, cudaMemcpyDeviceToHost, st));
    IKR_CUDA(cudaStreamSynchronize(st));
    double kmax = 0.0, g2min = 1e300;
    for (double v : kx) kmax = std::max(kmax, std::fabs(v));
    // the smallest nonzero |G|^2 over the grid frequencies K^H acts on (for an oblique
    // cell a combination of reciprocal vectors can be shorter than each of them)
    const double* B = c->recip;
    for (int a = 0; a < c->N[0]; ++a)
      for (int b = 0; b < c->N[1]; ++b)
        for (int d = 0; d < c->N[2]; ++d) {
          const int j[3] = {signed_index(a, c->N[0]), signed_index(b, c->N[1]), signed_index(d, c->N[2])};
          if (j[0] == 0 && j[1] == 0 && j[2] == 0) continue;
          double g2 = 0.0;
          for (int r = 0; r < 3; ++r) {
            const double gr = B[3 * r] * j[0] + B[3 * r + 1] * j[1] + B[3 * r + 2] * j[2];
            g2 += gr * gr;
          }
          g2min = std::min(g2min, g2);
        }
    c->knorm = 4.0 * M_PI / g2min + kmax;
  }
  // ||F_k^-1 Phi_k||_{2,inf} and ||Re F_k^-1 Phi_k||_{2,inf} per k-point (largest
  // row norm over grid points; F^-1 phi = psi / sqrt|Omega| for the unnormalised
  // syntheses psi of the cached planes); the real part of every orbital is taken in
  // its most-real gauge, so neither norm depends on the eigenvectors' phases
  c->ws.grid1.reserve(c->Ng);
  c->ws.grid2.reserve(c->Ng);
  c->ws.scal.reserve(64);
  c->ws.cgrid.reserve(c->Ng);   // the orbitals' gauge phases (N_occ,k <= Ng entries)
  for (int ik = 0; ik < nk; ++ik) {
    orbital_sq_sums(c, c->d_psir.p + (size_t)off[ik] * c->Ng, noccs[ik], c->ws.grid1.p, c->ws.grid2.p,
                    c->ws.cgrid.p);
    grid_max(c, c->ws.grid1.p, c->Ng, c->ws.scal.p);
    grid_max(c, c->ws.grid2.p, c->Ng, c->ws.scal.p + 1);
    double mx[2] = {0, 0};
    IKR_CUDA(cudaMemcpyAsync(mx, c->ws.scal.p, sizeof(mx), cudaMemcpyDeviceToHost, st));
    IKR_CUDA(cudaStreamSynchronize(st));
    c->k[ik].rownorm = std::sqrt(mx[0] / c->volume);
    c->k[ik].rownorm_re = std::sqrt(mx[1] / c->volume);
  }
  IKR_CUDA(cudaStreamSynchronize(st));
  c->have_gs = true;
}

}  // namespace ikr
