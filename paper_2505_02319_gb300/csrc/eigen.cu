// Lowest eigenpairs of the plane-wave Hamiltonians H_k (eq. Hamiltonian, the
// k-form of Sec. 4.1.1) on the GPU, without forming H_k: Chebyshev-filtered
// subspace iteration (Zhou, Saad, Tiago, Chelikowsky, J. Comput. Phys. 219
// (2006), with their scaled three-term filter).  Per k-point, a block of m
// vectors (the wanted bands plus a buffer) is
//   1. filtered by the Chebyshev polynomial of degree d that damps the
//      interval [theta_max, b_up] (theta_max the largest Ritz value of the
//      block, b_up >= lambda_max(H_k)), using the library's H_k kernels;
//   2. orthonormalised by SVQB twice (Stathopoulos & Wu 2002): with
//      S = Y^H Y and D = diag(S)^-1/2, D S D = U L U^H gives
//      Y <- Y D U L^-1/2;
//   3. rotated to Ritz vectors by the Rayleigh-Ritz step on Y^H H Y.
// It stops when every wanted band has ||H x - theta x|| <= tol.  The Gram and
// rotation products are cuBLAS ZGEMMs; the m x m Hermitian eigenproblems are
// solved on the host by cyclic Jacobi rotations.  This is setup (the paper
// takes the ground state from an SCF); the response solver is unchanged.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>

#include "solver.hpp"

namespace ikr {

using zc = std::complex<double>;

// ---------------------------------------------------------- host Jacobi --
// A (n x n, row-major, Hermitian) is diagonalised by rotations in the (p, q)
// planes: with a_pq = |a_pq| e^{i phi}, D = diag(1, e^{-i phi}) makes the 2 x 2
// block real, and the classical real rotation (cot 2t = (a_qq - a_pp) / 2|a_pq|)
// zeroes it; U = D P is applied as A <- U^H A U, V <- V U.  On return w holds
// the eigenvalues in ascending order and column j of V (V[i n + j]) the
// eigenvector of w[j].
void herm_jacobi(int n, std::vector<zc>& A, std::vector<double>& w, std::vector<zc>& V) {
  V.assign((size_t)n * n, zc(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = std::norm(A[(size_t)i * n + j]);
        tot += a;
        if (i != j) off += a;
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const zc apq = A[(size_t)p * n + q];
        const double mag = std::abs(apq);
        if (mag == 0.0) continue;
        const double app = A[(size_t)p * n + p].real(), aqq = A[(size_t)q * n + q].real();
        if (mag < 1e-18 * (std::fabs(app) + std::fabs(aqq)) && sweep > 3) {
          A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
          continue;
        }
        const zc ph = apq / mag;
        const double th = (aqq - app) / (2.0 * mag);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        const zc cph = std::conj(ph);
        for (int i = 0; i < n; ++i) {   // A <- A U
          const zc aip = A[(size_t)i * n + p], aiq = A[(size_t)i * n + q];
          A[(size_t)i * n + p] = c * aip - s * cph * aiq;
          A[(size_t)i * n + q] = s * aip + c * cph * aiq;
        }
        for (int j = 0; j < n; ++j) {   // A <- U^H A
          const zc apj = A[(size_t)p * n + j], aqj = A[(size_t)q * n + j];
          A[(size_t)p * n + j] = c * apj - s * ph * aqj;
          A[(size_t)q * n + j] = s * apj + c * ph * aqj;
        }
        for (int i = 0; i < n; ++i) {   // V <- V U
          const zc vip = V[(size_t)i * n + p], viq = V[(size_t)i * n + q];
          V[(size_t)i * n + p] = c * vip - s * cph * viq;
          V[(size_t)i * n + q] = s * vip + c * cph * viq;
        }
        A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
        A[(size_t)p * n + p] = app - t * mag;
        A[(size_t)q * n + q] = aqq + t * mag;
      }
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return A[(size_t)a * n + a].real() < A[(size_t)b * n + b].real(); });
  std::vector<zc> Vs((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]].real();
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(Vs);
}

namespace {

// out = al (HY - c Y) + be X, element by element (out may alias X)
__global__ void k_cheb(double2* out, const double2* __restrict__ HY, const double2* __restrict__ Y, const double2* X,
                       size_t n, double al, double c, double be) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 h = HY[i], y = Y[i];
    double2 o = make_double2(al * (h.x - c * y.x), al * (h.y - c * y.y));
    if (be != 0.0) {
      const double2 x = X[i];
      o.x += be * x.x;
      o.y += be * x.y;
    }
    out[i] = o;
  }
}

// starting block: column j is the plane wave idx[j] plus 1e-2 times a
// deterministic pseudo-random vector (a 32-bit integer hash of (j, g))
__global__ void k_block_init(double2* X, int nb, int m, const int* __restrict__ idx) {
  const size_t n = (size_t)nb * m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / nb), g = (int)(e - (size_t)j * nb);
    unsigned h = 2654435761u * (unsigned)(j + 1) ^ (2246822519u * (unsigned)(g + 7));
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    const double r = ((double)(h & 0xffffu) / 65536.0 - 0.5) * 1e-2;
    const double i = ((double)(h >> 16) / 65536.0 - 0.5) * 1e-2;
    X[e] = make_double2((g == idx[j] ? 1.0 : 0.0) + r, i);
  }
}

// res[j] = ||HX_j - theta_j X_j||^2 (one block per column, fixed-order reduction)
__global__ void k_col_res(const double2* __restrict__ HX, const double2* __restrict__ X,
                          const double* __restrict__ theta, int nb, double* __restrict__ res) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const double t = theta[j];
  double a = 0.0;
  for (int g = threadIdx.x; g < nb; g += blockDim.x) {
    const double2 h = HX[(size_t)j * nb + g], x = X[(size_t)j * nb + g];
    const double rx = h.x - t * x.x, ry = h.y - t * x.y;
    a += rx * rx + ry * ry;
  }
  a = block_sum(a, sh);
  if (threadIdx.x == 0) res[j] = a;
}

void cublas_check(cublasStatus_t s, const char* what) {
  if (s != CUBLAS_STATUS_SUCCESS) throw Error(IKR_ERR_CUDA, std::string("cuBLAS failed: ") + what);
}

struct Chfsi {
  ikr_ctx* c;
  cublasHandle_t h;
  int nb, m;
  DBuf<double2> S;
  std::vector<zc> hS;

  // S (m x m, host row-major) = A^H B
  void gram(const double2* A, const double2* B) {
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    cublas_check(cublasZgemm(h, CUBLAS_OP_C, CUBLAS_OP_N, m, m, nb, &one, reinterpret_cast<const cuDoubleComplex*>(A),
                             nb, reinterpret_cast<const cuDoubleComplex*>(B), nb, &zero,
                             reinterpret_cast<cuDoubleComplex*>(S.p), m),
                 "gram");
    std::vector<double2> t((size_t)m * m);
    IKR_CUDA(cudaMemcpyAsync(t.data(), S.p, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, c->stream));
    IKR_CUDA(cudaStreamSynchronize(c->stream));
    hS.resize((size_t)m * m);
    for (int i = 0; i < m; ++i)   // column-major (i, j) at i + j m
      for (int j = 0; j < m; ++j) hS[(size_t)i * m + j] = zc(t[i + (size_t)j * m].x, t[i + (size_t)j * m].y);
  }
  // out = A T, T (m x m) given host row-major
  void rotate(const double2* A, const std::vector<zc>& T, double2* out) {
    std::vector<double2> t((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) t[i + (size_t)j * m] = make_double2(T[(size_t)i * m + j].real(), T[(size_t)i * m + j].imag());
    IKR_CUDA(cudaMemcpyAsync(S.p, t.data(), sizeof(double2) * m * m, cudaMemcpyHostToDevice, c->stream));
    const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
    cublas_check(cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, nb, m, m, &one, reinterpret_cast<const cuDoubleComplex*>(A),
                             nb, reinterpret_cast<const cuDoubleComplex*>(S.p), m, &zero,
                             reinterpret_cast<cuDoubleComplex*>(out), nb),
                 "rotate");
    IKR_CUDA(cudaStreamSynchronize(c->stream));   // t is a host temporary
  }
  // out = A orthonormalised (SVQB)
  void svqb(const double2* A, double2* out) {
    gram(A, A);
    std::vector<double> d(m);
    for (int i = 0; i < m; ++i) {
      const double sii = hS[(size_t)i * m + i].real();
      d[i] = sii > 0.0 ? 1.0 / std::sqrt(sii) : 1.0;
    }
    std::vector<zc> M((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const zc v = 0.5 * (hS[(size_t)i * m + j] + std::conj(hS[(size_t)j * m + i]));
        M[(size_t)i * m + j] = d[i] * v * d[j];
      }
    std::vector<double> lam;
    std::vector<zc> U;
    herm_jacobi(m, M, lam, U);
    const double lmax = std::max(lam[m - 1], 1e-300);
    std::vector<zc> T((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) T[(size_t)i * m + j] = d[i] * U[(size_t)i * m + j] / std::sqrt(std::max(lam[j], 1e-15 * lmax));
    rotate(A, T, out);
  }
  // Rayleigh-Ritz: theta ascending, X = Y Q, HX = HY Q
  void rr(const double2* Y, const double2* HY, double2* X, double2* HX, std::vector<double>& theta) {
    gram(Y, HY);
    std::vector<zc> M((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) M[(size_t)i * m + j] = 0.5 * (hS[(size_t)i * m + j] + std::conj(hS[(size_t)j * m + i]));
    std::vector<zc> Q;
    herm_jacobi(m, M, theta, Q);
    rotate(Y, Q, X);
    rotate(HY, Q, HX);
  }
};

void elementwise_grid(size_t n, int* blocks) { *blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

std::vector<EigenStats> compute_eigenpairs(ikr_ctx* c, int nbands, double tol, int maxit, int degree,
                                           std::vector<DBuf<double2>>& vecs, std::vector<double>& eps) {
  const int nk = (int)c->k.size();
  IKR_REQUIRE(nbands >= 1 && tol > 0.0 && maxit >= 1 && degree >= 2, IKR_ERR_ARG, "invalid eigensolver options");
  std::vector<EigenStats> stats(nk);
  vecs.resize(nk);
  eps.assign((size_t)nk * nbands, 0.0);
  cublasHandle_t h = nullptr;
  cublas_check(cublasCreate(&h), "create");
  struct Guard {
    cublasHandle_t h;
    ~Guard() { cublasDestroy(h); }
  } guard{h};
  cublas_check(cublasSetStream(h, c->stream), "stream");
  for (int k = 0; k < nk; ++k) {
    const KPoint& K = c->k[k];
    const int nb = K.nb;
    IKR_REQUIRE(nbands <= nb, IKR_ERR_ARG, "nbands exceeds the basis size");
    const int m = std::min(nb, nbands + std::max(4, nbands / 4));
    Chfsi ch{c, h, nb, m, {}, {}};
    ch.S.reserve((size_t)m * m);
    DBuf<double2> B0, B1, B2, B3;
    for (auto* b : {&B0, &B1, &B2, &B3}) b->reserve((size_t)nb * m);
    DBuf<double> dres, dth;
    dres.reserve(m);
    dth.reserve(m);
    DBuf<int> didx;
    // starting block: the m plane waves of lowest kinetic energy
    std::vector<int> ord(nb);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return K.kin[a] < K.kin[b]; });
    ord.resize(m);
    didx.reserve(m);
    IKR_CUDA(cudaMemcpyAsync(didx.p, ord.data(), sizeof(int) * m, cudaMemcpyHostToDevice, c->stream));
    const size_t n = (size_t)nb * m;
    int blocks = 0;
    elementwise_grid(n, &blocks);
    k_block_init<<<blocks, 256, 0, c->stream>>>(B0.p, nb, m, didx.p);
    IKR_CUDA(cudaGetLastError());
    // upper bound of the spectrum: max kinetic energy + max V + ||V_nl||, with
    // ||B diag(D) B^H|| <= max(D, 0) ||B^H B|| <= max(D, 0) max_i sum_j |(B^H B)_ij|
    double vnl = 0.0;
    if (c->nproj > 0) {
      const int np = c->nproj;
      DBuf<double2> G;
      G.reserve((size_t)np * np);
      const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
      const cuDoubleComplex* Bk = reinterpret_cast<const cuDoubleComplex*>(c->d_kb.p + (size_t)k * np * c->ld);
      cublas_check(cublasZgemm(h, CUBLAS_OP_C, CUBLAS_OP_N, np, np, nb, &one, Bk, c->ld, Bk, c->ld, &zero,
                               reinterpret_cast<cuDoubleComplex*>(G.p), np),
                   "projector gram");
      std::vector<double2> hg((size_t)np * np);
      IKR_CUDA(cudaMemcpyAsync(hg.data(), G.p, sizeof(double2) * np * np, cudaMemcpyDeviceToHost, c->stream));
      IKR_CUDA(cudaStreamSynchronize(c->stream));
      double rowmax = 0.0;
      for (int i = 0; i < np; ++i) {
        double r = 0.0;
        for (int j = 0; j < np; ++j) r += std::hypot(hg[i + (size_t)j * np].x, hg[i + (size_t)j * np].y);
        rowmax = std::max(rowmax, r);
      }
      vnl = std::max(c->kb_dmax, 0.0) * rowmax;
    }
    const double bup = (*std::max_element(K.kin.begin(), K.kin.end()) + c->vmax + vnl) * 1.01 + 0.1;
    double2 *X = B0.p, *Y = B1.p, *HX = B2.p, *T = B3.p;
    ch.svqb(X, Y);
    ch.svqb(Y, X);
    hamiltonian<double>(c, k, X, HX, nb, m);
    std::vector<double> theta;
    ch.rr(X, HX, Y, T, theta);
    std::swap(X, Y);
    std::swap(HX, T);
    int it = 0;
    double rmax = 0.0;
    for (;; ++it) {
      IKR_CUDA(cudaMemcpyAsync(dth.p, theta.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
      k_col_res<<<nbands, 256, 0, c->stream>>>(HX, X, dth.p, nb, dres.p);
      IKR_CUDA(cudaGetLastError());
      std::vector<double> r2(nbands);
      IKR_CUDA(cudaMemcpyAsync(r2.data(), dres.p, sizeof(double) * nbands, cudaMemcpyDeviceToHost, c->stream));
      IKR_CUDA(cudaStreamSynchronize(c->stream));
      rmax = 0.0;
      for (double v : r2) rmax = std::max(rmax, std::sqrt(std::max(v, 0.0)));
      if (rmax <= tol || it >= maxit) break;
      // scaled Chebyshev filter of degree `degree` damping [theta_max, bup]
      const double a = theta[m - 1], a0 = theta[0];
      const double e = (bup - a) / 2.0, cen = (bup + a) / 2.0;
      double sigma = e / (a0 - cen);
      const double tau = 2.0 / sigma;
      // Y = (H X - c X) sigma / e   (HX holds H X)
      k_cheb<<<blocks, 256, 0, c->stream>>>(Y, HX, X, nullptr, n, sigma / e, cen, 0.0);
      IKR_CUDA(cudaGetLastError());
      for (int d = 2; d <= degree; ++d) {
        const double s2 = 1.0 / (tau - sigma);
        hamiltonian<double>(c, k, Y, T, nb, m);
        // X <- 2 s2 / e (H Y - c Y) - sigma s2 X, then (X, Y) <- (Y, X)
        k_cheb<<<blocks, 256, 0, c->stream>>>(X, T, Y, X, n, 2.0 * s2 / e, cen, -sigma * s2);
        IKR_CUDA(cudaGetLastError());
        std::swap(X, Y);
        sigma = s2;
      }
      // orthonormalise the filtered block (in Y), Rayleigh-Ritz
      ch.svqb(Y, X);
      ch.svqb(X, Y);
      hamiltonian<double>(c, k, Y, T, nb, m);
      ch.rr(Y, T, X, HX, theta);
    }
    stats[k].iters = it;
    stats[k].max_residual = rmax;
    for (int j = 0; j < nbands; ++j) eps[(size_t)k * nbands + j] = theta[j];
    vecs[k].reserve((size_t)nb * nbands);
    IKR_CUDA(cudaMemcpyAsync(vecs[k].p, X, sizeof(double2) * nb * nbands, cudaMemcpyDeviceToDevice, c->stream));
    IKR_CUDA(cudaStreamSynchronize(c->stream));
  }
  return stats;
}

}  // namespace ikr
