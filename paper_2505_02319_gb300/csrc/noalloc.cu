// H_k psi without any device allocation at call time.
//
// Some callers cannot allocate device memory when they apply the Hamiltonian:
// code that records its GPU work into a CUDA graph by stream capture (a
// cudaMalloc during capture invalidates the capture), applications whose
// device memory is handed out by their own pool and must not be fragmented
// or exceeded, and latency-critical loops that must not enter the CUDA
// allocator.  ikr_apply_hamiltonian may grow the context's workspace; this
// entry point instead keeps its scratch (the z-transformed columns of every
// vector and the per-vector k index) in one file-scope device array of
// kScratchBytes, which every GPU that loads the library holds until the
// process exits.  It calls no cudaMalloc, cudaFree or allocating library
// routine.
#include <mutex>

#include "ops.hpp"

namespace ikr {

void launch_hamiltonian_raw(ikr_ctx* c, int n, const int* d_sysk, const double2* psi, int ld, double2* b1,
                            double2* b4, double2* hpsi);

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The host name g_scratch is only a stand-in: kernels need the device address,
// which cudaGetSymbolAddress gives per device (once, with that device current).
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

void* scratch_address() {
  int dev = 0;
  IKR_CUDA(cudaGetDevice(&dev));
  IKR_REQUIRE(dev >= 0 && dev < kMaxDevices, IKR_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      throw Error(IKR_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

__global__ void k_fill(int* __restrict__ p, int n, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

void hamiltonian_noalloc(ikr_ctx* c, int k, const double2* psi, double2* hpsi, int nvec) {
  const size_t per_vec = 2 * sizeof(double2) * (size_t)c->N[2] * c->ncp;   // b1 + b4 of one vector
  // chunk of nv vectors: 256-aligned index block, then b1 and b4
  int nv = 0;
  for (int t = 1; t <= nvec; t *= 2) {
    if (align256(sizeof(int) * t) + align256(per_vec / 2 * t) * 2 > kScratchBytes) break;
    nv = t;
  }
  if (nv == 0) {
    throw Error(IKR_ERR_ARG, "the grid needs " + std::to_string(per_vec) +
                                 " bytes of scratch per vector, more than the 32 MiB of the no-allocation path");
  }
  while (nv * 2 <= nvec && align256(sizeof(int) * nv * 2) + align256(per_vec / 2 * nv * 2) * 2 <= kScratchBytes)
    nv *= 2;
  unsigned char* base = static_cast<unsigned char*>(scratch_address());
  int* d_sysk = reinterpret_cast<int*>(base);
  double2* b1 = reinterpret_cast<double2*>(base + align256(sizeof(int) * nv));
  double2* b4 = reinterpret_cast<double2*>(base + align256(sizeof(int) * nv) + align256(per_vec / 2 * nv));
  // the k index block must hold k for every vector of a chunk; b1/b4 are fully
  // written before they are read, so nothing else needs clearing
  k_fill<<<(nv + 255) / 256, 256, 0, c->stream>>>(d_sysk, nv, k);
  IKR_CUDA(cudaGetLastError());
  const int nb = c->k[k].nb;
  for (int v0 = 0; v0 < nvec; v0 += nv) {
    const int n = std::min(nv, nvec - v0);
    launch_hamiltonian_raw(c, n, d_sysk, psi + (size_t)v0 * nb, nb, b1, b4, hpsi + (size_t)v0 * nb);
  }
}

}  // namespace ikr
