// Integrals of a state vector without any device allocation.
//
// dg_integrals() reduces through a partial-sum buffer that the handle
// allocates.  This file provides the same reduction for callers that cannot
// allocate device memory: its scratch is a fixed array compiled into the
// library, and it needs no handle.  The paper has no counterpart; it is a
// convenience of this library.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dg_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 1LL << 20;          // DoFs reduced by one block
constexpr int kMaxBlocks = 4096;                 // so at most 2^32 DoFs per call
constexpr int kScratchDoubles = 3 * kMaxBlocks + 3;

// Per-block partial sums (3 per block) followed by the 3 final results:
// 98,328 bytes, resident on every device that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on device `dev` (which must be the
// current device); looked up once per device and kept for the life of the
// process.  The address belongs to the device context that was current at
// the lookup, so the cache is not valid across cudaDeviceReset.
cudaError_t scratch_on(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct Weights {
  double w[dg::kMaxN];
};

// Block b reduces DoFs [b * kChunk, min((b + 1) * kChunk, n_dofs)): sums of
// |J| W_q u_q and |J| W_q u_q^2 and the max of |u_q| (cell quadrature at the
// collocation nodes, W_q the product of the 1D weights of node q).
__global__ void k_block_partials(const double* __restrict__ u, long long n_dofs, int npc, int d,
                                 int n, Weights wt, double detJ, double* __restrict__ partial) {
  __shared__ double s_m[kThreads], s_l[kThreads], s_x[kThreads];
  const long long begin = static_cast<long long>(blockIdx.x) * kChunk;
  const long long end = begin + kChunk < n_dofs ? begin + kChunk : n_dofs;
  double m = 0.0, l = 0.0, x = 0.0;
  for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
    int q = static_cast<int>(i % npc);
    double w = detJ;
    for (int k = 0; k < d; ++k) {
      w *= wt.w[q % n];
      q /= n;
    }
    const double v = u[i];
    m += w * v;
    l += w * v * v;
    x = fmax(x, fabs(v));
  }
  s_m[threadIdx.x] = m;
  s_l[threadIdx.x] = l;
  s_x[threadIdx.x] = x;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_m[threadIdx.x] += s_m[threadIdx.x + o];
      s_l[threadIdx.x] += s_l[threadIdx.x + o];
      s_x[threadIdx.x] = fmax(s_x[threadIdx.x], s_x[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x + 0] = s_m[0];
    partial[3 * blockIdx.x + 1] = s_l[0];
    partial[3 * blockIdx.x + 2] = s_x[0];
  }
}

// One block folds the `blocks` partial triples into result[0..2].
__global__ void k_fold(const double* __restrict__ partial, int blocks, double* __restrict__ result) {
  __shared__ double s_m[kThreads], s_l[kThreads], s_x[kThreads];
  double m = 0.0, l = 0.0, x = 0.0;
  for (int b = threadIdx.x; b < blocks; b += kThreads) {
    m += partial[3 * b];
    l += partial[3 * b + 1];
    x = fmax(x, partial[3 * b + 2]);
  }
  s_m[threadIdx.x] = m;
  s_l[threadIdx.x] = l;
  s_x[threadIdx.x] = x;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_m[threadIdx.x] += s_m[threadIdx.x + o];
      s_l[threadIdx.x] += s_l[threadIdx.x + o];
      s_x[threadIdx.x] = fmax(s_x[threadIdx.x], s_x[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    result[0] = s_m[0];
    result[1] = s_l[0];
    result[2] = s_x[0];
  }
}

}  // namespace

extern "C" dg_status dg_integrals_noalloc(const double* u, long long n_cells, int dim, int degree,
                                          int basis, double det_jacobian, double* out,
                                          void* stream) {
  char msg[256];
  if (u == nullptr || out == nullptr) return dg::report(DG_ERR_INVALID_ARG, "u and out must not be NULL");
  if (reinterpret_cast<uintptr_t>(u) % 16 != 0)
    return dg::report(DG_ERR_INVALID_ARG, "u is not 16-byte aligned");
  if (dim < 2 || dim > 6 || degree < 1 || degree > 5)
    return dg::report(DG_ERR_UNSUPPORTED, "dim must be in [2, 6] and degree in [1, 5]");
  if (n_cells < 1) return dg::report(DG_ERR_INVALID_ARG, "n_cells must be >= 1");
  // the collocated bases integrate at their own nodes; the Lobatto-node,
  // Gauss-quadrature element needs a change of basis (dg_integrals does it)
  if (basis == DG_BASIS_GLL_GAUSS)
    return dg::report(DG_ERR_UNSUPPORTED,
                      "dg_integrals_noalloc covers the collocated bases only; use dg_integrals "
                      "for DG_BASIS_GLL_GAUSS");
  if (basis != DG_BASIS_GL && basis != DG_BASIS_GLL)
    return dg::report(DG_ERR_INVALID_ARG, "unknown basis");
  if (!(det_jacobian > 0.0) || !std::isfinite(det_jacobian))
    return dg::report(DG_ERR_INVALID_ARG, "det_jacobian must be positive and finite");
  const int n = degree + 1;
  int npc = 1;
  for (int k = 0; k < dim; ++k) npc *= n;
  const long long limit = kChunk * kMaxBlocks;
  if (n_cells > limit / npc) {
    std::snprintf(msg, sizeof(msg),
                  "n_cells * (degree+1)^dim exceeds the %lld DoFs that the fixed scratch of "
                  "dg_integrals_noalloc covers; use dg_integrals",
                  limit);
    return dg::report(DG_ERR_INVALID_ARG, msg);
  }
  const long long n_dofs = n_cells * npc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return dg::report(DG_ERR_CUDA, "dg_integrals_noalloc: no usable current device");
  double* scratch = nullptr;
  if ((e = scratch_on(dev, &scratch)) != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "dg_integrals_noalloc: scratch lookup failed: %s",
                  cudaGetErrorString(e));
    return dg::report(DG_ERR_CUDA, msg);
  }
  Weights wt{};
  double nodes[dg::kMaxN];
  if (basis == DG_BASIS_GL)
    dg::gauss_legendre(n, nodes, wt.w);
  else
    dg::gauss_lobatto(n, nodes, wt.w);
  const int blocks = static_cast<int>((n_dofs + kChunk - 1) / kChunk);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every partial slot read by k_fold is written by this call first, so the
  // array needs no clearing
  k_block_partials<<<blocks, kThreads, 0, s>>>(u, n_dofs, npc, dim, n, wt, det_jacobian, scratch);
  k_fold<<<1, kThreads, 0, s>>>(scratch, blocks, scratch + 3 * kMaxBlocks);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(out, scratch + 3 * kMaxBlocks, 3 * sizeof(double),
                           cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "dg_integrals_noalloc: %s", cudaGetErrorString(e));
    return dg::report(DG_ERR_CUDA, msg);
  }
  return DG_OK;
}
