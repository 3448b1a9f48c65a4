// Small kernels: stage-vector initialisation and the quadrature integrals.
#include "dg_convert.cuh"
#include "dg_internal.h"

namespace dg {

template <typename TW>
__global__ void k_convert(const double* __restrict__ u, TW* __restrict__ w, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    w[i] = cvt<TW>(u[i]);  // the same rounding as the fused stages' FP32 stage vectors
}

cudaError_t launch_convert(const double* u, void* w, int w_is_float, long long n, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 255) / 256;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  if (blocks < 1) blocks = 1;
  if (w_is_float)
    k_convert<float><<<static_cast<unsigned>(blocks), 256, 0, s>>>(u, static_cast<float*>(w), n);
  else
    k_convert<double><<<static_cast<unsigned>(blocks), 256, 0, s>>>(u, static_cast<double*>(w), n);
  return cudaGetLastError();
}

// Per-block partial sums of |J| W_q u_q, |J| W_q u_q^2 and max |u_q| (cell
// quadrature at the collocation nodes, Sec. 2.5).  FP64.
__global__ void k_integrals(const double* __restrict__ u, long long n_dofs, int npc, int d, int n,
                            Tab1D<double> t, double detJ, double* __restrict__ partial) {
  __shared__ double s_m[256], s_l[256], s_x[256];
  double m = 0.0, l = 0.0, x = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_dofs;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    int q = static_cast<int>(i % npc);
    double w = detJ;
    for (int k = 0; k < d; ++k) {
      w *= t.w[q % n];
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
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
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

cudaError_t launch_integrals(const KParams& p, int n, const double* u, double* partial,
                             int blocks, double detJ, cudaStream_t s) {
  const int d = p.dx + p.dv;
  int npc = 1;
  for (int k = 0; k < d; ++k) npc *= n;
  const long long n_dofs = p.ncells * npc;
  k_integrals<<<blocks, 256, 0, s>>>(u, n_dofs, npc, d, n, p.t64, detJ, partial);
  return cudaGetLastError();
}

}  // namespace dg
