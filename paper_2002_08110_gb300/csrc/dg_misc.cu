// Small kernels: stage-vector initialisation and the quadrature integrals.
#include <algorithm>

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
                            Tab1D<double> t, double detJ, const double* __restrict__ jx, int nqx,
                            long long ncx, double* __restrict__ partial) {
  __shared__ double s_m[256], s_l[256], s_x[256];
  double m = 0.0, l = 0.0, x = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_dofs;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    int q = static_cast<int>(i % npc);
    // curved x-mesh: detJ holds |J_v| and jx the |J_x| of each x point
    double w = jx ? detJ * jx[((i / npc) % ncx) * nqx + q % nqx] : detJ;
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
                             int blocks, double detJ, const double* jx, int nqx, cudaStream_t s) {
  const int d = p.dx + p.dv;
  int npc = 1;
  for (int k = 0; k < d; ++k) npc *= n;
  const long long n_dofs = p.ncells * npc;
  k_integrals<<<blocks, 256, 0, s>>>(u, n_dofs, npc, d, n, p.t64, detJ, jx, nqx, p.ncx, partial);
  return cudaGetLastError();
}

}  // namespace dg

namespace dg {

// Charge density rho = 1 - int f dv at every x node (Sec. 6: the reduction
// over velocity space that feeds the Poisson problem).  One block per x cell;
// thread (qx, lane) handles x node qx and every lanes-th (v cell, v node) pair
// in turn, accumulating |J_v| W_v(q_v) f in FP64; the lanes are then summed
// in a fixed order (deterministic).  A warp reads contiguous runs of the x
// nodes of consecutive v nodes.  n^dv <= 216 (degree <= 5, dim_v <= 3).
constexpr int kMaxNqv = 216;

template <typename TF>
__global__ void k_charge_density(const TF* __restrict__ f, long long ncx, long long ncv, int npc,
                                 int nqx, int nqv, int dv, int n, Tab1D<double> t, double detJv,
                                 double* __restrict__ rho) {
  __shared__ double s_w[kMaxNqv];
  extern __shared__ double s_part[];
  for (int q = threadIdx.x; q < nqv; q += blockDim.x) {
    double w = detJv;
    int r = q;
    for (int k = 0; k < dv; ++k) {
      w *= t.w[r % n];
      r /= n;
    }
    s_w[q] = w;
  }
  __syncthreads();
  const long long cx = blockIdx.x;
  const int lanes = blockDim.x / nqx;            // threads per x node (blockDim.x = lanes * nqx)
  const int qx = threadIdx.x % nqx;
  const int lane = threadIdx.x / nqx;
  double acc = 0.0;
  long long cv = lane / nqv;
  int qv = lane % nqv;
  const int step_cv = lanes / nqv, step_qv = lanes % nqv;
  while (cv < ncv) {
    acc += s_w[qv] * static_cast<double>(f[(cx + ncx * cv) * npc + qx + nqx * qv]);
    qv += step_qv;
    cv += step_cv;
    if (qv >= nqv) {
      qv -= nqv;
      ++cv;
    }
  }
  s_part[threadIdx.x] = acc;
  __syncthreads();
  if (lane == 0) {
    double s = 0.0;
    for (int l = 0; l < lanes; ++l) s += s_part[l * nqx + qx];
    rho[cx * nqx + qx] = 1.0 - s;
  }
}

cudaError_t launch_charge_density(const void* f, int f_is_float, long long ncx, long long ncv,
                                  int npc, int nqx, int nqv, int dv, int n,
                                  const Tab1D<double>& t, double detJv, double* rho,
                                  cudaStream_t s) {
  if (nqv > kMaxNqv || nqx > 256) return cudaErrorInvalidValue;
  const int threads = (256 / nqx) * nqx;         // a multiple of the x nodes per cell
  const size_t smem = sizeof(double) * threads;
  if (f_is_float)
    k_charge_density<float><<<static_cast<unsigned>(ncx), threads, smem, s>>>(
        static_cast<const float*>(f), ncx, ncv, npc, nqx, nqv, dv, n, t, detJv, rho);
  else
    k_charge_density<double><<<static_cast<unsigned>(ncx), threads, smem, s>>>(
        static_cast<const double*>(f), ncx, ncv, npc, nqx, nqv, dv, n, t, detJv, rho);
  return cudaGetLastError();
}

}  // namespace dg

namespace dg {

// Deterministic sum over the block (fixed shuffle tree, then the warp sums in
// order by thread 0); the result is returned to every thread.
__device__ double block_sum(double v, double* s_warp) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();                 // s_warp may still be read from the last call
  if (lane == 0) s_warp[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) s += s_warp[i];
    s_warp[32] = s;
  }
  __syncthreads();
  return s_warp[32];
}

// Periodic 1D Poisson problem of Sec. 6 (dim_x = 1): with E = -phi' and
// -phi'' = rho, E' = rho; periodicity needs the mean of rho removed and fixes
// E up to a constant, taken so that E has zero mean (phi periodic).  rho is
// the degree-k nodal polynomial of each cell; E is its exact antiderivative,
//   E(x_iq) = P_i + (h/2) sum_p Iq[q][p] (rho_ip - rho_bar),
// P_i = sum_{j<i} (h/2) sum_p w_p (rho_jp - rho_bar), evaluated at the nodes.
// One block: a chunked exclusive scan over the cells in a fixed order.
__global__ void k_poisson_1d(const double* __restrict__ rho, double* __restrict__ e,
                             long long ncx, int n, PoissonTab t, double hphys) {
  __shared__ double s_warp[33];
  __shared__ double s_scan[32];
  double loc = 0.0;
  for (long long c = threadIdx.x; c < ncx; c += blockDim.x)
    for (int p = 0; p < n; ++p) loc += t.w[p] * rho[c * n + p];
  // sum_c sum_p w_p rho = 2 ncx rho_bar (the cells' reference measure is 2)
  const double rho_bar = block_sum(loc, s_warp) / (2.0 * static_cast<double>(ncx));
  const double hh = 0.5 * hphys;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double carry = 0.0, emean = 0.0;
  for (long long base = 0; base < ncx; base += blockDim.x) {
    const long long c = base + threadIdx.x;
    double r[kMaxN] = {0.0};
    double ci = 0.0;
    if (c < ncx) {
      for (int p = 0; p < n; ++p) {
        r[p] = rho[c * n + p] - rho_bar;
        ci += t.w[p] * r[p];
      }
      ci *= hh;
    }
    // inclusive scan of ci over the chunk
    double incl = ci;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_scan[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      double run = 0.0;
      for (int i = 0; i < nw; ++i) {
        const double v = s_scan[i];
        s_scan[i] = run;
        run += v;
      }
      s_warp[32] = run;            // chunk total
    }
    __syncthreads();
    const double prefix = carry + s_scan[wid] + incl - ci;
    if (c < ncx) {
      double m = 0.0;
      for (int q = 0; q < n; ++q) {
        double s = 0.0;
        for (int p = 0; p < n; ++p) s += t.Iq[q * kMaxN + p] * r[p];
        const double eq = prefix + hh * s;
        e[c * n + q] = eq;
        m += t.w[q] * eq;
      }
      emean += 0.5 * m;
    }
    carry += s_warp[32];
    __syncthreads();               // s_scan and s_warp[32] are rewritten next chunk
  }
  const double e_bar = block_sum(emean, s_warp) / static_cast<double>(ncx);
  for (long long i = threadIdx.x; i < ncx * n; i += blockDim.x) e[i] -= e_bar;
}

cudaError_t launch_poisson_1d(const double* rho, double* e, long long ncx, int n,
                              const PoissonTab& t, double hphys, cudaStream_t s) {
  k_poisson_1d<<<1, 1024, 0, s>>>(rho, e, ncx, n, t, hphys);
  return cudaGetLastError();
}

struct Scale3 {
  double v[3];
};

// Contravariant v speeds from a device field: a_v = scale * e (the first
// comps components; the others zero), c_j = (2 / h_j) a_j at every x node.
// One thread per (x cell, v direction) also records whether the sign of
// c_j changes inside the cell (flag bit 0).  Non-finite values latch the
// handle's error word (bit 0, reported as non-finite by dg_check).
__global__ void k_field_speeds(const double* __restrict__ e, int comps, double scale,
                               long long ncx, int nq, int dv, Scale3 two_over_h,
                               double* __restrict__ cv64, float* __restrict__ cv32,
                               int* __restrict__ flags, int* __restrict__ err) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= ncx * dv) return;
  const long long cx = i / dv;
  const int j = static_cast<int>(i - cx * dv);
  // the cell's side is the sign of its largest speed; speeds of at most
  // 1e-12 of it are stored in FP32 as a zero with that sign (as on the host)
  double big = 0.0;
  bool bad = false;
  for (int q = 0; q < nq; ++q) {
    const long long node = cx * nq + q;
    const double c = two_over_h.v[j] * (j < comps ? scale * e[node * comps + j] : 0.0);
    bad |= !isfinite(c);
    if (fabs(c) > fabs(big)) big = c;
  }
  const double thr = 1e-12 * fabs(big);
  bool mixed = false;
  for (int q = 0; q < nq; ++q) {
    const long long node = cx * nq + q;
    const double c = two_over_h.v[j] * (j < comps ? scale * e[node * comps + j] : 0.0);
    cv64[node * dv + j] = c;
    if (fabs(c) <= thr) {
      cv32[node * dv + j] = big < 0.0 ? -0.0f : 0.0f;
    } else {
      cv32[node * dv + j] = static_cast<float>(c);
      mixed |= (c > 0.0) != (big > 0.0);
    }
  }
  if (mixed) atomicOr(flags, 1);
  if (bad) atomicOr(err, 1);
}

cudaError_t launch_field_speeds(const double* e, int comps, double scale, long long ncx, int nq,
                                int dv, const double* two_over_hv, double* cv64, float* cv32,
                                int* flags, int* err, cudaStream_t s) {
  Scale3 sc{{0.0, 0.0, 0.0}};
  for (int j = 0; j < dv; ++j) sc.v[j] = two_over_hv[j];
  const long long n = ncx * dv;
  const long long blocks = (n + 255) / 256;
  k_field_speeds<<<static_cast<unsigned>(blocks), 256, 0, s>>>(e, comps, scale, ncx, nq, dv, sc,
                                                               cv64, cv32, flags, err);
  return cudaGetLastError();
}

}  // namespace dg

namespace dg {

// Change of basis on every cell: y = (M (x) M (x) ... (x) M) x, the n x n
// matrix M applied along each of the d directions (tensor product, Sec. 2.3).
// With M = V (V_qi = phi_i(zeta_q)) it maps nodal values at the Gauss-Lobatto
// points to values at the Gauss-Legendre points; M = V^{-1} maps back; the
// transposes serve the adjoint.  Arithmetic in FP64.
//
// Shared-memory form: one block per cell at a time, the cell's values
// ping-pong between two shared arrays, one direction per pass.
template <typename TI, typename TO>
__global__ void k_basis_cells(const TI* __restrict__ x, TO* __restrict__ y, long long ncells, int d,
                              int n, int npc, BasisMat M) {
  extern __shared__ double sb[];
  for (long long cell = blockIdx.x; cell < ncells; cell += gridDim.x) {
    const size_t off = static_cast<size_t>(cell) * npc;
    for (int i = threadIdx.x; i < npc; i += blockDim.x) sb[i] = static_cast<double>(x[off + i]);
    __syncthreads();
    double* a = sb;
    double* b = sb + npc;
    int stride = 1;
    for (int j = 0; j < d; ++j) {
      for (int i = threadIdx.x; i < npc; i += blockDim.x) {
        const int pj = (i / stride) % n;
        const int base = i - pj * stride;
        double s = 0.0;
        for (int p = 0; p < n; ++p) s += M.m[pj * kMaxN + p] * a[base + p * stride];
        b[i] = s;
      }
      __syncthreads();
      double* tmp = a;
      a = b;
      b = tmp;
      stride *= n;
    }
    for (int i = threadIdx.x; i < npc; i += blockDim.x) y[off + i] = static_cast<TO>(a[i]);
    __syncthreads();
  }
}

// Global-memory form for cells too large for shared memory: one direction
// per launch, one output value per thread.
template <typename TI, typename TO>
__global__ void k_basis_dir(const TI* __restrict__ x, TO* __restrict__ y, long long n_dofs, int npc,
                            int stride, int n, BasisMat M) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_dofs;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(i % npc);
    const int pj = (q / stride) % n;
    const long long base = i - static_cast<long long>(pj) * stride;
    double s = 0.0;
    for (int p = 0; p < n; ++p) s += M.m[pj * kMaxN + p] * static_cast<double>(x[base + p * stride]);
    y[i] = static_cast<TO>(s);
  }
}

cudaError_t launch_basis_change(const void* x, int x_is_float, void* y, int y_is_float, double* tmp,
                                long long ncells, int d, int n, const BasisMat& M, cudaStream_t s) {
  int npc = 1;
  for (int j = 0; j < d; ++j) npc *= n;
  const size_t smem = 2 * static_cast<size_t>(npc) * sizeof(double);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem <= 200 * 1024) {
    const long long blocks = std::min<long long>(ncells, 8LL * sms);
    const int threads = npc >= 1024 ? 512 : 128;
    cudaError_t e;
#define DG_BC(TI, TO)                                                                            \
  do {                                                                                           \
    e = cudaFuncSetAttribute(k_basis_cells<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             static_cast<int>(smem));                                            \
    if (e != cudaSuccess) return e;                                                              \
    k_basis_cells<TI, TO><<<static_cast<unsigned>(blocks), threads, smem, s>>>(                  \
        static_cast<const TI*>(x), static_cast<TO*>(y), ncells, d, n, npc, M);                   \
  } while (0)
    if (x_is_float && y_is_float) DG_BC(float, float);
    else if (x_is_float) DG_BC(float, double);
    else if (y_is_float) DG_BC(double, float);
    else DG_BC(double, double);
#undef DG_BC
    return cudaGetLastError();
  }
  // d passes through FP64 temporaries: x -> tmp -> y -> tmp ... ending in y
  if (tmp == nullptr || x_is_float || y_is_float) return cudaErrorNotSupported;
  const long long n_dofs = ncells * npc;
  const long long blocks = std::min<long long>((n_dofs + 255) / 256, 16LL * sms);
  const double* in = static_cast<const double*>(x);
  int stride = 1;
  for (int j = 0; j < d; ++j) {
    double* out = ((d - 1 - j) % 2 == 0) ? static_cast<double*>(y) : tmp;
    k_basis_dir<double, double><<<static_cast<unsigned>(blocks), 256, 0, s>>>(in, out, n_dofs, npc,
                                                                               stride, n, M);
    in = out;
    stride *= n;
  }
  return cudaGetLastError();
}

}  // namespace dg

namespace dg {

// Element-wise helpers of the delta-f form (grid-stride loops).
__global__ void k_sub_to_f32(const double* __restrict__ a, const double* __restrict__ b,
                             float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = f64_to_f32(a[i] - b[i]);
}
__global__ void k_add_f32(const double* __restrict__ k, const float* __restrict__ y,
                          double* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    z[i] = k[i] + f32_to_f64(y[i]);
}
__global__ void k_axpy(double* __restrict__ x, double sc, const double* __restrict__ r, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    x[i] += sc * r[i];
}

static unsigned ew_blocks(long long n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return static_cast<unsigned>(std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * sms)));
}

cudaError_t launch_sub_to_f32(const double* a, const double* b, float* y, long long n, cudaStream_t s) {
  k_sub_to_f32<<<ew_blocks(n), 256, 0, s>>>(a, b, y, n);
  return cudaGetLastError();
}
cudaError_t launch_add_f32(const double* k, const float* y, double* z, long long n, cudaStream_t s) {
  k_add_f32<<<ew_blocks(n), 256, 0, s>>>(k, y, z, n);
  return cudaGetLastError();
}
cudaError_t launch_axpy(double* x, double sc, const double* r, long long n, cudaStream_t s) {
  k_axpy<<<ew_blocks(n), 256, 0, s>>>(x, sc, r, n);
  return cudaGetLastError();
}

// Scales every cell's values by a per-node factor (the node weights of the
// adjoint steps): blocks stride over cells, threads over the cell's nodes.
__global__ void k_scale_nodes(double* __restrict__ u, long long ncells, int npc,
                              const double* __restrict__ f) {
  for (long long c = blockIdx.x; c < ncells; c += gridDim.x)
    for (int q = threadIdx.x; q < npc; q += blockDim.x) u[c * npc + q] *= f[q];
}

cudaError_t launch_scale_nodes(double* u, long long ncells, int npc, const double* f, cudaStream_t s) {
  const int threads = npc >= 256 ? 256 : ((npc + 31) / 32) * 32;
  const long long grid = std::min<long long>(ncells, 152LL * 32);
  k_scale_nodes<<<static_cast<unsigned>(std::max<long long>(1, grid)), threads, 0, s>>>(u, ncells, npc, f);
  return cudaGetLastError();
}

}  // namespace dg
