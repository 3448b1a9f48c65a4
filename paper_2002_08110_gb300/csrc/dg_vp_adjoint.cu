// Pieces of the adjoint of one Vlasov-Poisson stage (Sec. 6, dim_x = 1).
//
// A stage's right-hand side is F(w) = L(a(w)) w with the field a_v1 = -E,
// E = P rho (the periodic Poisson solve) and rho = 1 - R w (R: the v
// quadrature at every x node).  For the upwind flux with its upwind sides
// fixed by the current field, L(a) w is linear in the field, so
//   dF = L(a) dw + B(w) da,   da = -dE = P R dw,
// where B(w) da is the operator along v1 with the speed (2/h_v1) da at every
// x node, applied to w.  The transpose is
//   J^T lam = L(a)^T lam + R^T P^T B(w)^T lam,
// and this file holds B^T, P^T and R^T (L^T is the library's transposed
// operator).  All three are FP64.
#include "dg_internal.h"

namespace dg {
namespace {

// sum of v over the block (every thread receives it); s: 33 doubles
__device__ double vpa_block_sum(double v, double* s) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();                       // s may still be read from a previous call
  if (lane == 0) s[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) t += s[i];
    s[32] = t;
  }
  __syncthreads();
  return s[32];
}

// g[x node] = (2 / h_v1) sum over the x node's DoFs of lam * (Gs w + Ls t),
// the unit-speed v1 operator of the line through the DoF (upwind side s
// fixed by the sign of the current speed c_v1 at the node, c >= 0 taken as
// positive; t the upwind v1 neighbour's trace).  One block per x cell,
// threads = lanes x (x nodes of the cell); a fixed summation order.
__global__ void k_field_adjoint(const double* __restrict__ w, const double* __restrict__ lam,
                                const double* __restrict__ cv64, long long ncx, long long ncv, int npc,
                                int nqx, int nqv, int n, int dv, long long ncv1, Tab1D<double> t,
                                double two_over_h, double* __restrict__ g) {
  extern __shared__ double s_part[];
  const long long cx = blockIdx.x;
  const int lanes = blockDim.x / nqx;
  const int qx = threadIdx.x % nqx;
  const int lane = threadIdx.x / nqx;
  const long long node = cx * nqx + qx;
  const bool pos = !(cv64[node * dv] < 0.0);
  const int nlines = nqv / n;                    // v1 lines of a cell at one x node
  double acc = 0.0;
  for (long long it = lane; it < ncv * nlines; it += lanes) {
    const long long cv = it / nlines;
    const int m = static_cast<int>(it - cv * nlines);
    const long long c1 = cv % ncv1;              // v1 cell coordinate
    long long nbv;                               // upwind v1 neighbour (periodic)
    if (pos) nbv = c1 == 0 ? cv + (ncv1 - 1) : cv - 1;
    else nbv = c1 == ncv1 - 1 ? cv - (ncv1 - 1) : cv + 1;
    const double* wc = w + (cx + ncx * cv) * npc + qx + static_cast<long long>(nqx) * n * m;
    const double* wn = w + (cx + ncx * nbv) * npc + qx + static_cast<long long>(nqx) * n * m;
    const double* lc = lam + (cx + ncx * cv) * npc + qx + static_cast<long long>(nqx) * n * m;
    double tr = 0.0;
    for (int p = 0; p < n; ++p) tr += (pos ? t.lp[p] : t.lm[p]) * wn[static_cast<long long>(nqx) * p];
    for (int q = 0; q < n; ++q) {
      double y = (pos ? t.Lm[q] : -t.Lp[q]) * tr;
      for (int p = 0; p < n; ++p) y += (pos ? t.Gp[q * n + p] : t.Gn[q * n + p]) * wc[static_cast<long long>(nqx) * p];
      acc += lc[static_cast<long long>(nqx) * q] * y;
    }
  }
  s_part[threadIdx.x] = acc;
  __syncthreads();
  if (lane == 0) {
    double s = 0.0;
    for (int l = 0; l < lanes; ++l) s += s_part[l * nqx + qx];
    g[node] = two_over_h * s;
  }
}

// out = P^T y for the periodic Poisson map rho -> E of k_poisson_1d:
//   r = rho - a (a . rho) ... written as E = (I - 1 b^T) M (I - 1 a^T) rho with
//   a_ip = w_p / (2 ncx), b_iq = w_q / (2 ncx),
//   M: E'_iq = sum_{j<i} hh sum_p w_p r_jp + hh sum_p Iq[q][p] r_ip,
// so P^T = (I - a 1^T) M^T (I - b 1^T):
//   y'_iq = y_iq - b_iq S (S = sum y),
//   z_jp = hh (w_p sum_{i>j} sum_q y'_iq + sum_q Iq[q][p] y'_jq),
//   out_jp = z_jp - a_jp Z (Z = sum z).
// sum_i sum_q y'_iq = 0, so the suffix sum is minus the inclusive prefix sum.
// One block: a chunked scan over the cells in a fixed order.
__global__ void k_poisson_1d_adjoint(const double* __restrict__ y, double* __restrict__ out,
                                     long long ncx, int n, PoissonTab t, double hphys) {
  __shared__ double s_red[33];
  __shared__ double s_scan[32];
  const double hh = 0.5 * hphys;
  double loc = 0.0;
  for (long long i = threadIdx.x; i < ncx * n; i += blockDim.x) loc += y[i];
  const double S = vpa_block_sum(loc, s_red);
  const double bS = S / (2.0 * static_cast<double>(ncx));   // b_iq S = w_q bS
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double carry = 0.0, zloc = 0.0;
  for (long long base = 0; base < ncx; base += blockDim.x) {
    const long long c = base + threadIdx.x;
    double yp[kMaxN] = {0.0};
    double Yc = 0.0;
    if (c < ncx) {
      for (int q = 0; q < n; ++q) {
        yp[q] = y[c * n + q] - t.w[q] * bS;
        Yc += yp[q];
      }
    }
    double incl = Yc;
    for (int o = 1; o < 32; o <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
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
      s_red[32] = run;
    }
    __syncthreads();
    const double prefix_incl = carry + s_scan[wid] + incl;   // sum_{i <= c} Y_i
    if (c < ncx) {
      const double suffix = -prefix_incl;                   // sum_{i > c} Y_i
      for (int p = 0; p < n; ++p) {
        double s = t.w[p] * suffix;
        for (int q = 0; q < n; ++q) s += t.Iq[q * kMaxN + p] * yp[q];
        const double z = hh * s;
        out[c * n + p] = z;
        zloc += z;
      }
    }
    carry += s_red[32];
    __syncthreads();
  }
  const double Z = vpa_block_sum(zloc, s_red);
  const double aZ = Z / (2.0 * static_cast<double>(ncx));
  for (long long i = threadIdx.x; i < ncx * n; i += blockDim.x) out[i] -= t.w[i % n] * aZ;
}

// out[i] += s_w[qv] m[x node of i], s_w[qv] = detJv prod of the v weights:
// R^T m for rho = 1 - R f (the v quadrature of k_charge_density).
__global__ void k_charge_adjoint_add(double* __restrict__ out, const double* __restrict__ m,
                                     long long ncx, long long ncells, int npc, int nqx, int n,
                                     int dv, Tab1D<double> t, double detJv) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < ncells * npc;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long cell = i / npc;
    const int q = static_cast<int>(i - cell * npc);
    const int qx = q % nqx;
    int qv = q / nqx;
    double sw = detJv;
    for (int k = 0; k < dv; ++k) {
      sw *= t.w[qv % n];
      qv /= n;
    }
    out[i] += sw * m[(cell % ncx) * nqx + qx];
  }
}

// y = a x + b z
__global__ void k_lincomb(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                          const double* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + b * z[i];
}

unsigned vpa_blocks(long long n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long b = (n + 255) / 256;
  return static_cast<unsigned>(b < 1 ? 1 : (b > 8LL * sms ? 8LL * sms : b));
}

}  // namespace

cudaError_t launch_field_adjoint(const double* w, const double* lam, const double* cv64, long long ncx,
                                 long long ncv, int npc, int nqx, int nqv, int n, int dv, long long ncv1,
                                 const Tab1D<double>& t, double two_over_h, double* g, cudaStream_t s) {
  if (nqx > 256) return cudaErrorInvalidValue;
  const int threads = (256 / nqx) * nqx;
  k_field_adjoint<<<static_cast<unsigned>(ncx), threads, sizeof(double) * threads, s>>>(
      w, lam, cv64, ncx, ncv, npc, nqx, nqv, n, dv, ncv1, t, two_over_h, g);
  return cudaGetLastError();
}

cudaError_t launch_poisson_1d_adjoint(const double* y, double* out, long long ncx, int n,
                                      const PoissonTab& t, double hphys, cudaStream_t s) {
  k_poisson_1d_adjoint<<<1, 1024, 0, s>>>(y, out, ncx, n, t, hphys);
  return cudaGetLastError();
}

cudaError_t launch_charge_adjoint_add(double* out, const double* m, long long ncx, long long ncells,
                                      int npc, int nqx, int n, int dv, const Tab1D<double>& t,
                                      double detJv, cudaStream_t s) {
  k_charge_adjoint_add<<<vpa_blocks(ncells * npc), 256, 0, s>>>(out, m, ncx, ncells, npc, nqx, n, dv, t,
                                                               detJv);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(double* y, double a, const double* x, double b, const double* z, long long n,
                           cudaStream_t s) {
  k_lincomb<<<vpa_blocks(n), 256, 0, s>>>(y, a, x, b, z, n);
  return cudaGetLastError();
}

}  // namespace dg
