// Specialised 5D cell kernel (dim_x = 2, dim_v = 3), n = 4 (k = 3), FP32
// sweeps and fluxes, FP32 or FP64 vectors.
//
// It computes the operator of the generic kernel (Algorithm 2: per direction
// the collocated 1D operator with the upwind flux and the inverse mass folded
// in, Gp / Gn and the lifts Lm / Lp of the tables; the weak form and upwind
// flux of Sec. 1.3, Eq. into:adv:ref) with every line a thread works on in
// registers.  A cell's 1024 values are indexed q = x + 16 m, x = x1 + 4 x2 the
// x node and m = v1 + 4 v2 + 16 v3 the v node.  64 threads per cell work in
// three phases, 16 values each:
//   phase A: thread m holds the x block of v node m (x1 and x2 lines local);
//            the x speeds depend on the v node only (a_x = v, Sec. 6);
//   phase B: thread (x, v3) holds the v1-v2 plane of x node x at v3 (v1 and
//            v2 lines local); the v speeds depend on the x node only (E(x));
//   phase C: thread (x, v1) holds the four v3 lines of x node x at v1.
// The residual passes between the phases through shared memory (columns of
// a v node padded to 20 floats, and a 16-float shift per v3 slab, so that the
// three views are free of bank conflicts); each thread reads its upwind
// neighbours' lines from global memory (L2) at the start of the phase, and the
// upwind side is chosen per thread, so speeds may change sign inside a cell
// (the 5D workload's E_3 does).  Phase C ends with the scatter or the fused
// LSRK stage update.  negate: the operator of the negated field (the adjoint
// steps run it on states scaled by the node weights).
#include "dg_convert.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kS5 = 1024;          // values per cell
constexpr int kCpb5 = 2;           // cells per block
constexpr int kT5 = 64 * kCpb5;    // threads per block

// shared-memory offset of element (x node, v node m): columns of 20 floats,
// plus 16 per v3 slab
__device__ __forceinline__ int off5(int x, int m) { return x + 20 * m + 16 * (m >> 4); }
constexpr int kCell5Smem = 20 * 64 + 16 * 4;   // floats per cell buffer

// One direction over the thread's 4 lines of 4 values: v[l][p] (line l,
// point p), nb the upwind neighbour's values at the same positions, c the
// speed of every line (per thread: the lines share their node outside the
// direction).  r += c (G u + L t).
__device__ __forceinline__ void dir5(float (&r)[4][4], const float (&u)[4][4], const float (&nb)[4][4],
                                     float c, const Tab1D<float>& T) {
  if (c == 0.f) return;
  const bool pos = c > 0.f;
  float G[16], L[4], l[4];
#pragma unroll
  for (int i = 0; i < 16; ++i) G[i] = pos ? T.Gp[i] : T.Gn[i];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L[q] = pos ? T.Lm[q] : -T.Lp[q];
    l[q] = pos ? T.lp[q] : T.lm[q];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) t = fmaf(l[q], nb[a][q], t);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float acc = L[q] * t;
#pragma unroll
      for (int s = 0; s < 4; ++s) acc = fmaf(G[q * 4 + s], u[a][s], acc);
      r[a][q] = fmaf(c, acc, r[a][q]);
    }
  }
}

// the same values seen along the other local digit: w[b][a] = v[a][b]
__device__ __forceinline__ void transpose4(float (&w)[4][4], const float (&v)[4][4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) w[b][a] = v[a][b];
}

template <typename TIN, typename TW, int MODE>
__global__ void __launch_bounds__(kT5, 4) k_cell5d(const KParams p) {
  __shared__ __align__(16) float su[kCpb5 * kCell5Smem];
  __shared__ __align__(16) float sr[kCpb5 * kCell5Smem];
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  const Tab1D<float>& T = p.t32;
  const unsigned ncells = static_cast<unsigned>(p.ncells);
  const unsigned cell0 = blockIdx.x * static_cast<unsigned>(kCpb5);
  const int nc = static_cast<int>(min(static_cast<unsigned>(kCpb5), ncells - cell0));
  const int c = threadIdx.x >> 6;            // cell slot
  const int t = threadIdx.x & 63;
  const bool active = c < nc;
  const unsigned cell = cell0 + static_cast<unsigned>(active ? c : 0);
  unsigned co[5];
  {
    unsigned rem = cell;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const unsigned nj = static_cast<unsigned>(p.ncell[j]);
      co[j] = rem % nj;
      rem /= nj;
    }
  }
  auto upwind = [&](int j, bool pos) -> unsigned {
    const unsigned st = static_cast<unsigned>(p.cstride[j]);
    const unsigned nj = static_cast<unsigned>(p.ncell[j]);
    unsigned nb;
    if (pos) nb = co[j] == 0 ? cell + (nj - 1) * st : cell - st;
    else nb = co[j] == nj - 1 ? cell - (nj - 1) * st : cell + st;
    DG_BOUND(p.err, nb, ncells);
    return nb;
  };
  const unsigned cx = co[0] + static_cast<unsigned>(p.ncell[0]) * co[1];
  const unsigned cv = co[2] + static_cast<unsigned>(p.ncell[2]) * (co[3] + static_cast<unsigned>(p.ncell[3]) * co[4]);
  const float sgn = p.negate ? -1.f : 1.f;
  float* const bu = su + c * kCell5Smem;
  float* const br = sr + c * kCell5Smem;
  auto ld = [&](unsigned cl, int q) { return cvt<float>(__ldg(src + static_cast<size_t>(cl) * kS5 + q)); };

  // gather the block's cells
  for (int i = threadIdx.x; i < nc * kS5; i += kT5) {
    const int cc = i >> 10, q = i & 1023;
    su[cc * kCell5Smem + off5(q & 15, q >> 4)] = cvt<float>(src[static_cast<size_t>(cell0) * kS5 + i]);
  }
  float u[4][4], r[4][4], nA[4][4], nB[4][4];

  // ---- phase A: thread t = v node m: x block, lines along x1 (u[x2][x1]) and x2
  const int m = t;
  float c0 = 0.f, c1 = 0.f;
  if (active) {
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * 64 + m) * 2;
    c0 = sgn * ctx[0];
    c1 = sgn * ctx[1];
    // the upwind neighbours' x blocks at v node m (16 contiguous values)
    const unsigned n0 = c0 != 0.f ? upwind(0, c0 > 0.f) : cell;
    const unsigned n1 = c1 != 0.f ? upwind(1, c1 > 0.f) : cell;
    if constexpr (sizeof(TIN) == 4) {
      // 16-byte aligned: the vectors are, and 16 m floats are 64 bytes
      const float4* pa = reinterpret_cast<const float4*>(src + static_cast<size_t>(n0) * kS5 + 16 * m);
      const float4* pb = reinterpret_cast<const float4*>(src + static_cast<size_t>(n1) * kS5 + 16 * m);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float4 va = __ldg(pa + b), vb = __ldg(pb + b);
        nA[b][0] = va.x; nA[b][1] = va.y; nA[b][2] = va.z; nA[b][3] = va.w;
        nB[b][0] = vb.x; nB[b][1] = vb.y; nB[b][2] = vb.z; nB[b][3] = vb.w;
      }
    } else {
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          nA[b][a] = ld(n0, a + 4 * b + 16 * m);
          nB[b][a] = ld(n1, a + 4 * b + 16 * m);
        }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4 v = *reinterpret_cast<const float4*>(bu + off5(4 * b, m));
      u[b][0] = v.x;
      u[b][1] = v.y;
      u[b][2] = v.z;
      u[b][3] = v.w;
#pragma unroll
      for (int a = 0; a < 4; ++a) r[b][a] = 0.f;
    }
    dir5(r, u, nA, c0, T);                       // x1: lines b (= x2), points a
    float ut[4][4], nt[4][4], rt[4][4];
    transpose4(ut, u);
    transpose4(nt, nB);
    transpose4(rt, r);
    dir5(rt, ut, nt, c1, T);                     // x2: lines a (= x1), points b
    transpose4(r, rt);
#pragma unroll
    for (int b = 0; b < 4; ++b)
      *reinterpret_cast<float4*>(br + off5(4 * b, m)) = make_float4(r[b][0], r[b][1], r[b][2], r[b][3]);
  }

  // ---- phase B: thread (x node xk, v3 j): the v1-v2 plane, u[v2][v1]
  const int xk = t & 15, j = t >> 4;
  float e0 = 0.f, e1 = 0.f, e2 = 0.f;
  if (active) {
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(cx) * 16 + xk) * 3;
    e0 = sgn * ctv[0];
    e1 = sgn * ctv[1];
    e2 = sgn * ctv[2];
    const unsigned n2 = e0 != 0.f ? upwind(2, e0 > 0.f) : cell;
    const unsigned n3 = e1 != 0.f ? upwind(3, e1 > 0.f) : cell;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int mm = a + 4 * b + 16 * j;
        nA[b][a] = ld(n2, xk + 16 * mm);
        nB[b][a] = ld(n3, xk + 16 * mm);
      }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int mm = a + 4 * b + 16 * j;
        u[b][a] = bu[off5(xk, mm)];
        r[b][a] = br[off5(xk, mm)];
      }
    dir5(r, u, nA, e0, T);                       // v1: lines b (= v2), points a
    float ut[4][4], nt[4][4], rt[4][4];
    transpose4(ut, u);
    transpose4(nt, nB);
    transpose4(rt, r);
    dir5(rt, ut, nt, e1, T);                     // v2: lines a (= v1), points b
    transpose4(r, rt);
  }
  __syncthreads();                               // every thread has read its phase B residual
  if (active) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) br[off5(xk, a + 4 * b + 16 * j)] = r[b][a];
  }

  // ---- phase C: thread (x node xk, v1 a3): four v3 lines (one per v2), u[v2][v3]
  const int a3 = t >> 4;
  if (active) {
    const unsigned n4 = e2 != 0.f ? upwind(4, e2 > 0.f) : cell;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) nA[b][jj] = ld(n4, xk + 16 * (a3 + 4 * b + 16 * jj));
  }
  __syncthreads();
  if (!active) return;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int mm = a3 + 4 * b + 16 * jj;
      u[b][jj] = bu[off5(xk, mm)];
      r[b][jj] = br[off5(xk, mm)];
    }
  dir5(r, u, nA, e2, T);                         // v3: lines b (= v2), points jj

  // ---- scatter / fused LSRK stage update (consecutive threads: consecutive x nodes)
  TW* __restrict__ dst = static_cast<TW*>(p.dst);
  const size_t g0 = static_cast<size_t>(cell) * kS5 + xk;
  float nanacc = 0.f;
  if constexpr (MODE == 0) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float K = r[b][jj];
        nanacc = fmaf(K, 0.f, nanacc);
        __stcs(dst + g0 + 16 * (a3 + 4 * b + 16 * jj), cvt<TW>(K));
      }
  } else {
    const float bf = static_cast<float>(p.b_dt), af = static_cast<float>(p.a_dt);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double ua[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) ua[jj] = __ldcs(p.u + g0 + 16 * (a3 + 4 * b + 16 * jj));
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const size_t g = g0 + 16 * (a3 + 4 * b + 16 * jj);
        const float K = r[b][jj];
        nanacc = fmaf(K, 0.f, nanacc);
        const double un = ua[jj] + f32_to_f64_finite(bf * K);
        __stcs(p.u + g, un);
        if constexpr (sizeof(TW) == 4)
          __stcs(dst + g, p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(ua[jj])));
        else
          __stcs(dst + g, p.last_stage ? un : ua[jj] + p.a_dt * f32_to_f64(K));
      }
    }
  }
  if (nanacc != 0.f) atomicOr(p.err, 1);
}

template <typename TIN, typename TW>
cudaError_t launch5(KParams& p, cudaStream_t s) {
  auto kern = p.mode == 0 ? k_cell5d<TIN, TW, 0> : k_cell5d<TIN, TW, 1>;
  const long long grid = (p.ncells + kCpb5 - 1) / kCpb5;
  kern<<<static_cast<unsigned>(grid), kT5, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cell_5d(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.dx != 2 || p.dv != 3 || n != 4 || cfg.variant != 2) return cudaErrorNotSupported;
  // not covered: the transpose (adjoint steps use the negated field on
  // scaled states), the delta-f stage, curved meshes, partial pencils
  if (p.adjoint || p.kref != nullptr || p.geo_c != nullptr || p.v3_n > 0) return cudaErrorNotSupported;
  if (p.ncells >= (1LL << 31) / kS5) return cudaErrorNotSupported;   // 32-bit cell indices
  if (combo == kFFF) return launch5<float, float>(p, s);
  if (combo == kFDD) return launch5<double, double>(p, s);
  return cudaErrorNotSupported;
}

}  // namespace dg
