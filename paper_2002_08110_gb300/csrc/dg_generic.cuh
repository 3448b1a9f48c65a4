// Generic element-centric DG advection cell kernel (any d <= 6, n <= 6).
//
// One block processes ``cells_per_block`` cells (Algorithm 1: the loop over
// cell pairs (c_x, c_v) is the grid).  Per cell (Algorithm 2):
//   1. gather the n^d values of the input into shared memory;
//   2./3. for each direction j, every line of n values along j is contracted
//      with the collocated 1D operator (cell term of direction j, both faces
//      normal to j with the upwind flux, inverse mass; see Tab1D).  The
//      neighbour's trace is needed on inflow faces only; it is computed from
//      the neighbour's line read from global memory (periodic wrap, tensor
//      product cell index);
//   4. the inverse mass is already folded into the 1D operator;
//   5. scatter (or the fused LSRK stage update).
// Directions are processed one after another with a block barrier between
// them; within a direction the lines are disjoint, so the accumulation into
// the per-cell residual needs no atomics (the element-centric loop writes
// every DoF exactly once, Sec. 2.6).  Each direction is a separate
// instantiation (its line stride is a constant), and the cells' x / v cell
// indices and upwind neighbours are computed once per cell into shared
// memory, so the lines do no 64-bit integer division.
//
// Large cells (6D with n >= 5 in FP64, n = 6 in FP32) do not fit in shared
// memory: then the block reads the cell from global memory and accumulates in
// a per-block slab of scratch memory, looping over cells persistently.
#pragma once

#include "dg_convert.cuh"
#include "dg_internal.h"

namespace dg {

template <int B, int E>
struct Pow { static constexpr int v = B * Pow<B, E - 1>::v; };
template <int B>
struct Pow<B, 0> { static constexpr int v = 1; };

template <typename T>
__device__ __forceinline__ const Tab1D<T>& tab(const KParams& p);
template <>
__device__ __forceinline__ const Tab1D<double>& tab<double>(const KParams& p) { return p.t64; }
template <>
__device__ __forceinline__ const Tab1D<float>& tab<float>(const KParams& p) { return p.t32; }

// Product of the 1D weights (or inverse weights) over the d digits of node q.
template <int D, int N, typename TC>
__device__ __forceinline__ TC node_weight(const TC* w1, int q) {
  TC r = TC(1);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    r *= w1[q % N];
    q /= N;
  }
  return r;
}


// Per-cell bookkeeping kept in shared memory for a block's cells: the x cell,
// the v cell and the upwind neighbours (below, above) in every direction, so
// that the lines of a direction do no 64-bit division.
template <int D>
struct CellInfo {
  static constexpr int kLen = 2 + 2 * D;
};

// One x line of a curved x-mesh (DXN = dim_x at compile time, so that the
// loops over the Jacobian's components unroll).  Curved x-mesh: the flux speed
// g = |J_x| c_j varies along the line.  With collocation the line's weak form
// divided by the diagonal mass reads du_q = (1/|J_x,q|) [sum_p Dt[q][p] g_p u_p
// - Lp[q] F(+1) + Lm[q] F(-1)], F(+-1) = g(+-1) u*(+-1) with the upwind state
// at each face.
template <int DXN, int D, int N, typename TC, typename TIN, bool SMEM, int J>
__device__ __forceinline__ void curved_line(const KParams& p, const Tab1D<TC>& T, const TIN* src,
                                            const TC* su, TC* sr, const long long* ci, int c,
                                            long long cell, int base, int qx, int qv, int nqx, int nqv) {
  constexpr int NP = Pow<N, D>::v;
  constexpr int sj = Pow<N, J>::v;
  const long long cx = ci[0], cv = ci[1];
  constexpr int dxn = DXN, sc = 1 + DXN * DXN;
  const TC* A = static_cast<const TC*>(p.ax_tab) + (cv * nqv + qv) * dxn;
  const TC* Gc = static_cast<const TC*>(p.geo_c) + cx * nqx * sc;
  TC uu[N], g[N], ij[N];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    uu[q] = SMEM ? su[c * NP + base + q * sj] : cvt<TC>(src[cell * NP + base + q * sj]);
    const TC* gq = Gc + (qx + q * sj) * sc;
    TC cq = TC(0);
#pragma unroll
    for (int m = 0; m < dxn; ++m) cq += gq[1 + J * dxn + m] * A[m];
    g[q] = cq;
    ij[q] = gq[0];                       // 1 / |J_x| at the point
  }
  int f = 0, mul = 1, rr = qx, nf = 1;
#pragma unroll
  for (int m = 0; m < dxn; ++m) {
    const int dg = rr % N;
    rr /= N;
    if (m != J) {
      f += dg * mul;
      mul *= N;
      nf *= N;
    }
  }
  const TC* Fm = static_cast<const TC*>(p.geo_f) + ((((cx * dxn + J) * 2 + 0) * nf) + f) * dxn;
  const TC* Fp = static_cast<const TC*>(p.geo_f) + ((((cx * dxn + J) * 2 + 1) * nf) + f) * dxn;
  TC gm = TC(0), gp = TC(0);
#pragma unroll
  for (int m = 0; m < dxn; ++m) {
    gm += Fm[m] * A[m];
    gp += Fp[m] * A[m];
  }
  TC tp = TC(0), tm = TC(0);
#pragma unroll
  for (int q = 0; q < N; ++q) {
    tp += T.lp[q] * uu[q];
    tm += T.lm[q] * uu[q];
  }
  TC up = tp, um = tm;
  if (!(gp > TC(0))) {           // inflow at +1: the neighbour above's -1 trace
    const TIN* ns = src + ci[2 + 2 * J + 1] * NP + base;
    up = TC(0);
#pragma unroll
    for (int q = 0; q < N; ++q) up += T.lm[q] * cvt<TC>(ns[q * sj]);
  }
  if (gm > TC(0)) {              // inflow at -1: the neighbour below's +1 trace
    const TIN* ns = src + ci[2 + 2 * J] * NP + base;
    um = TC(0);
#pragma unroll
    for (int q = 0; q < N; ++q) um += T.lp[q] * cvt<TC>(ns[q * sj]);
  }
  const TC Fplus = gp * up, Fminus = gm * um;
  TC* r = sr + c * NP + base;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    TC acc = T.Lm[q] * Fminus - T.Lp[q] * Fplus;
#pragma unroll
    for (int s2 = 0; s2 < N; ++s2) acc += T.Dt[q * N + s2] * (g[s2] * uu[s2]);
    r[q * sj] += ij[q] * acc;
  }
}

// The lines of direction J of the block's cells (J compile-time, so that the
// line stride N^J is a constant).
template <int D, int N, typename TC, typename TIN, bool SMEM, bool CURVED, int J>
__device__ __forceinline__ void sweep_dir(const KParams& p, const Tab1D<TC>& T, const TIN* src,
                                          const TC* su, TC* sr, const long long* info,
                                          long long cell0, int nc, int nqx, int nqv) {
  constexpr int NP = Pow<N, D>::v;
  constexpr int NL = NP / N;
  constexpr int sj = Pow<N, J>::v;
  for (int it = threadIdx.x; it < nc * NL; it += blockDim.x) {
    const int c = it / NL;
    const int l = it - c * NL;
    const int base = (l % sj) + (l / sj) * (sj * N);
    const long long cell = cell0 + c;
    const long long* ci = info + c * CellInfo<D>::kLen;
    const long long cx = ci[0], cv = ci[1];
    // the x digits of base (n^dx of them, dx = 1..3) and the v digits
    const int qv = p.dx == 1 ? base / N : (p.dx == 2 ? base / (N * N) : base / (N * N * N));
    const int qx = base - qv * nqx;
    if (CURVED && J < p.dx) {
      if constexpr (CURVED) {
        if (p.dx == 3) {
          if constexpr (J < 3 && D >= 4) curved_line<3, D, N, TC, TIN, SMEM, J>(p, T, src, su, sr, ci, c, cell, base, qx, qv, nqx, nqv);
        } else if (p.dx == 2) {
          if constexpr (J < 2 && D >= 3) curved_line<2, D, N, TC, TIN, SMEM, J>(p, T, src, su, sr, ci, c, cell, base, qx, qv, nqx, nqv);
        } else {
          if constexpr (J < 1) curved_line<1, D, N, TC, TIN, SMEM, J>(p, T, src, su, sr, ci, c, cell, base, qx, qv, nqx, nqv);
        }
      }
      continue;
    }
    // contravariant speed of the line: x directions depend on the v node
    // only, v directions on the x node only (phase-space structure)
    TC cj = J < p.dx ? static_cast<const TC*>(p.cx_tab)[(cv * nqv + qv) * p.dx + J]
                     : static_cast<const TC*>(p.cv_tab)[(cx * nqx + qx) * p.dv + (J - p.dx)];
    if (p.adjoint || p.negate) cj = -cj;
    if (cj == TC(0)) continue;
    const bool pos = cj > TC(0);
    TC uu[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if (SMEM) {
        uu[q] = su[c * NP + base + q * sj];
      } else {
        TC v = cvt<TC>(src[cell * NP + base + q * sj]);
        if (p.adjoint) v *= node_weight<D, N, TC>(T.winv, base + q * sj);
        uu[q] = v;
      }
    }
    // trace of the upwind neighbour's line at the shared face
    const TIN* ns = src + ci[2 + 2 * J + (pos ? 0 : 1)] * NP + base;
    TC t = TC(0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      TC v = cvt<TC>(ns[q * sj]);
      if (p.adjoint) v *= node_weight<D, N, TC>(T.winv, base + q * sj);
      t += (pos ? T.lp[q] : T.lm[q]) * v;
    }
    TC* r = sr + c * NP + base;
    if (pos) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        TC acc = T.Lm[q] * t;
#pragma unroll
        for (int s = 0; s < N; ++s) acc += T.Gp[q * N + s] * uu[s];
        r[q * sj] += cj * acc;
      }
    } else {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        TC acc = -T.Lp[q] * t;
#pragma unroll
        for (int s = 0; s < N; ++s) acc += T.Gn[q * N + s] * uu[s];
        r[q * sj] += cj * acc;
      }
    }
  }
}

// CURVED: the curved x-mesh path for the x directions (a separate
// instantiation, so the affine kernel carries none of its registers or code).
template <int D, int N, typename TC, typename TIN, typename TW, bool SMEM, bool CURVED>
__global__ void __launch_bounds__(512) k_generic(const KParams p) {
  constexpr int NP = Pow<N, D>::v;
  const Tab1D<TC>& T = tab<TC>(p);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_info1[CellInfo<D>::kLen];   // the global-memory variant's one cell
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  int nqx = 1, nqv = 1;
  for (int m = 0; m < p.dx; ++m) nqx *= N;
  for (int m = 0; m < p.dv; ++m) nqv *= N;
  const int cpb = SMEM ? p.cells_per_block : 1;
  int bad = 0;

  for (long long cell0 = static_cast<long long>(blockIdx.x) * cpb; cell0 < p.ncells;
       cell0 += static_cast<long long>(gridDim.x) * cpb) {
    const int nc = static_cast<int>(min(static_cast<long long>(cpb), p.ncells - cell0));
    TC* su = reinterpret_cast<TC*>(smem_raw);
    TC* sr = SMEM ? su + cpb * NP : static_cast<TC*>(p.scratch) + static_cast<long long>(blockIdx.x) * NP;
    long long* info = SMEM ? reinterpret_cast<long long*>(su + 2 * cpb * NP) : s_info1;

    // step 1: gather (and the M^{-1} scaling of the adjoint's input), and the
    // cells' bookkeeping
    for (int i = threadIdx.x; i < nc * NP; i += blockDim.x) {
      if (SMEM) {
        TC v = cvt<TC>(src[cell0 * NP + i]);
        if (p.adjoint) v *= node_weight<D, N, TC>(T.winv, i % NP);
        su[i] = v;
      }
      sr[i] = TC(0);
    }
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const long long cell = cell0 + c;
      long long* ci = info + c * CellInfo<D>::kLen;
      ci[0] = cell % p.ncx;
      ci[1] = cell / p.ncx;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const long long st = p.cstride[j];
        const int nj = p.ncell[j];
        const int cj = static_cast<int>((cell / st) % nj);
        ci[2 + 2 * j] = cj == 0 ? cell + (nj - 1) * st : cell - st;
        ci[3 + 2 * j] = cj == nj - 1 ? cell - (nj - 1) * st : cell + st;
        DG_BOUND(p.err, ci[2 + 2 * j], p.ncells);
        DG_BOUND(p.err, ci[3 + 2 * j], p.ncells);
      }
      DG_BOUND(p.err, ci[0], p.ncx);
      DG_BOUND(p.err, ci[1], p.ncells / p.ncx);
    }
    __syncthreads();

    // steps 2-4, direction by direction
    for (int jj = 0; jj < D; ++jj) {
      switch (p.order[jj]) {
#define DG_SWEEP(JJ)                                                                            \
  case JJ:                                                                                      \
    if constexpr (JJ < D)                                                                       \
      sweep_dir<D, N, TC, TIN, SMEM, CURVED, JJ>(p, T, src, su, sr, info, cell0, nc, nqx, nqv); \
    break;
        DG_SWEEP(0)
        DG_SWEEP(1)
        DG_SWEEP(2)
        DG_SWEEP(3)
        DG_SWEEP(4)
        DG_SWEEP(5)
#undef DG_SWEEP
        default:
          break;
      }
      __syncthreads();
    }

    // step 5: scatter / fused LSRK stage update
    const float bf = static_cast<float>(p.b_dt), af = static_cast<float>(p.a_dt);
    for (int i = threadIdx.x; i < nc * NP; i += blockDim.x) {
      TC K = sr[i];
      if (p.adjoint) K *= node_weight<D, N, TC>(T.w, i % NP);
      if (!isfinite(K)) bad = 1;
      const long long g = cell0 * NP + i;
      if (p.mode == 0) {
        static_cast<TW*>(p.dst)[g] = cvt<TW>(K);
      } else {
        if (p.kref) K += static_cast<TC>(p.kref[g]);    // delta-f form
        const double uo = p.u[g];
        if constexpr (sizeof(TC) == 8) {
          const double un = uo + p.b_dt * K;
          p.u[g] = un;
          static_cast<TW*>(p.dst)[g] = cvt<TW>(p.last_stage ? un : uo + p.a_dt * K);
        } else {
          // FP32 sweeps: one FP64 add for the state, the rest in FP32 / integer
          const double un = uo + f32_to_f64(bf * K);
          p.u[g] = un;
          if constexpr (sizeof(TW) == 4)
            static_cast<TW*>(p.dst)[g] = p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(uo));
          else
            static_cast<TW*>(p.dst)[g] = p.last_stage ? un : uo + p.a_dt * f32_to_f64(K);
        }
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(p.err, 1);
}

constexpr size_t kSmemLimit = 200 * 1024;

// shared memory of one cell: input and residual, plus its bookkeeping
template <int D, int N, typename TC>
constexpr size_t cell_smem() {
  return static_cast<size_t>(Pow<N, D>::v) * sizeof(TC) * 2 + CellInfo<D>::kLen * sizeof(long long);
}
template <int D, int N, typename TC>
constexpr bool fits_smem() {
  return cell_smem<D, N, TC>() <= kSmemLimit;
}

template <int D, int N, typename TC, typename TIN, typename TW>
cudaError_t launch_generic(KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  if constexpr (fits_smem<D, N, TC>()) {
    int cpb = cfg.cells_per_block < 1 ? 1 : cfg.cells_per_block;
    size_t smem = static_cast<size_t>(cpb) * cell_smem<D, N, TC>();
    while (smem > kSmemLimit && cpb > 1) {
      --cpb;
      smem = static_cast<size_t>(cpb) * cell_smem<D, N, TC>();
    }
    p.cells_per_block = cpb;
    auto kern = p.geo_c != nullptr ? k_generic<D, N, TC, TIN, TW, true, true>
                                   : k_generic<D, N, TC, TIN, TW, true, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const long long grid = (p.ncells + cpb - 1) / cpb;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<static_cast<unsigned>(grid), cfg.threads, smem, s>>>(p);
  } else {
    // curved meshes are limited to cells that fit in shared memory (checked
    // when the handle is created)
    if (p.scratch == nullptr || p.geo_c != nullptr) return cudaErrorInvalidValue;
    p.cells_per_block = 1;
    const int blocks = generic_grid_blocks(D, N, p.ncells, 1, cfg.threads);
    k_generic<D, N, TC, TIN, TW, false, false><<<blocks, cfg.threads, 0, s>>>(p);
  }
  return cudaGetLastError();
}

template <int D, int N>
cudaError_t launch_generic_combo(int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  switch (combo) {
    case kDDD: return launch_generic<D, N, double, double, double>(p, cfg, s);
    case kFFF: return launch_generic<D, N, float, float, float>(p, cfg, s);
    case kFDD: return launch_generic<D, N, float, double, double>(p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int D>
cudaError_t launch_generic_dim(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  switch (n) {
    case 2: return launch_generic_combo<D, 2>(combo, p, cfg, s);
    case 3: return launch_generic_combo<D, 3>(combo, p, cfg, s);
    case 4: return launch_generic_combo<D, 4>(combo, p, cfg, s);
    case 5: return launch_generic_combo<D, 5>(combo, p, cfg, s);
    case 6: return launch_generic_combo<D, 6>(combo, p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
