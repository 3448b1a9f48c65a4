// Building blocks of the 4D (dim_x = dim_v = 2) register kernels with FP32
// sweeps, shared by the single-problem kernel (dg_cell4d.cu) and the batched
// one (dg_batch.cu).  A cell's n^4 values are an (n^2) x (n^2) matrix: a
// column is the n^2 x values at one v node (contiguous in memory), a row the
// n^2 v values at one x node; a thread holds a column (phase X) or a row
// (phase V) in registers and does both directions of that phase on it.
#pragma once

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_tma.cuh"

namespace dg {
namespace {

// Asynchronous 4-byte copy global -> shared (completion tracked per thread
// in commit groups); the thread sees the value after cp_async_wait, the
// others after that and a block barrier.
__device__ __forceinline__ void cp_async4(float* smem, const float* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(float2* smem, const float* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(float* smem, const float* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most N of this thread's commit groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int N>
struct Cell4 {
  static constexpr int S = N * N;                 // values of a column or a row
  static constexpr int NP = S * S;                // values of a cell
  static constexpr int PAD = S + 1;               // column stride in shared memory
  static constexpr int THREADS = N == 6 ? 256 : 128;
  static constexpr int CPB = THREADS / S;         // cells per block
  static constexpr int BUF = CPB * S * PAD;       // floats per shared buffer
  // blocks per SM asked of the register allocator (n = 4: 96 registers, 5
  // blocks, measured 6% faster than 120 registers and 4 blocks)
  static constexpr int MINB = N <= 3 ? 8 : (N == 4 ? 5 : 1);
};

// The lines of one direction over a thread's S = n^2 values v[d1 + n d2]:
// ST = 1 runs along d1 (lines indexed by d2), ST = n along d2.  nb holds the
// upwind neighbour's values at the same positions; c is the contravariant
// speed (nonzero).  Positive speed: r += c (Gp u + Lm t), t the neighbour
// below's trace at +1; negative: r += c (Gn u - Lp t), t the neighbour
// above's trace at -1.
// The side is a template argument, so the 1D tables are constant operands (no
// registers, no per-thread selects); dir4 branches on the sign.
template <int N, int ST, bool POS>
__device__ __forceinline__ void dir4s(float (&r)[N * N], const float (&u)[N * N],
                                      const float (&nb)[N * N], float c, const Tab1D<float>& T) {
  const float* G = POS ? T.Gp : T.Gn;
  float L[N], l[N];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    L[q] = POS ? T.Lm[q] : -T.Lp[q];
    l[q] = POS ? T.lp[q] : T.lm[q];
  }
  constexpr int OT = ST == 1 ? N : 1;     // stride between the lines
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int b = a * OT;
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < N; ++q) t = fmaf(l[q], nb[b + q * ST], t);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float acc = L[q] * t;
#pragma unroll
      for (int s = 0; s < N; ++s) acc = fmaf(G[q * N + s], u[b + s * ST], acc);
      r[b + q * ST] = fmaf(c, acc, r[b + q * ST]);
    }
  }
}

template <int N, int ST>
__device__ __forceinline__ void dir4(float (&r)[N * N], const float (&u)[N * N],
                                     const float (&nb)[N * N], float c, const Tab1D<float>& T) {
  if (c > 0.f) dir4s<N, ST, true>(r, u, nb, c, T);
  else dir4s<N, ST, false>(r, u, nb, c, T);
}

// A neighbour's column k (S contiguous values) into registers.
template <int N, typename TIN>
__device__ __forceinline__ void load_col(float (&v)[N * N], const TIN* __restrict__ src,
                                         unsigned cell, int k) {
  constexpr int S = N * N;
  const TIN* col = src + static_cast<size_t>(cell) * (S * S) + static_cast<size_t>(S) * k;
  if constexpr (sizeof(TIN) == 4 && S % 4 == 0) {
    // 16-byte aligned: the vector is, and S * k * 4 and S * S * 4 are multiples of 16
#pragma unroll
    for (int i = 0; i < S / 4; ++i) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(col) + i);
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
  } else if constexpr (sizeof(TIN) == 8 && S % 2 == 0) {
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(col) + i);
      v[2 * i] = f64_to_f32(x.x);
      v[2 * i + 1] = f64_to_f32(x.y);
    }
  } else {
#pragma unroll
    for (int i = 0; i < S; ++i) v[i] = cvt<float>(__ldg(col + i));
  }
}

// A neighbour's row k (S values at stride S; consecutive threads read
// consecutive addresses).
template <int N, typename TIN>
__device__ __forceinline__ void load_row(float (&v)[N * N], const TIN* __restrict__ src,
                                         unsigned cell, int k) {
  constexpr int S = N * N;
  const TIN* row = src + static_cast<size_t>(cell) * (S * S) + k;
#pragma unroll
  for (int m = 0; m < S; ++m) v[m] = cvt<float>(__ldg(row + S * m));
}

// Product of the 1D weights over the two digits of position i of a column
// or a row.
template <int N>
__device__ __forceinline__ float w2(const float* w, int i) {
  return w[i % N] * w[i / N];
}

}  // namespace
}  // namespace dg

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// Pair split for n = 6: two threads per column (phase X) and per row (phase
// V), lanes 2k + h of a warp.  With n^2 = 36 values a column or a row is too
// much for one thread's registers next to its neighbour's; thread h holds the
// 18 values whose second digit is 3h + i (i = 0, 1, 2): v[i][a], a the first
// digit.  Lines along the first digit are thread-local (3 per thread); lines
// along the second digit are split between the two threads, which exchange
// their three values of each line and add their partial traces by shuffles.
constexpr int kP = 6;     // n
constexpr int kPS = 36;   // n^2
constexpr int kPad6 = 36; // column stride in shared memory (unpadded: a cell's global layout)

// the lines along the first digit (3 per thread); POS: the upwind side
template <bool POS>
__device__ __forceinline__ void pdir_local(float (&r)[3][kP], const float (&u)[3][kP],
                                           const float (&nb)[3][kP], float c, const Tab1D<float>& T) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kP; ++q) t = fmaf(POS ? T.lp[q] : T.lm[q], nb[i][q], t);
#pragma unroll
    for (int q = 0; q < kP; ++q) {
      float acc = (POS ? T.Lm[q] : -T.Lp[q]) * t;
#pragma unroll
      for (int s = 0; s < kP; ++s) acc = fmaf(POS ? T.Gp[q * kP + s] : T.Gn[q * kP + s], u[i][s], acc);
      r[i][q] = fmaf(c, acc, r[i][q]);
    }
  }
}

// Coefficients of the split direction for each upwind side and half h, in
// shared memory so that a thread reads its set with six 16-byte loads
// (indexed by its own side and h) instead of computed constant-memory loads:
// entry (side s, h) at tab[24 (2 s + h) ...]: Go[i][j] = G[q][3h + j] (9),
// Gq[i][j] = G[q][3 (1 - h) + j] (9), L[i] (3), the trace weights lo[j] of the
// thread's own points (3), q = 3h + i; s = 0: Gp, Lm, lp; s = 1: Gn, -Lp, lm.
constexpr int kSplitTab = 96;
__device__ __forceinline__ void split_tab_build(float* tab, const Tab1D<float>& T, int tid) {
  if (tid >= kSplitTab) return;
  const int v = tid / 24, e = tid - 24 * (tid / 24);
  const bool pos = (v >> 1) == 0;
  const int h = v & 1, own = 3 * h, par = 3 * (1 - h);
  float x;
  if (e < 9) {
    const int q = own + e / 3, j = e % 3;
    x = pos ? T.Gp[q * kP + own + j] : T.Gn[q * kP + own + j];
  } else if (e < 18) {
    const int q = own + (e - 9) / 3, j = (e - 9) % 3;
    x = pos ? T.Gp[q * kP + par + j] : T.Gn[q * kP + par + j];
  } else if (e < 21) {
    const int q = own + e - 18;
    x = pos ? T.Lm[q] : -T.Lp[q];
  } else {
    const int q = own + e - 21;
    x = pos ? T.lp[q] : T.lm[q];
  }
  tab[tid] = x;
}

// the 6 lines along the second digit, split between the pair (lane ^ 1): the
// thread computes its own points q = 3h + i; every lane of the warp runs this
// (the shuffles need all of them), with zero speed where there is no work
__device__ __forceinline__ void pdir_split(float (&r)[3][kP], const float (&u)[3][kP],
                                           const float (&nb)[3][kP], float c, int h,
                                           const float* tab) {
  float cf[24];
  {
    const float4* t4 = reinterpret_cast<const float4*>(tab + 24 * (2 * (c > 0.f ? 0 : 1) + h));
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 x = t4[i];
      cf[4 * i] = x.x;
      cf[4 * i + 1] = x.y;
      cf[4 * i + 2] = x.z;
      cf[4 * i + 3] = x.w;
    }
  }
  // lines a and a + 1 (a even) hold adjacent values: they go through the
  // packed FP32 FMA together (per lane the same sequence as one line alone)
  const float2 c2 = make_float2(c, c);
#pragma unroll
  for (int a = 0; a < kP; a += 2) {
    float2 v[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      v[j] = make_float2(__shfl_xor_sync(0xffffffffu, u[j][a], 1), __shfl_xor_sync(0xffffffffu, u[j][a + 1], 1));
    // the upwind neighbour's traces of lines a, a + 1: own half, then the partner's
    float t0 = 0.f, t1 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      t0 = fmaf(cf[21 + j], nb[j][a], t0);
      t1 = fmaf(cf[21 + j], nb[j][a + 1], t1);
    }
    t0 += __shfl_xor_sync(0xffffffffu, t0, 1);
    t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
    const float2 t = make_float2(t0, t1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float2 acc = __fmul2_rn(make_float2(cf[18 + i], cf[18 + i]), t);
#pragma unroll
      for (int j = 0; j < 3; ++j)
        acc = __ffma2_rn(make_float2(cf[3 * i + j], cf[3 * i + j]), make_float2(u[j][a], u[j][a + 1]), acc);
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = __ffma2_rn(make_float2(cf[9 + 3 * i + j], cf[9 + 3 * i + j]), v[j], acc);
      const float2 rr = __ffma2_rn(c2, acc, make_float2(r[i][a], r[i][a + 1]));
      r[i][a] = rr.x;
      r[i][a + 1] = rr.y;
    }
  }
}

__device__ __forceinline__ void pdir_local_any(float (&r)[3][kP], const float (&u)[3][kP],
                                               const float (&nb)[3][kP], float c, const Tab1D<float>& T) {
  if (c > 0.f) pdir_local<true>(r, u, nb, c, T);
  else if (c < 0.f) pdir_local<false>(r, u, nb, c, T);
}

// product of the 1D weights of the two digits of position m of a column/row
__device__ __forceinline__ float w2p(const float* w, int m) { return w[m % kP] * w[m / kP]; }

// One block's cells, n = 6, FP32 sweeps: cells [cell0, cell0 + nc), 2 n^2
// threads per cell.  Geometry: ncell / cstride of the 4 cell coordinates
// (x1, x2, v1, v2).  speeds(cell, co, k, c0, c1, e0, e1): the x speeds at v
// node k and the v speeds at x node k (for ADJ already negated).  MODE 0:
// dst = K; MODE 1: u += b dt K (FP64), dst = u_old + a dt K (or u_new at the
// last stage).  ADJ: L^T = M L(-a) M^{-1} (input and neighbours scaled by
// the inverse node weights, output by the weights).  su / sr: shared buffers
// of CPB cells (kPS columns of kPad6 floats); sn: 72 floats per thread of the
// block (the staged neighbour values, FP32 input) followed by the kSplitTab
// floats of the split direction's coefficients (16-byte aligned).  Returns
// the non-finite flag.
template <typename TIN, typename TW, int MODE, bool ADJ, int CPB, int NT, typename Speeds>
__device__ __forceinline__ bool cell4p_block(const TIN* __restrict__ src, TW* __restrict__ dst,
                                             double* __restrict__ uvec, unsigned cell0, int nc,
                                             unsigned ncells, const int (&ncell)[4], const unsigned (&cst)[4],
                                             float b_dt, float a_dt, double a_dt64, bool last_stage,
                                             const Speeds& speeds, const Tab1D<float>& T, float* su,
                                             float* sr, float* sn, int* err) {
  constexpr int S = kPS, NP = S * S, PAD = kPad6;
  const int tid = threadIdx.x;
  const int cslot = tid / (2 * S);
  const int rem = tid - cslot * 2 * S;
  const int k = rem >> 1, h = rem & 1;
  const bool active = cslot < nc;
  const int cs = cslot < CPB ? cslot : CPB - 1;     // smem slot (idle lanes read a valid one)
  const unsigned cell = cell0 + static_cast<unsigned>(active ? cslot : 0);
  unsigned co[4];
  {
    unsigned rm = cell;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      co[j] = rm % static_cast<unsigned>(ncell[j]);
      rm /= static_cast<unsigned>(ncell[j]);
    }
  }
  auto upwind = [&](int j, bool p) -> unsigned {
    const unsigned st = cst[j], nj = static_cast<unsigned>(ncell[j]);
    unsigned nb;
    if (p) nb = co[j] == 0 ? cell + (nj - 1) * st : cell - st;
    else nb = co[j] == nj - 1 ? cell - (nj - 1) * st : cell + st;
    DG_BOUND(err, nb, ncells);
    return nb;
  };
  float c0 = 0.f, c1 = 0.f, e0 = 0.f, e1 = 0.f;
  if (active) speeds(cell, co, k, c0, c1, e0, e1);
  float u[3][kP], r[3][kP], nA[3][kP], nB[3][kP];
  auto zero = [](float (&v)[3][kP]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int a = 0; a < kP; ++a) v[i][a] = 0.f;
  };
  // offsets of the thread's 18 values in a neighbour: its column k (own half,
  // contiguous) for phase X, its row k for phase V; and the adjoint's factor
  // M^{-1} of either (the same product of node weights)
  auto col_off = [&](int i, int a) { return static_cast<size_t>(S) * k + 18 * h + kP * i + a; };
  auto row_off = [&](int i, int a) { return static_cast<size_t>(k) + static_cast<size_t>(S) * (a + kP * (3 * h + i)); };
  auto winv = [&](int i, int a) { return w2p(T.winv, a + kP * (3 * h + i)) * w2p(T.winv, k); };
  constexpr int nt = NT;
  // the split direction's coefficient table, after the staged values
  float* const stab = sn + 72 * NT;
  split_tab_build(stab, T, tid);
  float2* const sn2 = reinterpret_cast<float2*>(sn);   // 8-byte aligned by the callers
  if constexpr (sizeof(TIN) == 4) {
    // FP32 input: every value the block reads arrives by asynchronous copies
    // into shared memory (no registers held while in flight), issued at once
    // in two groups -- the cells and their x neighbours' columns, then the v
    // neighbours' rows -- so that phase X waits only for the first and the
    // second lands during it; the FP64 state of the epilogue is asked of L2
    // ahead.  sn holds the thread's neighbour values: the two columns as 18
    // pairs (8-byte copies of contiguous values) at sn2[p * nt + tid], the two
    // rows at sn[(36 + v) * nt + tid].
    if (MODE == 1 && tid == 0)
      prefetch_l2(uvec + static_cast<size_t>(cell0) * NP, static_cast<unsigned>(nc) * NP * 8u);
    // the block's cells keep their global layout (columns of 36 values):
    // 16-byte copies where the vector is 16-byte aligned (a cell is 5184 bytes)
    const float* gc = src + static_cast<size_t>(cell0) * NP;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
      for (int i = tid; i < nc * (NP / 4); i += nt) cp_async16(su + 4 * i, gc + 4 * i);
    } else {
      for (int i = tid; i < nc * NP; i += nt) cp_async4(su + i, gc + i);
    }
    auto stage_col = [&](int p0, unsigned nbc) {
      const TIN* g = src + static_cast<size_t>(nbc) * NP;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int ap = 0; ap < kP / 2; ++ap) cp_async8(sn2 + (p0 + 3 * i + ap) * nt + tid, g + col_off(i, 2 * ap));
    };
    auto stage_row = [&](int v0, unsigned nbc) {
      const TIN* g = src + static_cast<size_t>(nbc) * NP;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < kP; ++a) cp_async4(sn + (v0 + kP * i + a) * nt + tid, g + row_off(i, a));
    };
    if (active) {
      if (c0 != 0.f) stage_col(0, upwind(0, c0 > 0.f));
      if (c1 != 0.f) stage_col(9, upwind(1, c1 > 0.f));
    }
    cp_async_commit();
    if (active) {
      if (e0 != 0.f) stage_row(36, upwind(2, e0 > 0.f));
      if (e1 != 0.f) stage_row(54, upwind(3, e1 > 0.f));
    }
    cp_async_commit();
    cp_async_wait<1>();
    if (ADJ) {
      // each thread scales the values it copied itself (its copies are complete)
      auto scale = [&](int e) {
        const int r0 = e % NP, t = r0 / S, q = r0 - t * S;
        su[e] *= w2p(T.winv, q) * w2p(T.winv, t);
      };
      if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        for (int i = tid; i < nc * (NP / 4); i += nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) scale(4 * i + e);
      } else {
        for (int i = tid; i < nc * NP; i += nt) scale(i);
      }
    }
  } else {
    // gather the block's cells (padded columns)
    for (int i = tid; i < nc * NP; i += nt) {
      const int cc = i / NP, r0 = i - cc * NP, t = r0 / S, q = r0 - t * S;
      float v = cvt<float>(src[static_cast<size_t>(cell0) * NP + i]);
      if (ADJ) v *= w2p(T.winv, q) * w2p(T.winv, t);
      su[(cc * S + t) * PAD + q] = v;
    }
  }
  // the thread's neighbour values of a direction: from the staging slots
  // v0.. (FP32 input) or loaded now (FP64 input); zero where the speed is zero
  auto nbvals = [&](float (&v)[3][kP], int v0, float c, int j, bool rows) {
    zero(v);
    if (!active || c == 0.f) return;
    if constexpr (sizeof(TIN) == 4) {
      if (!rows) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int ap = 0; ap < kP / 2; ++ap) {
            const float2 x = sn2[(v0 / 2 + 3 * i + ap) * nt + tid];
            v[i][2 * ap] = x.x * (ADJ ? winv(i, 2 * ap) : 1.f);
            v[i][2 * ap + 1] = x.y * (ADJ ? winv(i, 2 * ap + 1) : 1.f);
          }
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int a = 0; a < kP; ++a) v[i][a] = sn[(v0 + kP * i + a) * nt + tid] * (ADJ ? winv(i, a) : 1.f);
      }
    } else {
      const TIN* g = src + static_cast<size_t>(upwind(j, c > 0.f)) * NP;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < kP; ++a)
          v[i][a] = cvt<float>(__ldg(g + (rows ? row_off(i, a) : col_off(i, a)))) * (ADJ ? winv(i, a) : 1.f);
    }
  };
  if constexpr (sizeof(TIN) != 4) {
    nbvals(nA, 0, c0, 0, false);
    nbvals(nB, 18, c1, 1, false);
  }
  __syncthreads();
  if constexpr (sizeof(TIN) == 4) {
    nbvals(nA, 0, c0, 0, false);
    nbvals(nB, 18, c1, 1, false);
  }
  // ---- phase X: column k, directions x1 (local), x2 (split)
  {
    // the thread's 18 values of column k: contiguous, 8-byte aligned
    const float2* col = reinterpret_cast<const float2*>(su + (cs * S + k) * PAD + 18 * h);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const float2 x = col[j];
      u[(2 * j) / kP][(2 * j) % kP] = x.x;
      u[(2 * j) / kP][(2 * j) % kP + 1] = x.y;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int a = 0; a < kP; ++a) r[i][a] = 0.f;
  }
  pdir_local_any(r, u, nA, c0, T);
  pdir_split(r, u, nB, c1, h, stab);
  // lanes without a cell (they ran the split direction for the shuffles
  // only) must not write: their slot is clamped onto a real cell's
  if (active) {
    float2* col = reinterpret_cast<float2*>(sr + (cs * S + k) * PAD + 18 * h);
#pragma unroll
    for (int j = 0; j < 9; ++j)
      col[j] = make_float2(r[(2 * j) / kP][(2 * j) % kP], r[(2 * j) / kP][(2 * j) % kP + 1]);
  }
  if constexpr (sizeof(TIN) == 4) {
    cp_async_wait<0>();
  } else {
    nbvals(nA, 36, e0, 2, true);
    nbvals(nB, 54, e1, 3, true);
  }
  __syncthreads();
  if constexpr (sizeof(TIN) == 4) {
    nbvals(nA, 36, e0, 2, true);
    nbvals(nB, 54, e1, 3, true);
  }
  // ---- phase V: row k, directions v1 (local), v2 (split)
  const size_t g0 = static_cast<size_t>(cell) * NP + k;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < kP; ++a) {
      const int m = a + kP * (3 * h + i);
      u[i][a] = su[(cs * S + m) * PAD + k];
      r[i][a] = sr[(cs * S + m) * PAD + k];
    }
  pdir_local_any(r, u, nA, e0, T);
  pdir_split(r, u, nB, e1, h, stab);
  if (ADJ) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int a = 0; a < kP; ++a) r[i][a] *= w2p(T.w, a + kP * (3 * h + i)) * w2p(T.w, k);
  }
  float nanacc = 0.f;
  if (active) {
    // the FP64 state: all 18 values requested at once (one round trip)
    double ua[3][kP];
    if constexpr (MODE == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < kP; ++a) ua[i][a] = __ldcs(uvec + g0 + static_cast<size_t>(S) * (a + kP * (3 * h + i)));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int a = 0; a < kP; ++a) {
        const size_t g = g0 + static_cast<size_t>(S) * (a + kP * (3 * h + i));
        const float K = r[i][a];
        nanacc = fmaf(K, 0.f, nanacc);
        if constexpr (MODE == 0) {
          __stcs(dst + g, cvt<TW>(K));
        } else {
          const double un = ua[i][a] + f32_to_f64_finite(b_dt * K);
          __stcs(uvec + g, un);
          if constexpr (sizeof(TW) == 4)
            __stcs(dst + g, last_stage ? f64_to_f32(un) : fmaf(a_dt, K, f64_to_f32(ua[i][a])));
          else
            __stcs(dst + g, last_stage ? un : ua[i][a] + a_dt64 * f32_to_f64(K));
        }
      }
    }
  }
  (void)err;
  (void)ncells;
  return nanacc != 0.f;
}

}  // namespace
}  // namespace dg
