// Batched execution of many independent advection problems.
//
// Every member is a constant-velocity problem (Sec. 5.1 setting) of its own
// dimension (dim_x = 2, dim_v = 1 or 2 here: d = 3 or 4), degree and mesh.
// Members are grouped by (d, n); each LSRK(5,4) stage of a group is ONE
// persistent launch of a kernel specialised for that (d, n): blocks take work
// tiles (a member and a run of its cells) from a device queue with an atomic
// counter.  Tiles of one member are consecutive in the queue so that
// neighbouring cells are processed close in time (L2 reuse); load balance
// comes from the dynamic assignment.  One step = 5 x (number of groups)
// launches (+ counter resets), replayed from a CUDA graph.
//
// Kernels: for FP32 stage vectors, the d = 4 groups (dim_x = dim_v = 2) run
// the register-resident 4D cell algorithm (dg_cell4d.cuh: a thread holds a
// column, then a row, of a cell's n^2 x n^2 matrix; a tile is one block's
// cells); every other group runs the shared-memory cell algorithm below
// (tiles of about tile_dofs DoFs).  Block sizes (so cells per block), tile
// size and the order of the directions are chosen by dg_batch_autotune,
// which keeps a record of the configurations it timed.
//
// Per member and stage: K = M^{-1} A(w_in); u += b_s dt K (FP64);
// w_out = u_old + a_s dt K (s < 4) or u_new (s = 4), exactly as the
// single-problem fused stage; stage vectors ping-pong between w0 and w1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_cell4d.cuh"
#include "dg_generic.cuh"

namespace dg {
namespace {

constexpr int kBatchMaxDim = 4;

// Collocated 1D tables per n (index n), FP64 and FP32.
__constant__ Tab1D<double> c_bt64[kMaxN + 1];
__constant__ Tab1D<float> c_bt32[kMaxN + 1];

struct BInst {
  int d, n, npc, ncells;
  int ncell[kBatchMaxDim];
  int cstride[kBatchMaxDim];
  double c64[kBatchMaxDim];   // contravariant speeds (constant field)
  float c32[kBatchMaxDim];
  double dt;
  const void* w[2];           // stage vectors w0, w1
  double* u;
};

struct Tile {
  int inst, cell0, ncells;
};

struct BParams {
  const BInst* inst;
  const Tile* tiles;
  int ntiles;
  int* counter;
  int* err;
  int mode;        // 1: stage (the only mode)
  int stage, parity;
  int nbt_off;     // byte offset of the per-cell neighbour table in shared memory
  double a, b;     // a_s (or b_4 at the last stage), b_s
  int last_stage;
  int ninst;       // number of members (bounds checks)
  int order;       // bit 0 / 1: second x / v direction first (4D register kernel);
                   // bit 2: directions in reverse order (shared-memory kernel)
};

template <typename T>
__device__ __forceinline__ const Tab1D<T>& btab(int n);
template <>
__device__ __forceinline__ const Tab1D<double>& btab<double>(int n) { return c_bt64[n]; }
template <>
__device__ __forceinline__ const Tab1D<float>& btab<float>(int n) { return c_bt32[n]; }

template <typename TC>
__device__ __forceinline__ TC speed(const BInst& I, int j);
template <>
__device__ __forceinline__ double speed<double>(const BInst& I, int j) { return I.c64[j]; }
template <>
__device__ __forceinline__ float speed<float>(const BInst& I, int j) { return I.c32[j]; }

__device__ __forceinline__ int nb_cell(const BInst& I, int cell, int j, int s, int* err) {
  const int st = I.cstride[j], nj = I.ncell[j];
  const int cj = (cell / st) % nj;
  int nb;
  if (s < 0) nb = cj == 0 ? cell + (nj - 1) * st : cell - st;
  else nb = cj == nj - 1 ? cell - (nj - 1) * st : cell + st;
  DG_BOUND(err, nb, I.ncells);
  (void)err;
  return nb;
}

// The lines of direction J (compile-time, so the line stride N^J is a
// constant) of a tile's cells, one line per thread and round.
template <int D, int N, int J, typename TC, typename TW>
__device__ __forceinline__ void bdir(const BInst& I, const TW* src, const TC* su, TC* sr, const int* nbt,
                                     int nc) {
  constexpr int NP = Pow<N, D>::v;
  constexpr int NL = NP / N;
  constexpr int sj = Pow<N, J>::v;
  const Tab1D<TC>& T = btab<TC>(N);
  const TC cj = speed<TC>(I, J);
  if (cj == TC(0)) return;
  const bool pos = cj > TC(0);
  for (int it = threadIdx.x; it < nc * NL; it += blockDim.x) {
    const int c = it / NL;
    const int l = it - c * NL;
    const int base = (l % sj) + (l / sj) * sj * N;
    TC uu[N];
#pragma unroll
    for (int q = 0; q < N; ++q) uu[q] = su[c * NP + base + q * sj];
    const int nb = nbt[c * 2 * kBatchMaxDim + 2 * J + (pos ? 0 : 1)];
    const TW* ns = src + static_cast<size_t>(nb) * NP + base;
    TC t = TC(0);
#pragma unroll
    for (int q = 0; q < N; ++q) t += (pos ? T.lp[q] : T.lm[q]) * ns[q * sj];
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

// One tile of member I: cells [c0, c0 + nc), d = D, n = N, compute type TC,
// stage vectors of type TW (TC == TW here).
template <int D, int N, typename TC, typename TW>
__device__ void process_tile(const BInst& I, const BParams& bp, int c0, int nc, TC* su, TC* sr,
                             int* nbt, int& bad) {
  constexpr int NP = Pow<N, D>::v;
  const TW* src = static_cast<const TW*>(I.w[(bp.stage + bp.parity) & 1]);
  TW* dst = static_cast<TW*>(const_cast<void*>(I.w[(bp.stage + 1 + bp.parity) & 1]));
  const size_t base0 = static_cast<size_t>(c0) * NP;
  for (int i = threadIdx.x; i < nc * NP; i += blockDim.x) {
    su[i] = src[base0 + i];
    sr[i] = TC(0);
  }
  // upwind neighbours of the tile's cells (below, above), once per cell
  for (int c = threadIdx.x; c < nc; c += blockDim.x)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      nbt[c * 2 * kBatchMaxDim + 2 * j] = nb_cell(I, c0 + c, j, -1, bp.err);
      nbt[c * 2 * kBatchMaxDim + 2 * j + 1] = nb_cell(I, c0 + c, j, 1, bp.err);
    }
  __syncthreads();
  // the directions in natural order, or reversed (order bit 2, FP32
  // sweeps); each direction its own instantiation
  if (sizeof(TC) == 4 && (bp.order & 4)) {
    if constexpr (D > 3) {
      bdir<D, N, (D > 3 ? 3 : 0), TC, TW>(I, src, su, sr, nbt, nc);
      __syncthreads();
    }
    bdir<D, N, 2, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
    bdir<D, N, 1, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
    bdir<D, N, 0, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
  } else {
    bdir<D, N, 0, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
    bdir<D, N, 1, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
    bdir<D, N, 2, TC, TW>(I, src, su, sr, nbt, nc);
    __syncthreads();
    if constexpr (D > 3) {
      bdir<D, N, (D > 3 ? 3 : 0), TC, TW>(I, src, su, sr, nbt, nc);
      __syncthreads();
    }
  }
  const double a_dt = bp.a * I.dt, b_dt = bp.b * I.dt;
  for (int i = threadIdx.x; i < nc * NP; i += blockDim.x) {
    const TC K = sr[i];
    bad |= !isfinite(K);
    const size_t g = base0 + i;
    const double uo = I.u[g];
    if constexpr (sizeof(TC) == 8) {
      const double un = uo + b_dt * K;
      I.u[g] = un;
      dst[g] = static_cast<TW>(bp.last_stage ? un : uo + a_dt * K);
    } else {
      // one FP64 add per value; the rest in FP32 / integer arithmetic
      const double un = uo + f32_to_f64(static_cast<float>(b_dt) * K);
      I.u[g] = un;
      dst[g] = bp.last_stage ? f64_to_f32(un) : fmaf(static_cast<float>(a_dt), K, f64_to_f32(uo));
    }
  }
  __syncthreads();
}

template <typename TC, typename TW>
__global__ void __launch_bounds__(512) k_batch(const BParams bp) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ int s_tile;
  int bad = 0;
  if (threadIdx.x == 0) s_tile = atomicAdd(bp.counter, 1);
  for (;;) {
    __syncthreads();
    const int tix = s_tile;
    __syncthreads();
    if (tix >= bp.ntiles) break;
    // the next tile is asked for now; its number is needed only at the end
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(bp.counter, 1);
    const Tile tl = bp.tiles[tix];
#ifdef DG_BOUNDS_CHECK
    // a tile names a member and a run of its cells
    if (tl.inst < 0 || tl.inst >= bp.ninst || tl.cell0 < 0 || tl.ncells < 1 ||
        tl.cell0 + tl.ncells > bp.inst[tl.inst < 0 || tl.inst >= bp.ninst ? 0 : tl.inst].ncells) {
      if (threadIdx.x == 0) {
        atomicOr(bp.err, 4);
        s_tile = next;
      }
      continue;
    }
#endif
    const BInst I = bp.inst[tl.inst];
    TC* su = reinterpret_cast<TC*>(bsm);
    const int cap = tl.ncells * I.npc;
    TC* sr = su + cap;
    int* nbt = reinterpret_cast<int*>(bsm + bp.nbt_off);
    switch (I.d * 8 + I.n) {
      case 3 * 8 + 2: process_tile<3, 2, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 3 * 8 + 3: process_tile<3, 3, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 3 * 8 + 4: process_tile<3, 4, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 3 * 8 + 5: process_tile<3, 5, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 3 * 8 + 6: process_tile<3, 6, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 4 * 8 + 2: process_tile<4, 2, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 4 * 8 + 3: process_tile<4, 3, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 4 * 8 + 4: process_tile<4, 4, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 4 * 8 + 5: process_tile<4, 5, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      case 4 * 8 + 6: process_tile<4, 6, TC, TW>(I, bp, tl.cell0, tl.ncells, su, sr, nbt, bad); break;
      default: break;
    }
    if (threadIdx.x == 0) s_tile = next;
  }
  if (bad) atomicOr(bp.err, 1);
}

// The 4D register kernel over the tiles of one (d = 4, n) group: each tile is
// up to CPB consecutive cells of one member, n^2 threads per cell, the cell
// algorithm of k_cell4d (stage mode, FP32 stage vectors, FP64 state) with the
// member's constant speeds.  bp.order picks which x and which v direction
// goes first.
template <int N, int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch4(const BParams bp) {
  constexpr int S = N * N, NP = S * S, PAD = S + 1, CPB = THREADS / S, BUF = CPB * S * PAD;
  constexpr int NCH = (S + 7) / 8;
  extern __shared__ __align__(16) unsigned char bsm4[];
  float* const su = reinterpret_cast<float*>(bsm4);
  float* const sr = su + BUF;
  float* const sn = sr + BUF;     // the thread's phase V neighbour rows: sn[v * THREADS + tid]
  __shared__ int s_tile;
  const Tab1D<float>& T = c_bt32[N];
  const int c = threadIdx.x / S;
  const int k = threadIdx.x - c * S;
  float nanacc = 0.f;
  if (threadIdx.x == 0) s_tile = atomicAdd(bp.counter, 1);
  for (;;) {
    __syncthreads();
    const int tix = s_tile;
    if (tix >= bp.ntiles) break;
    // the next tile is asked for now; its number is needed only at the end
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(bp.counter, 1);
    const Tile tl = bp.tiles[tix];
#ifdef DG_BOUNDS_CHECK
    // a tile names a member and a run of its cells
    if (tl.inst < 0 || tl.inst >= bp.ninst || tl.cell0 < 0 || tl.ncells < 1 ||
        tl.cell0 + tl.ncells > bp.inst[tl.inst < 0 || tl.inst >= bp.ninst ? 0 : tl.inst].ncells) {
      __syncthreads();      // every thread has read s_tile
      if (threadIdx.x == 0) {
        atomicOr(bp.err, 4);
        s_tile = next;
      }
      continue;
    }
#endif
    const BInst& I = bp.inst[tl.inst];
    const float* __restrict__ src = static_cast<const float*>(I.w[(bp.stage + bp.parity) & 1]);
    float* __restrict__ dst = static_cast<float*>(const_cast<void*>(I.w[(bp.stage + 1 + bp.parity) & 1]));
    const unsigned cell0 = static_cast<unsigned>(tl.cell0);
    const int nc = tl.ncells;
    const bool active = c < nc;
    const unsigned cell = cell0 + static_cast<unsigned>(c);
    unsigned co[4];
    {
      unsigned rem = cell;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned nj = static_cast<unsigned>(I.ncell[j]);
        co[j] = rem % nj;
        rem /= nj;
      }
    }
    auto upwind = [&](int j, bool pos) -> unsigned {
      const unsigned st = static_cast<unsigned>(I.cstride[j]);
      const unsigned nj = static_cast<unsigned>(I.ncell[j]);
      unsigned nb;
      if (pos) nb = co[j] == 0 ? cell + (nj - 1) * st : cell - st;
      else nb = co[j] == nj - 1 ? cell - (nj - 1) * st : cell + st;
      DG_BOUND(bp.err, nb, I.ncells);
      return nb;
    };
    const float c0 = I.c32[0], c1 = I.c32[1], e0 = I.c32[2], e1 = I.c32[3];
    // the tile's FP64 state is asked of L2 now (whole 16-byte units inside it)
    if (threadIdx.x == 0) {
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(I.u + static_cast<size_t>(cell0) * NP);
      const uintptr_t lo = (b0 + 15) & ~static_cast<uintptr_t>(15);
      const uintptr_t hi = (b0 + static_cast<size_t>(nc) * NP * sizeof(double)) & ~static_cast<uintptr_t>(15);
      if (hi > lo) prefetch_l2(reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo));
    }
    // asynchronous copies: the tile's cells (group 1), then the thread's two
    // v neighbour rows (group 2, they land during phase X); the x
    // neighbours' columns come into registers meanwhile
    for (int i = threadIdx.x; i < nc * NP; i += THREADS) {
      const int cc = i / NP, rem = i - cc * NP, t = rem / S, q = rem - t * S;
      cp_async4(su + (cc * S + t) * PAD + q, src + static_cast<size_t>(cell0) * NP + i);
    }
    cp_async_commit();
    if (active) {
      if (e0 != 0.f) {
        const float* row = src + static_cast<size_t>(upwind(2, e0 > 0.f)) * NP + k;
#pragma unroll
        for (int m = 0; m < S; ++m) cp_async4(sn + m * THREADS + threadIdx.x, row + S * m);
      }
      if (e1 != 0.f) {
        const float* row = src + static_cast<size_t>(upwind(3, e1 > 0.f)) * NP + k;
#pragma unroll
        for (int m = 0; m < S; ++m) cp_async4(sn + (S + m) * THREADS + threadIdx.x, row + S * m);
      }
    }
    cp_async_commit();
    float u[S], r[S], nbA[S], nbB[S];
    if (active) {
      if (c0 != 0.f) load_col<N>(nbA, src, upwind(0, c0 > 0.f), k);
      if (c1 != 0.f) load_col<N>(nbB, src, upwind(1, c1 > 0.f), k);
    }
    cp_async_wait<1>();
    __syncthreads();
    // phase X: column k, directions x1, x2 (order by bit 0)
    if (active) {
#pragma unroll
      for (int q = 0; q < S; ++q) {
        u[q] = su[(c * S + k) * PAD + q];
        r[q] = 0.f;
      }
      if (bp.order & 1) {
        if (c1 != 0.f) dir4<N, N>(r, u, nbB, c1, T);
        if (c0 != 0.f) dir4<N, 1>(r, u, nbA, c0, T);
      } else {
        if (c0 != 0.f) dir4<N, 1>(r, u, nbA, c0, T);
        if (c1 != 0.f) dir4<N, N>(r, u, nbB, c1, T);
      }
#pragma unroll
      for (int q = 0; q < S; ++q) sr[(c * S + k) * PAD + q] = r[q];
    }
    cp_async_wait<0>();
    __syncthreads();
    if (active) {
      // phase V: row k, directions v1, v2 (order by bit 1)
      const size_t g0 = static_cast<size_t>(cell) * NP + k;
      double ua[8];
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (m < S) ua[m] = __ldcs(I.u + g0 + static_cast<size_t>(S) * m);
#pragma unroll
      for (int m = 0; m < S; ++m) {
        u[m] = su[(c * S + m) * PAD + k];
        r[m] = sr[(c * S + m) * PAD + k];
        nbA[m] = sn[m * THREADS + threadIdx.x];
        nbB[m] = sn[(S + m) * THREADS + threadIdx.x];
      }
      if (bp.order & 2) {
        if (e1 != 0.f) dir4<N, N>(r, u, nbB, e1, T);
        if (e0 != 0.f) dir4<N, 1>(r, u, nbA, e0, T);
      } else {
        if (e0 != 0.f) dir4<N, 1>(r, u, nbA, e0, T);
        if (e1 != 0.f) dir4<N, N>(r, u, nbB, e1, T);
      }
      // fused LSRK stage update: one FP64 add per value
      const float bf = static_cast<float>(bp.b * I.dt), af = static_cast<float>(bp.a * I.dt);
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        double ub[8];
        if (ch + 1 < NCH) {
#pragma unroll
          for (int m = 0; m < 8; ++m)
            if (8 * (ch + 1) + m < S) ub[m] = __ldcs(I.u + g0 + static_cast<size_t>(S) * (8 * (ch + 1) + m));
        }
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
          const int m = 8 * ch + mm;
          if (m >= S) break;
          const size_t g = g0 + static_cast<size_t>(S) * m;
          const float K = r[m];
          nanacc = fmaf(K, 0.f, nanacc);
          const double un = ua[mm] + f32_to_f64_finite(bf * K);
          __stcs(I.u + g, un);
          __stcs(dst + g, bp.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(ua[mm])));
        }
        if (ch + 1 < NCH) {
#pragma unroll
          for (int m = 0; m < 8; ++m) ua[m] = ub[m];
        }
      }
    }
    __syncthreads();        // su / sr and s_tile are reused by the next tile
    if (threadIdx.x == 0) s_tile = next;
  }
  if (nanacc != 0.f) atomicOr(bp.err, 1);
}

// n = 6: the pair-split register kernel (dg_cell4d.cuh), 3 cells per tile
// and per 224-thread block.
constexpr int kCpb6 = 3, kThreads6 = 224;

__global__ void __launch_bounds__(kThreads6, 2) k_batch4p(const BParams bp) {
  extern __shared__ __align__(16) float bsm4p[];
  float* const su = bsm4p;
  float* const sr = bsm4p + kCpb6 * kPS * kPad6;
  float* const sn = bsm4p + 2 * kCpb6 * kPS * kPad6;   // staged neighbour values, 72 per thread
  __shared__ int s_tile;
  bool bad = false;
  if (threadIdx.x == 0) s_tile = atomicAdd(bp.counter, 1);
  for (;;) {
    __syncthreads();
    const int tix = s_tile;
    if (tix >= bp.ntiles) break;
    // the next tile is asked for now; its number is needed only at the end
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(bp.counter, 1);
    const Tile tl = bp.tiles[tix];
#ifdef DG_BOUNDS_CHECK
    if (tl.inst < 0 || tl.inst >= bp.ninst || tl.cell0 < 0 || tl.ncells < 1 || tl.ncells > kCpb6 ||
        tl.cell0 + tl.ncells > bp.inst[tl.inst < 0 || tl.inst >= bp.ninst ? 0 : tl.inst].ncells) {
      __syncthreads();      // every thread has read s_tile
      if (threadIdx.x == 0) {
        atomicOr(bp.err, 4);
        s_tile = next;
      }
      continue;
    }
#endif
    const BInst& I = bp.inst[tl.inst];
    int ncell[4];
    unsigned cst[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ncell[j] = I.ncell[j];
      cst[j] = static_cast<unsigned>(I.cstride[j]);
    }
    const float s0 = I.c32[0], s1 = I.c32[1], s2 = I.c32[2], s3 = I.c32[3];
    auto speeds = [&](unsigned, const unsigned (&)[4], int, float& c0, float& c1, float& e0,
                      float& e1) {
      c0 = s0;
      c1 = s1;
      e0 = s2;
      e1 = s3;
    };
    const float* src = static_cast<const float*>(I.w[(bp.stage + bp.parity) & 1]);
    float* dst = static_cast<float*>(const_cast<void*>(I.w[(bp.stage + 1 + bp.parity) & 1]));
    bad |= cell4p_block<float, float, 1, false, kCpb6, kThreads6>(
        src, dst, I.u, static_cast<unsigned>(tl.cell0), tl.ncells, static_cast<unsigned>(I.ncells), ncell,
        cst, static_cast<float>(bp.b * I.dt), static_cast<float>(bp.a * I.dt), bp.a * I.dt,
        bp.last_stage != 0, speeds, c_bt32[6], su, sr, sn, bp.err);
    __syncthreads();        // su / sr and s_tile are reused by the next tile
    if (threadIdx.x == 0) s_tile = next;
  }
  if (bad) atomicOr(bp.err, 1);
}

cudaError_t launch_batch4p(const BParams& bp, cudaStream_t s) {
  const size_t smem = (2 * static_cast<size_t>(kCpb6) * kPS * kPad6 + 72 * kThreads6 + kSplitTab) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_batch4p, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch4p, kThreads6, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(bp.ntiles, std::max(1, sms * std::max(1, per_sm)));
  k_batch4p<<<std::max(1, grid), kThreads6, smem, s>>>(bp);
  return cudaGetLastError();
}

// the cell and residual buffers, and the staged v neighbour rows (2 n^2 floats
// per thread)
template <int N>
size_t batch4_smem(int threads) {
  const int S = N * N;
  return (2 * static_cast<size_t>(threads / S) * S * (S + 1) + 2 * static_cast<size_t>(S) * threads) *
         sizeof(float);
}

template <int N, int THREADS>
cudaError_t launch_batch4_t(const BParams& bp, cudaStream_t s) {
  auto kern = k_batch4<N, THREADS>;
  const size_t smem = batch4_smem<N>(THREADS);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(bp.ntiles, std::max(1, sms * std::max(1, per_sm)));
  kern<<<std::max(1, grid), THREADS, smem, s>>>(bp);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_batch4_n(int threads, const BParams& bp, cudaStream_t s) {
  if (threads == 128) return launch_batch4_t<N, 128>(bp, s);
  if (threads == 256) return launch_batch4_t<N, 256>(bp, s);
  if (threads == 512) return launch_batch4_t<N, 512>(bp, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch4(int n, int threads, const BParams& bp, cudaStream_t s) {
  switch (n) {
    case 2: return launch_batch4_n<2>(threads, bp, s);
    case 3: return launch_batch4_n<3>(threads, bp, s);
    case 4: return launch_batch4_n<4>(threads, bp, s);
    case 5: return launch_batch4_n<5>(threads, bp, s);
    case 6: return launch_batch4p(bp, s);     // the pair-split kernel (threads fixed)
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace dg

using namespace dg;

struct dg_batch_ctx {
  int count = 0;
  std::vector<dg_handle> members;
  std::vector<BInst> inst;        // host copy (pointers filled per call)
  std::vector<long long> npc;
  long long n_dofs = 0;
  // launch configuration (dg_batch_launch)
  int tile_dofs = 4096;           // shared-memory kernel: DoFs per tile
  int threads = 256;              // shared-memory kernel: threads per block
  int threads4 = 128;             // 4D register kernel: threads per block (n^2 per cell)
  int order = 0;                  // direction order bits (BParams::order)
  int r4_max_n = 6;               // FP32 4D groups with n <= this run the register kernels
  // members grouped by (d, n); each group's tiles for the two kernels
  struct Group {
    int d = 0, n = 0;
    std::vector<int> members;
    std::vector<Tile> tiles_sm, tiles_r4;   // shared-memory / 4D register tiles
    Tile* tiles_sm_d = nullptr;
    Tile* tiles_r4_d = nullptr;
    size_t smem64 = 0, smem32 = 0;          // shared-memory kernel, bytes
    int nbt_off64 = 0, nbt_off32 = 0;
  };
  std::vector<Group> groups;
  BInst* inst_d = nullptr;
  int* counters_d = nullptr;      // one per stage and group
  int* err_d = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::vector<dg_batch_trial> trials;   // the last autotune's record
  struct Key {
    std::vector<const void*> ptrs;
    std::vector<double> dts;
    int prec = -1, parity = -1;
    bool operator==(const Key& o) const {
      return ptrs == o.ptrs && dts == o.dts && prec == o.prec && parity == o.parity;
    }
  };
  Key key[2];
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
};

namespace {

void free_tiles(dg_batch b) {
  for (auto& g : b->groups) {
    cudaFree(g.tiles_sm_d);
    cudaFree(g.tiles_r4_d);
    g.tiles_sm_d = g.tiles_r4_d = nullptr;
  }
}

void free_batch(dg_batch b) {
  if (!b) return;
  for (int i = 0; i < 2; ++i)
    if (b->gexec[i]) cudaGraphExecDestroy(b->gexec[i]);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  free_tiles(b);
  cudaFree(b->inst_d);
  cudaFree(b->counters_d);
  cudaFree(b->err_d);
  delete b;
}

void drop_graphs(dg_batch b) {
  for (int i = 0; i < 2; ++i)
    if (b->gexec[i]) {
      cudaGraphExecDestroy(b->gexec[i]);
      b->gexec[i] = nullptr;
    }
}

// Does group g run the 4D register kernel at this precision?
bool uses_r4(const dg_batch_ctx* b, const dg_batch_ctx::Group& g, int prec) {
  return prec == DG_PREC_FP32 && g.d == 4 && g.n <= b->r4_max_n;
}

cudaError_t upload(Tile** dst, const std::vector<Tile>& v) {
  cudaFree(*dst);
  *dst = nullptr;
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(Tile));
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice);
  return e;
}

// Tiles of every group: `tile_dofs` DoFs (whole cells, at least one) for the
// shared-memory kernel, one block's cells (threads4 / n^2) for the 4D
// register kernel; member by member.
dg_status build_tiles(dg_batch b) {
  for (auto& g : b->groups) {
    g.tiles_sm.clear();
    g.tiles_r4.clear();
    size_t max_cells_dofs = 0, max_cells = 0;
    const int npc = static_cast<int>(b->npc[g.members[0]]);
    const int per = std::max(1, b->tile_dofs / npc);
    const int per4 = g.n == 6 ? kCpb6 : std::max(1, b->threads4 / (g.n * g.n));
    for (int m : g.members) {
      const int nc = b->inst[m].ncells;
      for (int c = 0; c < nc; c += per) g.tiles_sm.push_back(Tile{m, c, std::min(per, nc - c)});
      if (g.d == 4)
        for (int c = 0; c < nc; c += per4) g.tiles_r4.push_back(Tile{m, c, std::min(per4, nc - c)});
      max_cells_dofs = std::max(max_cells_dofs, static_cast<size_t>(per) * npc);
      max_cells = std::max(max_cells, static_cast<size_t>(per));
    }
    // the tile's values and residuals, then its cells' neighbour table
    g.nbt_off64 = static_cast<int>(max_cells_dofs * 2 * sizeof(double));
    g.nbt_off32 = static_cast<int>(max_cells_dofs * 2 * sizeof(float));
    const size_t nbt_bytes = max_cells * 2 * kBatchMaxDim * sizeof(int);
    g.smem64 = g.nbt_off64 + nbt_bytes;
    g.smem32 = g.nbt_off32 + nbt_bytes;
    if (g.smem64 > 200 * 1024) g.smem64 = 0;  // FP64 not possible at this tile size
    if (g.smem32 > 200 * 1024) return report(DG_ERR_INVALID_ARG, "tile too large for shared memory");
    cudaError_t e = upload(&g.tiles_sm_d, g.tiles_sm);
    if (e == cudaSuccess) e = upload(&g.tiles_r4_d, g.tiles_r4);
    if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
  }
  drop_graphs(b);
  return DG_OK;
}

long long tile_count(const dg_batch_ctx* b, int prec) {
  long long t = 0;
  for (const auto& g : b->groups) t += uses_r4(b, g, prec) ? g.tiles_r4.size() : g.tiles_sm.size();
  return t;
}

template <typename TC, typename TW>
cudaError_t launch_batch(dg_batch b, const BParams& bp, size_t smem, cudaStream_t s) {
  auto kern = k_batch<TC, TW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->threads, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(bp.ntiles, std::max(1, sms * std::max(1, per_sm)));
  kern<<<std::max(1, grid), b->threads, smem, s>>>(bp);
  return cudaGetLastError();
}

dg_status enqueue_step(dg_batch b, int prec, int parity, cudaStream_t s) {
  double A[4], B[5];
  lsrk_coefficients(A, B);
  const int G = static_cast<int>(b->groups.size());
  cudaError_t e = cudaMemsetAsync(b->counters_d, 0, 5 * G * sizeof(int), s);
  if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
  for (int st = 0; st < 5; ++st)
    for (int gi = 0; gi < G; ++gi) {
      const auto& g = b->groups[gi];
      const bool r4 = uses_r4(b, g, prec);
      BParams bp{};
      bp.inst = b->inst_d;
      bp.tiles = r4 ? g.tiles_r4_d : g.tiles_sm_d;
      bp.ntiles = static_cast<int>(r4 ? g.tiles_r4.size() : g.tiles_sm.size());
      bp.counter = b->counters_d + st * G + gi;
      bp.err = b->err_d;
      bp.mode = 1;
      bp.stage = st;
      bp.parity = parity;
      bp.a = st < 4 ? A[st] : B[4];
      bp.b = B[st];
      bp.last_stage = st == 4;
      bp.order = b->order;
      bp.ninst = b->count;
      bp.nbt_off = prec == DG_PREC_FP64 ? g.nbt_off64 : g.nbt_off32;
      if (r4)
        e = launch_batch4(g.n, b->threads4, bp, s);
      else
        e = prec == DG_PREC_FP64 ? launch_batch<double, double>(b, bp, g.smem64, s)
                                 : launch_batch<float, float>(b, bp, g.smem32, s);
      if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
    }
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_batch_create(int count, const dg_handle* handles, dg_batch* out) {
  if (out == nullptr || handles == nullptr) return report(DG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (count < 1) return report(DG_ERR_INVALID_ARG, "count must be >= 1");
  dg_batch b = new (std::nothrow) dg_batch_ctx();
  if (!b) return report(DG_ERR_OOM, "host allocation failed");
  b->count = count;
  for (int m = 0; m < count; ++m) {
    const dg_ctx* h = handles[m];
    if (h == nullptr) {
      free_batch(b);
      return report(DG_ERR_INVALID_ARG, "NULL handle in batch");
    }
    if (h->field_kind != DG_FIELD_CONSTANT || h->d < 3 || h->d > 4 || h->ncells > (1LL << 30) ||
        h->basis != DG_BASIS_GL || h->curved) {
      free_batch(b);
      return report(DG_ERR_UNSUPPORTED,
                    "batched members must be constant-velocity problems with d = 3 or 4 "
                    "in the Gauss-Legendre basis");
    }
    BInst I{};
    I.d = h->d;
    I.n = h->n;
    I.npc = h->npc;
    I.ncells = static_cast<int>(h->ncells);
    for (int j = 0; j < h->d; ++j) {
      I.ncell[j] = h->ncell[j];
      I.cstride[j] = static_cast<int>(h->cstride[j]);
      // constant field: every node carries the same speed
      I.c64[j] = j < h->dx ? h->cx_host[j] : h->cv_host[j - h->dx];
      I.c32[j] = static_cast<float>(I.c64[j]);
    }
    b->members.push_back(handles[m]);
    b->inst.push_back(I);
    b->npc.push_back(h->npc);
    b->n_dofs += h->n_dofs;
    // group by (d, n)
    int gi = 0;
    while (gi < static_cast<int>(b->groups.size()) &&
           !(b->groups[gi].d == h->d && b->groups[gi].n == h->n))
      ++gi;
    if (gi == static_cast<int>(b->groups.size())) {
      b->groups.emplace_back();
      b->groups.back().d = h->d;
      b->groups.back().n = h->n;
    }
    b->groups[gi].members.push_back(m);
  }
  // tables for every n
  Tab1D<double> t64[kMaxN + 1];
  Tab1D<float> t32[kMaxN + 1];
  std::memset(t64, 0, sizeof(t64));
  std::memset(t32, 0, sizeof(t32));
  for (int n = 2; n <= kMaxN; ++n) {
    HostTables ht;
    build_tables(n, DG_BASIS_GL, &ht);
    t64[n] = ht.t64;
    t32[n] = ht.t32;
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_bt64, t64, sizeof(t64))) != cudaSuccess ||
      (e = cudaMemcpyToSymbol(c_bt32, t32, sizeof(t32))) != cudaSuccess ||
      (e = cudaMalloc(&b->inst_d, sizeof(BInst) * count)) != cudaSuccess ||
      (e = cudaMalloc(&b->counters_d, 5 * b->groups.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->err_d, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(b->err_d, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    free_batch(b);
    return report(DG_ERR_CUDA, cudaGetErrorString(e));
  }
  dg_status st = build_tiles(b);
  if (st != DG_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return DG_OK;
}

dg_status dg_batch_destroy(dg_batch b) {
  free_batch(b);
  return DG_OK;
}

dg_status dg_batch_info(dg_batch b, long long* tiles, long long* n_dofs) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  if (tiles) *tiles = tile_count(b, DG_PREC_FP32);
  if (n_dofs) *n_dofs = b->n_dofs;
  return DG_OK;
}

dg_status dg_batch_rk_step(dg_batch b, double* const* u, void* const* w0, void* const* w1,
                           const double* dt, int nsteps, int prec, void* stream) {
  if (b == nullptr || u == nullptr || w0 == nullptr || w1 == nullptr || dt == nullptr)
    return report(DG_ERR_INVALID_ARG, "NULL argument");
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32)
    return report(DG_ERR_INVALID_ARG, "batched precision must be DG_PREC_FP64 or DG_PREC_FP32");
  if (nsteps < 0) return report(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  for (const auto& g : b->groups)
    if (prec == DG_PREC_FP64 && g.smem64 == 0)
      return report(DG_ERR_UNSUPPORTED, "FP64 batches need a smaller tile size");
  for (int m = 0; m < b->count; ++m) {
    if (!u[m] || !w0[m] || !w1[m] || !std::isfinite(dt[m]))
      return report(DG_ERR_INVALID_ARG, "NULL vector or non-finite dt in batch member");
    if (reinterpret_cast<uintptr_t>(u[m]) % 16 || reinterpret_cast<uintptr_t>(w0[m]) % 16 ||
        reinterpret_cast<uintptr_t>(w1[m]) % 16)
      return report(DG_ERR_INVALID_ARG, "batch vectors must be 16-byte aligned");
  }
  if (nsteps == 0) return DG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // member descriptors with this call's vectors
  for (int m = 0; m < b->count; ++m) {
    b->inst[m].u = u[m];
    b->inst[m].w[0] = w0[m];
    b->inst[m].w[1] = w1[m];
    b->inst[m].dt = dt[m];
  }
  cudaError_t e = cudaMemcpyAsync(b->inst_d, b->inst.data(), sizeof(BInst) * b->count,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
  // w0 = u for every member (one streaming pass per member)
  for (int m = 0; m < b->count; ++m) {
    const long long n = static_cast<long long>(b->inst[m].ncells) * b->inst[m].npc;
    if ((e = launch_convert(u[m], w0[m], prec == DG_PREC_FP32 ? 1 : 0, n, s)) != cudaSuccess)
      return report(DG_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess)
    return report(DG_ERR_CUDA, cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone) {
    for (int i = 0; i < nsteps; ++i) {
      dg_status st = enqueue_step(b, prec, i % 2, s);
      if (st != DG_OK) return st;
    }
    return DG_OK;
  }
  for (int parity = 0; parity < 2 && parity < nsteps; ++parity) {
    dg_batch_ctx::Key key;
    for (int m = 0; m < b->count; ++m) {
      key.ptrs.push_back(u[m]);
      key.ptrs.push_back(w0[m]);
      key.ptrs.push_back(w1[m]);
      key.dts.push_back(dt[m]);
    }
    key.prec = prec;
    key.parity = parity;
    if (b->gexec[parity] && b->key[parity] == key) continue;
    if (b->gexec[parity]) {
      cudaGraphExecDestroy(b->gexec[parity]);
      b->gexec[parity] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return report(DG_ERR_CUDA, cudaGetErrorString(e));
    dg_status st = enqueue_step(b, prec, parity, b->capture_stream);
    e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->gexec[parity] = nullptr;
      return report(DG_ERR_CUDA, cudaGetErrorString(e));
    }
    b->key[parity] = key;
  }
  for (int i = 0; i < nsteps; ++i)
    if ((e = cudaGraphLaunch(b->gexec[i % 2], s)) != cudaSuccess)
      return report(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

dg_status dg_batch_check(dg_batch b, void* stream) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flag = 0;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
      (e = cudaMemcpy(&flag, b->err_d, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemset(b->err_d, 0, sizeof(int))) != cudaSuccess)
    return report(DG_ERR_CUDA, cudaGetErrorString(e));
  if (flag & 4) return report(DG_ERR_BOUNDS, "a batched kernel computed an index out of its range");
  if (flag & 1) return report(DG_ERR_NONFINITE, "a batched kernel produced a non-finite value");
  return DG_OK;
}

dg_status dg_batch_set_launch_ex(dg_batch b, const dg_batch_launch* cfg) {
  if (b == nullptr || cfg == nullptr) return report(DG_ERR_INVALID_ARG, "NULL argument");
  if (cfg->tile_dofs < 64 || cfg->tile_dofs > (1 << 16) || cfg->threads < 32 || cfg->threads > 512 ||
      cfg->threads % 32)
    return report(DG_ERR_INVALID_ARG, "tile_dofs in [64, 65536], threads a multiple of 32 <= 512");
  if (cfg->threads4 != 128 && cfg->threads4 != 256 && cfg->threads4 != 512)
    return report(DG_ERR_INVALID_ARG, "threads4 must be 128, 256 or 512");
  if (cfg->order < 0 || cfg->order > 7) return report(DG_ERR_INVALID_ARG, "order bits in [0, 7]");
  if (cfg->r4_max_n < 1 || cfg->r4_max_n > kMaxN)
    return report(DG_ERR_INVALID_ARG, "r4_max_n in [1, 6]");
  for (const auto& g : b->groups)
    if (g.d == 4 && g.n <= cfg->r4_max_n && g.n < 6 &&
        (cfg->threads4 < g.n * g.n || (cfg->threads4 == 512 && g.n > 4)))
      return report(DG_ERR_INVALID_ARG,
                    "threads4 too small (or 512 with n > 4) for a 4D group of the register kernel");
  const dg_batch_launch old{b->tile_dofs, b->threads, b->threads4, b->order, b->r4_max_n};
  auto set = [b](const dg_batch_launch& c) {
    b->tile_dofs = c.tile_dofs;
    b->threads = c.threads;
    b->threads4 = c.threads4;
    b->order = c.order;
    b->r4_max_n = c.r4_max_n;
  };
  set(*cfg);
  dg_status st = build_tiles(b);
  if (st != DG_OK) {
    set(old);
    build_tiles(b);
  }
  return st;
}

dg_status dg_batch_get_launch(dg_batch b, dg_batch_launch* cfg) {
  if (b == nullptr || cfg == nullptr) return report(DG_ERR_INVALID_ARG, "NULL argument");
  *cfg = dg_batch_launch{b->tile_dofs, b->threads, b->threads4, b->order, b->r4_max_n};
  return DG_OK;
}

dg_status dg_batch_set_launch(dg_batch b, int tile_dofs, int threads) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  const dg_batch_launch c{tile_dofs, threads, b->threads4, b->order, b->r4_max_n};
  return dg_batch_set_launch_ex(b, &c);
}

dg_status dg_batch_autotune(dg_batch b, double* const* u, void* const* w0, void* const* w1,
                            const double* dt, int prec, void* stream, double* best_ms) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // candidates: the shared-memory kernel's tile size and block size, the 4D
  // register kernel's block size (cells per block = threads4 / n^2) and the
  // order of the directions (both kernels); what does not apply to any group
  // of this batch is not varied
  bool any4 = false, anysm = false;
  for (const auto& g : b->groups) {
    if (prec == DG_PREC_FP32 && g.d == 4) any4 = true;
    if (!(prec == DG_PREC_FP32 && g.d == 4 && g.n <= 4)) anysm = true;
  }
  b->trials.clear();
  double best = 1e300;
  dg_batch_launch bcfg{b->tile_dofs, b->threads, b->threads4, b->order, b->r4_max_n};
  const dg_batch_launch start = bcfg;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time two steps per candidate (after one untimed step that captures its
  // graphs) on the caller's buffers: their contents are advanced, as the
  // header states
  auto timed = [&](const dg_batch_launch& c, int steps) -> double {
    if (dg_batch_set_launch_ex(b, &c) != DG_OK) return -1.0;
    if (dg_batch_rk_step(b, u, w0, w1, dt, 1, prec, stream) != DG_OK) return -1.0;  // warm-up / capture
    cudaEventRecord(e0, s);
    if (dg_batch_rk_step(b, u, w0, w1, dt, steps, prec, stream) != DG_OK) return -1.0;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return static_cast<double>(ms) / steps;
  };
  auto trial = [&](const dg_batch_launch& c) {
    const double ms = timed(c, 2);
    if (ms < 0.0) return;
    b->trials.push_back(dg_batch_trial{c.tile_dofs, c.threads, c.threads4, c.order, c.r4_max_n, ms});
    if (ms < best) {
      best = ms;
      bcfg = c;
    }
  };
  // The groups are separate launches whose times add up, so the parameters
  // are tuned one after the other (coordinate descent):
  // 1. which FP32 4D groups run the register kernel (n <= r4_max_n), then its
  //    block size (cells per block) and which x and which v direction goes first;
  if (any4) {
    const dg_batch_launch base = bcfg;
    for (int rn : {1, 3, 4, 5, 6}) trial(dg_batch_launch{base.tile_dofs, base.threads, 128, base.order, rn});
    const dg_batch_launch b1 = bcfg;
    if (b1.r4_max_n > 1)
      for (int t4 : {128, 256, 512})
        for (int o = 0; o < 4; ++o)
          trial(dg_batch_launch{b1.tile_dofs, b1.threads, t4, (b1.order & 4) | o, b1.r4_max_n});
  }
  // 2. the shared-memory kernel: tile size x block size, then the direction order
  if (anysm || bcfg.r4_max_n < 6) {
    const dg_batch_launch base = bcfg;
    for (int tdofs : {1024, 2048, 4096, 8192})
      for (int th : {128, 256, 512})
        trial(dg_batch_launch{tdofs, th, base.threads4, base.order, base.r4_max_n});
    const dg_batch_launch b2 = bcfg;
    trial(dg_batch_launch{b2.tile_dofs, b2.threads, b2.threads4, b2.order ^ 4, b2.r4_max_n});
  }
  if (b->trials.empty()) trial(bcfg);
  // the minimum over many two-step trials favours a lucky one: the three
  // fastest distinct configurations and the starting one are timed again
  // over four steps, and the fastest of those is kept (these timings are
  // recorded as trials too)
  {
    std::vector<dg_batch_trial> order(b->trials);
    std::stable_sort(order.begin(), order.end(),
                     [](const dg_batch_trial& x, const dg_batch_trial& y) { return x.ms < y.ms; });
    auto same = [](const dg_batch_launch& x, const dg_batch_launch& y) {
      return x.tile_dofs == y.tile_dofs && x.threads == y.threads && x.threads4 == y.threads4 &&
             x.order == y.order && x.r4_max_n == y.r4_max_n;
    };
    std::vector<dg_batch_launch> finals{start};
    for (const auto& t : order) {
      if (finals.size() >= 4) break;
      const dg_batch_launch c{t.tile_dofs, t.threads, t.threads4, t.order, t.r4_max_n};
      bool dup = false;
      for (const auto& f : finals) dup = dup || same(f, c);
      if (!dup) finals.push_back(c);
    }
    double fbest = 1e300;
    for (const auto& c : finals) {
      const double ms = timed(c, 4);
      if (ms < 0.0) continue;
      b->trials.push_back(dg_batch_trial{c.tile_dofs, c.threads, c.threads4, c.order, c.r4_max_n, ms});
      if (ms < fbest) {
        fbest = ms;
        bcfg = c;
      }
    }
    if (fbest < 1e300) best = fbest;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dg_status st = dg_batch_set_launch_ex(b, &bcfg);
  if (best_ms) *best_ms = best;
  return st;
}

dg_status dg_batch_autotune_record(dg_batch b, dg_batch_trial* trials, int max_trials, int* count) {
  if (b == nullptr || count == nullptr) return report(DG_ERR_INVALID_ARG, "NULL argument");
  *count = static_cast<int>(b->trials.size());
  if (trials)
    for (int i = 0; i < std::min(max_trials, *count); ++i) trials[i] = b->trials[i];
  return DG_OK;
}

}  // extern "C"
