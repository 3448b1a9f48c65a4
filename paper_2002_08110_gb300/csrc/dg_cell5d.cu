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
#include <algorithm>
#include <cstring>

#include "dg_convert.cuh"
#include "dg_internal.h"
#include "dg_tma.cuh"

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
// direction).  r += c (G u + L t).  The upwind side is a template argument,
// so the 1D tables are read as constant operands (no registers, no selects);
// dir5 branches on the thread's sign.
template <bool POS>
__device__ __forceinline__ void dir5s(float (&r)[4][4], const float (&u)[4][4], const float (&nb)[4][4],
                                      float c, const Tab1D<float>& T) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) t = fmaf(POS ? T.lp[q] : T.lm[q], nb[a][q], t);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float acc = (POS ? T.Lm[q] : -T.Lp[q]) * t;
#pragma unroll
      for (int s = 0; s < 4; ++s) acc = fmaf(POS ? T.Gp[q * 4 + s] : T.Gn[q * 4 + s], u[a][s], acc);
      r[a][q] = fmaf(c, acc, r[a][q]);
    }
  }
}
__device__ __forceinline__ void dir5(float (&r)[4][4], const float (&u)[4][4], const float (&nb)[4][4],
                                     float c, const Tab1D<float>& T) {
  if (c > 0.f) dir5s<true>(r, u, nb, c, T);
  else if (c < 0.f) dir5s<false>(r, u, nb, c, T);
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

// ---------------------------------------------------------------------------
// Persistent variant for FP32 input.  One block of 64 threads walks the cells
// blockIdx.x, blockIdx.x + gridDim.x, ... with the phases above.  The cell
// itself and its upwind neighbours along x1, x2, v1 and v2 arrive in shared
// memory by tensor copies (cp.async.bulk.tensor, issued by thread 0,
// completion counted on the buffer's mbarrier) instead of by the threads' own
// loads, so that the copies of the next cell are in flight while the current
// one is computed: the next cell itself at the start of the current cell (two
// own-cell buffers alternate), its four neighbours after phase B of the
// current cell.  The v3 neighbour's values of phase C are loaded by each
// thread (its own upwind side) at the start of phase B, into registers: one
// buffer less lets seven blocks share an SM instead of six (measured 538 ->
// 512 us per stage on the 5D workload).
// A copied cell is the 2D box (16 floats, 64 rows) of the view (16, 64 ncells)
// of the vector with the 64-byte swizzle: element (x, m) sits at
//   16 m + 4 ((x >> 2) ^ ((m >> 1) & 3)) + (x & 3),
// so that the 16-byte row reads of phase A are free of bank conflicts.
// Where the speeds of a copied direction change sign inside a cell, the side
// with more of the cell's nodes is copied and the threads of the other side
// read their neighbour's values from global memory.  Which side is copied is
// decided for the next cell by warp votes over its speeds.
// Waits are bounded: after the limit the block latches DG_ERR_TIMEOUT's flag,
// leaves the walk at the end of the cell, waits (bounded) for the copies it
// has in flight and returns.
constexpr int kT5p = 64;                  // threads per block, one cell at a time
constexpr int kBuf5 = 6;                  // own cell x 2, upwind neighbours along x1, x2, v1, v2
constexpr int kO5 = 0, kN5 = 2;           // buffer indices: own cells, neighbours

struct Cell5 {                            // block-uniform description of a cell
  unsigned cell;
  unsigned co[5];                         // coordinates (x1, x2, v1, v2, v3)
  unsigned nb[4];                         // copied upwind neighbour per direction (x1..v2)
  int side[4];                            // its side: 0 (speed > 0), 1 (< 0), -1 none
};

// the four rows of x block m (u[x2][x1]) from a swizzled cell buffer
__device__ __forceinline__ void rows5(float (&u)[4][4], const float* buf, int m) {
  const int s = (m >> 1) & 3;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float4 v = *reinterpret_cast<const float4*>(buf + 16 * m + 4 * (b ^ s));
    u[b][0] = v.x;
    u[b][1] = v.y;
    u[b][2] = v.z;
    u[b][3] = v.w;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kT5p, 7) k_cell5p(const KParams p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) float sm_raw[];
  // swizzled buffers need 512-byte alignment (one KB of slack is allocated)
  float* const sb = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u) / 4;
  float* const br = sb + kBuf5 * kS5;     // the residual between the phases (off5 layout)
  __shared__ unsigned long long bar[kBuf5];
  __shared__ Cell5 s_c[2];
  __shared__ int s_cnt[2][4][2];          // per warp and copied direction: nodes with speed > 0, < 0
  const int t = threadIdx.x;
  const unsigned ncells = static_cast<unsigned>(p.ncells);
  const float* __restrict__ src = static_cast<const float*>(p.src);
  const Tab1D<float>& T = p.t32;
  const float sgn = p.negate ? -1.f : 1.f;
  const unsigned long long pol = l2_evict_last();
  const unsigned stride = gridDim.x;
  unsigned cell = blockIdx.x;
  if (cell >= ncells) return;
  int ok = 1, bad = 0;
  unsigned ph = 0, pend = 0;              // mbarrier parities; copies not yet waited for (thread 0)

  auto coords = [&](unsigned cl, Cell5& c) {
    unsigned rem = cl;
    c.cell = cl;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const unsigned nj = static_cast<unsigned>(p.ncell[j]);
      c.co[j] = rem % nj;
      rem /= nj;
    }
  };
  auto upwind = [&](const Cell5& c, int j, int side) -> unsigned {
    const unsigned st = static_cast<unsigned>(p.cstride[j]);
    const unsigned nj = static_cast<unsigned>(p.ncell[j]);
    unsigned nb;
    if (side == 0) nb = c.co[j] == 0 ? c.cell + (nj - 1) * st : c.cell - st;
    else nb = c.co[j] == nj - 1 ? c.cell - (nj - 1) * st : c.cell + st;
    DG_BOUND(p.err, nb, ncells);
    return nb;
  };
  // the thread's speeds in a cell: x1, x2 at v node t; v1, v2, v3 at x node t & 15
  auto speeds = [&](const Cell5& c, float (&sp)[5]) {
    const unsigned cx = c.co[0] + static_cast<unsigned>(p.ncell[0]) * c.co[1];
    const unsigned cv = c.co[2] + static_cast<unsigned>(p.ncell[2]) * (c.co[3] + static_cast<unsigned>(p.ncell[3]) * c.co[4]);
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * 64 + t) * 2;
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(cx) * 16 + (t & 15)) * 3;
    sp[0] = sgn * ctx[0];
    sp[1] = sgn * ctx[1];
    sp[2] = sgn * ctv[0];
    sp[3] = sgn * ctv[1];
    sp[4] = sgn * ctv[2];
  };
  auto vote = [&](const float (&sp)[5]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int np = __popc(__ballot_sync(0xffffffffu, sp[j] > 0.f));
      const int nn = __popc(__ballot_sync(0xffffffffu, sp[j] < 0.f));
      if ((t & 31) == 0) {
        s_cnt[t >> 5][j][0] = np;
        s_cnt[t >> 5][j][1] = nn;
      }
    }
  };
  // thread 0: the copied side and neighbour of every direction
  auto sides = [&](Cell5& c) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int np = s_cnt[0][j][0] + s_cnt[1][j][0], nn = s_cnt[0][j][1] + s_cnt[1][j][1];
      const int sd = np == 0 && nn == 0 ? -1 : (np >= nn ? 0 : 1);
      c.side[j] = sd;
      c.nb[j] = sd < 0 ? c.cell : upwind(c, j, sd);
    }
  };
  auto stage = [&](int b, unsigned cl) {  // thread 0
    DG_BOUND(p.err, cl, ncells);
    mbar_expect_tx(&bar[b], kS5 * 4);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(sb + b * kS5)),
        "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(0), "r"(static_cast<int>(cl * 64u)),
        "r"(smem_u32(&bar[b])), "l"(pol)
        : "memory");
    pend |= 1u << b;
  };
  auto wait = [&](int b) {
    if (mbar_wait_bounded(&bar[b], (ph >> b) & 1u)) {
      ph ^= 1u << b;
      pend &= ~(1u << b);
    } else {
      ok = 0;
      atomicOr(p.err, 2);
    }
  };
  auto prefetch_u = [&](unsigned cl) {
    if (MODE == 1 && t < 8) prefetch_l2(p.u + static_cast<size_t>(cl) * kS5 + 128 * t, 1024);
  };

  // ---- the first cell: coordinates, votes, sides, copies
  if (t == 0) {
    for (int b = 0; b < kBuf5; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    coords(cell, s_c[0]);
  }
  __syncthreads();
  float sp[5];
  speeds(s_c[0], sp);
  vote(sp);
  prefetch_u(cell);
  __syncthreads();
  if (t == 0) {
    sides(s_c[0]);
    stage(kO5, cell);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (s_c[0].side[j] >= 0) stage(kN5 + j, s_c[0].nb[j]);
  }
  __syncthreads();

  int cur = 0;
  for (;;) {
    const Cell5& C = s_c[cur];
    const unsigned next = cell + stride;
    const bool has_next = next < ncells;
    float* const bo = sb + (kO5 + cur) * kS5;
    // the next cell: its coordinates, its own values in flight
    if (has_next && t == 0) {
      coords(next, s_c[cur ^ 1]);
      stage(kO5 + (cur ^ 1), next);
    }
    if (has_next) prefetch_u(next);
    float u[4][4], r[4][4], nA[4][4], nB[4][4], nC[4][4];

    // ---- phase A: thread t = v node m, lines along x1 and x2
    {
      const int m = t;
      wait(kO5 + cur);
      rows5(u, bo, m);
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) r[b][a] = 0.f;
      if (C.side[0] >= 0) wait(kN5 + 0);
      if (C.side[1] >= 0) wait(kN5 + 1);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float (&n)[4][4] = j == 0 ? nA : nB;
        if (sp[j] != 0.f) {
          const int sd = sp[j] > 0.f ? 0 : 1;
          if (sd == C.side[j]) {
            rows5(n, sb + (kN5 + j) * kS5, m);
          } else {
            const float4* g = reinterpret_cast<const float4*>(src + static_cast<size_t>(upwind(C, j, sd)) * kS5 + 16 * m);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float4 v = __ldg(g + b);
              n[b][0] = v.x;
              n[b][1] = v.y;
              n[b][2] = v.z;
              n[b][3] = v.w;
            }
          }
        }
      }
      dir5(r, u, nA, sp[0], T);                  // x1: lines b (= x2), points a
      float ut[4][4], nt[4][4], rt[4][4];
      transpose4(ut, u);
      transpose4(nt, nB);
      transpose4(rt, r);
      dir5(rt, ut, nt, sp[1], T);                // x2: lines a (= x1), points b
      transpose4(r, rt);
#pragma unroll
      for (int b = 0; b < 4; ++b)
        *reinterpret_cast<float4*>(br + off5(4 * b, m)) = make_float4(r[b][0], r[b][1], r[b][2], r[b][3]);
    }
    fence_async_smem();
    __syncthreads();                             // x1, x2 buffers free; the phase A residual visible

    // the next cell's speeds (loads in flight during phase B, votes after it)
    float spn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (has_next) speeds(s_c[cur ^ 1], spn);

    // ---- phase B: thread (x node xk, v3 j): the v1-v2 plane, u[v2][v1]
    const int xk = t & 15;
    {
      const int j = t >> 4;
      int xb[4];                                 // swizzled offsets of element (xk, a + 4 b + 16 j)
#pragma unroll
      for (int s = 0; s < 4; ++s) xb[s] = 256 * j + 4 * ((xk >> 2) ^ s) + (xk & 3);
      // the upwind v3 neighbour's values of phase C (this thread, a3 = j), per
      // thread side, requested now and used after phase B
      if (sp[4] != 0.f) {
        const float* g = src + static_cast<size_t>(upwind(C, 4, sp[4] > 0.f ? 0 : 1)) * kS5 + xk;
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) nC[b][jj] = __ldg(g + 16 * (j + 4 * b + 16 * jj));
      }
      if (C.side[2] >= 0) wait(kN5 + 2);
      if (C.side[3] >= 0) wait(kN5 + 3);
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int mm = a + 4 * b + 16 * j;
          u[b][a] = bo[xb[(a >> 1) + 2 * (b & 1)] + 16 * (a + 4 * b)];
          r[b][a] = br[off5(xk, mm)];
        }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        float (&n)[4][4] = jj == 0 ? nA : nB;
        const int d = 2 + jj;
        if (sp[d] != 0.f) {
          const int sd = sp[d] > 0.f ? 0 : 1;
          if (sd == C.side[d]) {
            const float* nb = sb + (kN5 + d) * kS5;
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
              for (int a = 0; a < 4; ++a) n[b][a] = nb[xb[(a >> 1) + 2 * (b & 1)] + 16 * (a + 4 * b)];
          } else {
            const float* g = src + static_cast<size_t>(upwind(C, d, sd)) * kS5 + xk;
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
              for (int a = 0; a < 4; ++a) n[b][a] = __ldg(g + 16 * (a + 4 * b + 16 * j));
          }
        }
      }
      dir5(r, u, nA, sp[2], T);                  // v1: lines b (= v2), points a
      float ut[4][4], nt[4][4], rt[4][4];
      transpose4(ut, u);
      transpose4(nt, nB);
      transpose4(rt, r);
      dir5(rt, ut, nt, sp[3], T);                // v2: lines a (= v1), points b
      transpose4(r, rt);
      if (has_next) vote(spn);
      fence_async_smem();
      __syncthreads();                           // v1, v2 buffers free; residual read; votes in
      if (t == 0 && has_next) {
        Cell5& N = s_c[cur ^ 1];
        sides(N);
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (N.side[d] >= 0) stage(kN5 + d, N.nb[d]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) br[off5(xk, a + 4 * b + 16 * j)] = r[b][a];
    }
    __syncthreads();

    // ---- phase C: thread (x node xk, v1 a3): four v3 lines (one per v2), u[v2][v3]
    const int a3 = t >> 4;
    {
      int xc[2];                                 // swizzled offsets of element (xk, a3 + 4 b), b & 1 = 0, 1
#pragma unroll
      for (int q = 0; q < 2; ++q) xc[q] = 16 * a3 + 4 * ((xk >> 2) ^ ((a3 >> 1) + 2 * q)) + (xk & 3);
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          u[b][jj] = bo[xc[b & 1] + 16 * (4 * b + 16 * jj)];
          r[b][jj] = br[off5(xk, a3 + 4 * b + 16 * jj)];
        }
      dir5(r, u, nC, sp[4], T);                  // v3: lines b (= v2), points jj
    }

    // ---- scatter / fused LSRK stage update (consecutive threads: consecutive x nodes)
    {
      float* __restrict__ dst = static_cast<float*>(p.dst);
      const size_t g0 = static_cast<size_t>(cell) * kS5 + xk;
      float nanacc = 0.f;
      if constexpr (MODE == 0) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const float K = r[b][jj];
            nanacc = fmaf(K, 0.f, nanacc);
            __stcs(dst + g0 + 16 * (a3 + 4 * b + 16 * jj), K);
          }
      } else {
        // all 16 FP64 state values requested at once (one L2 round trip)
        const float bf = static_cast<float>(p.b_dt), af = static_cast<float>(p.a_dt);
        double ua[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) ua[b][jj] = __ldcs(p.u + g0 + 16 * (a3 + 4 * b + 16 * jj));
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const size_t g = g0 + 16 * (a3 + 4 * b + 16 * jj);
            const float K = r[b][jj];
            nanacc = fmaf(K, 0.f, nanacc);
            const double un = ua[b][jj] + f32_to_f64_finite(bf * K);
            __stcs(p.u + g, un);
            __stcs(dst + g, p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(ua[b][jj])));
          }
      }
      bad |= nanacc != 0.f;
    }
    fence_async_smem();
    ok = __syncthreads_and(ok);                  // the own buffer free
    if (!ok || !has_next) break;
#pragma unroll
    for (int j = 0; j < 5; ++j) sp[j] = spn[j];
    cell = next;
    cur ^= 1;
  }
  // copies still in flight (only after a failed wait): wait for them, bounded
  if (t == 0 && pend != 0u) {
    for (int b = 0; b < kBuf5; ++b)
      if ((pend >> b) & 1u) mbar_wait_bounded(&bar[b], (ph >> b) & 1u);
  }
  if (bad) atomicOr(p.err, 1);
}

// 2D view (16 floats, 64 ncells rows) of an FP32 vector, box 16 x 64 (one
// cell), 64-byte swizzle.
cudaError_t encode_cell5_map(CUtensorMap* tm, const void* src, long long ncells) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {16, static_cast<cuuint64_t>(ncells) * 64};
  const cuuint64_t strides[1] = {64};
  const cuuint32_t box[2] = {16, 64};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(src), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t launch5p(KParams& p, cudaStream_t s) {
  // tensor-copy rows are 32-bit signed coordinates; 16-byte aligned vector
  if (p.ncells * 64 >= (1LL << 31) || (reinterpret_cast<uintptr_t>(p.src) & 15u) != 0)
    return cudaErrorNotSupported;
  alignas(64) CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  cudaError_t e;
  if ((e = encode_cell5_map(&tm, p.src, p.ncells)) != cudaSuccess) return e;
  const void* kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell5p<0>)
                                 : reinterpret_cast<const void*>(k_cell5p<1>);
  const size_t smem = 1024 + (static_cast<size_t>(kBuf5) * kS5 + kCell5Smem) * sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT5p, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long grid = std::min<long long>(p.ncells, static_cast<long long>(sms) * per_sm);
  (p.mode == 0 ? k_cell5p<0> : k_cell5p<1>)<<<static_cast<unsigned>(grid), kT5p, smem, s>>>(p, tm);
  return cudaGetLastError();
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
  if (combo == kFFF) {
    const cudaError_t e = launch5p(p, s);
    if (e != cudaErrorNotSupported) return e;
    return launch5<float, float>(p, s);
  }
  if (combo == kFDD) return launch5<double, double>(p, s);
  return cudaErrorNotSupported;
}

}  // namespace dg
