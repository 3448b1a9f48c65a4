// Specialised element-centric cell kernel for d = 6 (3 x + 3 v), n = 4 (k = 3),
// FP32 sweeps and fluxes.
//
// A cell has 4096 values, q = q_x + 64 q_v with q_x = (q1,q2,q3), q_v = (q4,q5,q6)
// (x_1 fastest).  Two variants: 64 threads per cell (described here) and 128
// threads per cell (the "pair variant" below, the default).  In the first, one
// block of 64 threads processes one cell at a time, in two
// phases that follow Algorithm 2's split of the cell work into the x-space
// part and the v-space part:
//   phase X: thread t owns the v node q_v = t and holds the 4x4x4 x-block of
//            that node in registers, so every line along x1, x2, x3 is
//            thread-local; the contravariant speeds c_1..c_3 depend on q_v
//            only (a_x = v), so they are thread constants;
//   phase V: thread t owns the x node q_x = t and holds the 4x4x4 v-block,
//            lines along v1, v2, v3 thread-local; c_4..c_6 = 2 E(x) / h_v
//            depend on q_x only.
// Per direction and line: du_q += c (sum_p G[q][p] u_p + L_nb[q] t_nb) with the
// collocated 1D operator (see Tab1D); t_nb is the upwind neighbour's trace on
// the shared face, computed from the neighbour's line (periodic wrap).  The
// two phases read different views of the padded shared buffers: rows of a
// block in phase X, columns across blocks in phase V.
// The host uses this kernel only when every cell has one upwind side per
// direction (no speed changes sign inside a cell).
//
// Data movement: every cell the block needs -- the cell itself and its six
// upwind neighbours -- is brought into shared memory by the TMA engine
// (cp.async.bulk, one 256-byte block per thread, completion counted on an
// mbarrier), into buffers whose 64-float blocks are padded to 68 floats so
// that the 16-byte row reads of phase X and the 4-byte column reads of phase V
// are free of bank conflicts.  Three buffers rotate (so that four blocks fit
// on an SM): the current cell and two landing buffers; the next cell lands in
// the cell buffer once phase V has its values in registers, and the phase X
// result passes to phase V through a landing buffer.  Every copy is issued as
// soon as its buffer is free, so the next cell and the next neighbours are in
// flight while the current direction is computed.
//
// Waits on mbarriers are bounded: after the poll limit the block latches an
// error flag (reported as DG_ERR_TIMEOUT), waits (bounded) for its copies in
// flight and returns.
//
// Modes: operator application (dst = K) or fused LSRK stage
// (u += b dt K in FP64; w_out = u + a dt K).  Adjoint: L^T = M L(-a) M^{-1}.
// FP64 input (DG_PREC_MIXED) is converted while the threads copy it into
// shared memory themselves.
#include <cstring>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "dg_convert.cuh"
#include "dg_generic.cuh"
#include "dg_tma.cuh"

namespace dg {
namespace {

constexpr int kPad = 68;              // padded floats per 64-value block
constexpr int kCellSmem = 64 * kPad;  // floats per cell buffer
constexpr int kNumBuf = 3;

__device__ __forceinline__ float4 ld4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  return make_float4(f64_to_f32(a.x), f64_to_f32(a.y), f64_to_f32(b.x), f64_to_f32(b.y));
}

// Element index inside a 4x4x4 block of point p on line (l1, l2) along local
// direction J.
template <int J>
__device__ __forceinline__ constexpr int eidx(int l1, int l2, int p) {
  return J == 0 ? p + 4 * l1 + 16 * l2 : (J == 1 ? l1 + 4 * p + 16 * l2 : l1 + 4 * l2 + 16 * p);
}

__device__ __forceinline__ float comp(const float4& v, int a) {
  return a == 0 ? v.x : (a == 1 ? v.y : (a == 2 ? v.z : v.w));
}

// Product of three 1D weights over the digits of a block element.
__device__ __forceinline__ float wprod(const float* w, int e) {
  return w[e & 3] * w[(e >> 2) & 3] * w[e >> 4];
}

// Upwind neighbour of `cell` along direction j (s = -1 below, +1 above) with
// periodic wrap, in 32-bit arithmetic (cell counts are below 2^31).
__device__ __forceinline__ unsigned nb32(const KParams& p, unsigned cell, int j, int s) {
  const unsigned st = static_cast<unsigned>(p.cstride[j]);
  const unsigned nj = static_cast<unsigned>(p.ncell[j]);
  const unsigned cj = (cell / st) % nj;
  if (s < 0) return cj == 0 ? cell + (nj - 1) * st : cell - st;
  return cj == nj - 1 ? cell - (nj - 1) * st : cell + st;
}

// The thread's block inside a padded buffer: row view (phase X: block t,
// element e at +e) or column view (phase V: element t of block e, at e*kPad).
template <bool ROWS>
__device__ __forceinline__ const float* view(const float* buf, int t) {
  return ROWS ? buf + t * kPad : buf + t;
}
template <bool ROWS>
__device__ __forceinline__ float4 row4(const float* v, int i) {
  if constexpr (ROWS) {
    return *reinterpret_cast<const float4*>(v + 4 * i);
  } else {
    return make_float4(v[(4 * i) * kPad], v[(4 * i + 1) * kPad], v[(4 * i + 2) * kPad],
                       v[(4 * i + 3) * kPad]);
  }
}
template <bool ROWS>
__device__ __forceinline__ void load_block(float (&x)[64], const float* v) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float4 a = row4<ROWS>(v, i);
    x[4 * i] = a.x;
    x[4 * i + 1] = a.y;
    x[4 * i + 2] = a.z;
    x[4 * i + 3] = a.w;
  }
}

// The collocated 1D tables of n = 4 for both upwind sides (index 0: c > 0,
// index 1: c < 0), in constant memory so that a block-uniform side selects
// them with one broadcast load: G = Gp / Gn, Ln = Lm / -Lp, lw = lp / lm.
__constant__ float c_G[4][16];
__constant__ float c_Ln[4][4];
__constant__ float c_lw[4][4];

// Traces, on the shared face, of the upwind neighbour's 16 lines along local
// direction J, read from a landing buffer (row or column view).  With the
// adjoint the neighbour values are scaled by M^{-1}: the element factor here,
// the thread factor by the caller (tscale of lines_dir).
template <int J, bool ROWS, bool ADJ>
__device__ __forceinline__ void nb_traces(float (&tr)[16], const float* nbv, float c, int tb,
                                          const Tab1D<float>& T) {
  const int side = tb + (signbit(c) ? 1 : 0);
  float lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) lw[i] = c_lw[side][i];
#pragma unroll
  for (int i = 0; i < 16; ++i) tr[i] = 0.f;
#pragma unroll
  for (int cc = 0; cc < 4; ++cc)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4 v = row4<ROWS>(nbv, b + 4 * cc);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int l1 = J == 0 ? b : a;
        const int l2 = J == 2 ? b : cc;
        const int pp = J == 0 ? a : (J == 1 ? b : cc);
        float x = comp(v, a);
        if (ADJ) x *= wprod(T.winv, a + 4 * b + 16 * cc);
        tr[l1 + 4 * l2] = fmaf(lw[pp], x, tr[l1 + 4 * l2]);
      }
    }
}

// Traces of the thread's own 16 lines along J on the outflow face: for the
// cell downstream they are exactly the inflow traces of its upwind neighbour.
template <int J>
__device__ __forceinline__ void own_traces(float (&tr)[16], const float (&u)[64], float c, int tb) {
  const int side = tb + (signbit(c) ? 1 : 0);
  float lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) lw[i] = c_lw[side][i];
#pragma unroll
  for (int l2 = 0; l2 < 4; ++l2)
#pragma unroll
    for (int l1 = 0; l1 < 4; ++l1) {
      float s = 0.f;
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) s = fmaf(lw[pp], u[eidx<J>(l1, l2, pp)], s);
      tr[l1 + 4 * l2] = s;
    }
}

// The 16 line contractions of direction J: r += c (G u + L_nb t_nb).  The
// upwind side is chosen at run time; the 1D matrices of that side (scaled by
// c) come from constant memory into registers, so one body serves both signs.
template <int J>
__device__ __forceinline__ void lines_dir(float (&r)[64], const float (&u)[64],
                                          const float (&tr)[16], float c, int tb, float tscale) {
  const int side = tb + (signbit(c) ? 1 : 0);
  float Ln[4], G[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) Ln[i] = c * c_Ln[side][i];
#pragma unroll
  for (int i = 0; i < 16; ++i) G[i] = c * c_G[side][i];
#pragma unroll
  for (int l2 = 0; l2 < 4; ++l2)
#pragma unroll
    for (int l1 = 0; l1 < 4; ++l1) {
      const float t = tscale * tr[l1 + 4 * l2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float acc = fmaf(Ln[q], t, r[eidx<J>(l1, l2, q)]);
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) acc = fmaf(G[q * 4 + pp], u[eidx<J>(l1, l2, pp)], acc);
        r[eidx<J>(l1, l2, q)] = acc;
      }
    }
}

template <int J, bool ROWS, bool ADJ>
__device__ __forceinline__ void direction(float (&r)[64], const float (&u)[64], const float* nbv,
                                          float c, int tb, float wthread, const Tab1D<float>& T) {
  float tr[16];
  nb_traces<J, ROWS, ADJ>(tr, nbv, c, tb, T);
  lines_dir<J>(r, u, tr, c, tb, ADJ ? wthread : 1.f);
}

struct Pipe {
  unsigned long long bar[kNumBuf];
  int failed;
};

// Moves cells into the padded buffers and waits for them.  FP32 input: TMA
// bulk copies (one padded 256-byte block per thread, counted on the buffer's
// mbarrier).  FP64 input: the threads load, convert and store their own block
// and the wait is a block barrier.
template <typename TIN>
struct Mover {
  float* sm;
  Pipe* pp;
  unsigned phase = 0;  // parity bit per buffer
  unsigned long long pol = l2_evict_last();

  __device__ __forceinline__ void issue(int b, const TIN* cellp, int t) {
    float* d = sm + b * kCellSmem + t * kPad;
    if constexpr (sizeof(TIN) == 4) {
      if (t == 0) mbar_expect_tx(&pp->bar[b], 4096 * 4);
      bulk_g2s(d, cellp + t * 64, 256, &pp->bar[b], pol);
    } else {
      const TIN* g = cellp + t * 64;
#pragma unroll
      for (int i = 0; i < 16; ++i) *reinterpret_cast<float4*>(d + 4 * i) = ld4(g + 4 * i);
    }
  }
  // returns false if the wait gave up
  __device__ __forceinline__ bool wait(int b, int* err) {
    if constexpr (sizeof(TIN) == 4) {
      const unsigned par = (phase >> b) & 1u;
      phase ^= 1u << b;
      if (mbar_try_wait(&pp->bar[b], par)) return true;
      const long long t0 = clock64();
      while (clock64() - t0 < kWaitCycles)
        if (mbar_try_wait(&pp->bar[b], par)) return true;
      atomicOr(err, 2);
      return false;
    } else {
      __syncthreads();
      return true;
    }
  }
};

// First cell (v3 = 0) of work item ``item``.  Items cover the cells of the
// v3 = 0 slab in tiles of 2 cells per direction (1 where the cell count is
// odd), tiles in lexicographic order, so that the pencils in flight at one
// time are close in all five other directions and more of their upwind
// neighbours are still in L2 when read.
__device__ __forceinline__ unsigned pencil_base(const KParams& p, unsigned item) {
  unsigned tsz = 1;
#pragma unroll
  for (int j = 0; j < 5; ++j) tsz *= (p.ncell[j] & 1) ? 1u : 2u;
  unsigned tile = item / tsz, r = item - (item / tsz) * tsz;
  unsigned base = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const unsigned bj = (p.ncell[j] & 1) ? 1u : 2u;
    const unsigned off = r % bj;
    r /= bj;
    const unsigned nt = static_cast<unsigned>(p.ncell[j]) / bj;
    const unsigned tj = tile % nt;
    tile /= nt;
    base += (tj * bj + off) * static_cast<unsigned>(p.cstride[j]);
  }
  return base;
}

template <typename TIN, typename TW, bool ADJ>
__global__ void __launch_bounds__(64, 4) k_cell6d4(const KParams p) {
  extern __shared__ __align__(128) float sm6[];
  __shared__ Pipe pipe;
  __shared__ unsigned s_item;
  const int t = threadIdx.x;
  const Tab1D<float>& T = p.t32;
  const int tb = 2 * p.tab;              // constant-table set of the basis
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  const unsigned ncx = static_cast<unsigned>(p.ncx);
  const unsigned S3 = static_cast<unsigned>(p.cstride[5]);   // pencils along v3
  const int N3 = p.ncell[5];
  const unsigned npencils = S3;
  const float winv_t = ADJ ? wprod(T.winv, t) : 1.f;
  const float w_t = ADJ ? wprod(T.w, t) : 1.f;
  // the thread's outflow traces along v3, carried to the next cell of the pencil
  float* carried = sm6 + 3 * kCellSmem + t * 17;
  int bad = 0;

  if (t == 0) {
    for (int b = 0; b < kNumBuf; ++b) mbar_init(&pipe.bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_item = atomicAdd(p.work, 1u);
  }
  __syncthreads();
  unsigned item = s_item;
  if (item >= npencils) return;
  Mover<TIN> mv{sm6, &pipe};
  auto cellp = [&](unsigned c) {
    DG_BOUND(p.err, c, p.ncells);
    return src + static_cast<size_t>(c) * 4096;
  };
  auto setup = [&](unsigned c, float (&sp)[6], unsigned (&nbr)[6]) {
    const unsigned cv = c / ncx, cx = c - cv * ncx;
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * 64 + t) * 3;
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(cx) * 64 + t) * 3;
    sp[0] = ctx[0];
    sp[1] = ctx[1];
    sp[2] = ctx[2];
    sp[3] = ctv[0];
    sp[4] = ctv[1];
    sp[5] = ctv[2];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (ADJ) sp[j] = -sp[j];
      nbr[j] = nb32(p, c, j, signbit(sp[j]) ? 1 : -1);
    }
  };
  // v3 direction of a pencil (the same for all its cells and threads)
  auto pencil_forward = [&](unsigned b) {
    const unsigned cx = b % ncx;
    float c5 = static_cast<const float*>(p.cv_tab)[(static_cast<size_t>(cx) * 64) * 3 + 2];
    if (ADJ) c5 = -c5;
    return !signbit(c5);
  };
  auto pencil_cell = [&](unsigned b, int i, bool fwd) {
    return b + static_cast<unsigned>(fwd ? i : N3 - 1 - i) * S3;
  };

  // buffers: A = 0 holds the current cell, P and Q (1 and 2) are landing
  // buffers holding the x1 and x2 neighbours at the top of an iteration
  constexpr int A = 0;
  int P = 1, Q = 2;
  unsigned base = pencil_base(p, item);
  bool fwd = pencil_forward(base);
  int i = 0;
  unsigned cell = pencil_cell(base, 0, fwd);
  float sp[6];
  unsigned nbr[6];
  setup(cell, sp, nbr);
  mv.issue(A, cellp(cell), t);
  mv.issue(P, cellp(nbr[0]), t);
  mv.issue(Q, cellp(nbr[1]), t);
  bool ok = true;
  __syncthreads();
  if (t == 0) s_item = atomicAdd(p.work, 1u);      // the item after this pencil
  __syncthreads();

  for (;;) {
    // next cell: along the pencil, else the first cell of the next item
    unsigned next_item = item, next_base = base;
    bool next_fwd = fwd;
    int next_i = i + 1;
    if (next_i >= N3) {
      next_item = s_item;           // read by all threads before it changes (barriers below)
      next_i = 0;
      if (next_item < npencils) {
        next_base = pencil_base(p, next_item);
        next_fwd = pencil_forward(next_base);
      }
    }
    const bool has_next = next_item < npencils;
    const unsigned next = has_next ? pencil_cell(next_base, next_i, next_fwd) : 0u;
    const bool need_v3 = i == 0;    // the first cell's upwind v3 neighbour is not carried
    float spn[6];
    unsigned nbn[6];
    if (has_next) setup(next, spn, nbn);
    float u[64], r[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) r[e] = 0.f;

    // ---- phase X: rows of the padded buffers, directions x1, x2, x3
    ok &= mv.wait(A, p.err);
    load_block<true>(u, view<true>(sm6 + A * kCellSmem, t));
    if (ADJ) {
#pragma unroll
      for (int e = 0; e < 64; ++e) u[e] *= winv_t * wprod(T.winv, e);
    }
    ok &= mv.wait(P, p.err);
    direction<0, true, ADJ>(r, u, view<true>(sm6 + P * kCellSmem, t), sp[0], tb, winv_t, T);
    fence_async_smem();
    __syncthreads();
    mv.issue(P, cellp(nbr[2]), t);               // x3
    ok &= mv.wait(Q, p.err);
    direction<1, true, ADJ>(r, u, view<true>(sm6 + Q * kCellSmem, t), sp[1], tb, winv_t, T);
    fence_async_smem();
    __syncthreads();
    mv.issue(Q, cellp(nbr[3]), t);               // v1
    ok &= mv.wait(P, p.err);
    direction<2, true, ADJ>(r, u, view<true>(sm6 + P * kCellSmem, t), sp[2], tb, winv_t, T);
    __syncthreads();                             // P is free: it takes the phase X result
    {
      float* rb = sm6 + P * kCellSmem + t * kPad;
#pragma unroll
      for (int k = 0; k < 16; ++k)
        *reinterpret_cast<float4*>(rb + 4 * k) =
            make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
    }
    __syncthreads();

    // ---- phase V: columns, directions v1, v2, v3
    load_block<false>(u, view<false>(sm6 + A * kCellSmem, t));
    load_block<false>(r, view<false>(sm6 + P * kCellSmem, t));
    if (ADJ) {
#pragma unroll
      for (int e = 0; e < 64; ++e) u[e] *= winv_t * wprod(T.winv, e);
    }
    fence_async_smem();
    __syncthreads();                             // A and P are free
    if (has_next) mv.issue(A, cellp(next), t);   // the next cell
    mv.issue(P, cellp(nbr[4]), t);               // v2
    ok &= mv.wait(Q, p.err);
    direction<0, false, ADJ>(r, u, view<false>(sm6 + Q * kCellSmem, t), sp[3], tb, winv_t, T);
    fence_async_smem();
    __syncthreads();
    if (need_v3)
      mv.issue(Q, cellp(nbr[5]), t);             // v3 (wrapped, not carried)
    else if (has_next)
      mv.issue(Q, cellp(nbn[0]), t);             // x1 of the next cell
    ok &= mv.wait(P, p.err);
    direction<1, false, ADJ>(r, u, view<false>(sm6 + P * kCellSmem, t), sp[4], tb, winv_t, T);
    fence_async_smem();
    __syncthreads();
    if (has_next) mv.issue(P, cellp(need_v3 ? nbn[0] : nbn[1]), t);  // x1 or x2 of the next cell
    float tr[16];
    if (need_v3) {
      ok &= mv.wait(Q, p.err);
      nb_traces<2, false, ADJ>(tr, view<false>(sm6 + Q * kCellSmem, t), sp[5], tb, T);
#pragma unroll
      for (int k = 0; k < 16; ++k) tr[k] *= ADJ ? winv_t : 1.f;
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) tr[k] = carried[k];
    }
    {
      // this cell's outflow traces become the next cell's inflow traces
      float to[16];
      own_traces<2>(to, u, sp[5], tb);
#pragma unroll
      for (int k = 0; k < 16; ++k) carried[k] = to[k];
    }

    // ---- last direction fused with step 5: scatter / LSRK stage update
    const size_t g0 = static_cast<size_t>(cell) * 4096 + t;
    if (p.mode == 0) {
      lines_dir<2>(r, u, tr, sp[5], tb, 1.f);
      TW* dst = static_cast<TW*>(p.dst);
#pragma unroll
      for (int m = 0; m < 64; ++m) {
        float K = r[m];
        if (ADJ) K *= w_t * wprod(T.w, m);
        bad |= !isfinite(K);
        __stcs(dst + g0 + 64 * m, cvt<TW>(K));   // streamed: not read again by this launch
      }
    } else {
      // the FP64 state of the first half of the cell is loaded while the
      // last direction is computed, the second half while the first is used
      double* uu = p.u;
      double uo[32];
#pragma unroll
      for (int m = 0; m < 32; ++m) uo[m] = __ldcs(uu + g0 + 64 * m);
      lines_dir<2>(r, u, tr, sp[5], tb, 1.f);
      TW* dst = static_cast<TW*>(p.dst);
      const float bf = static_cast<float>(p.b_dt);
      const float af = static_cast<float>(p.a_dt);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1) {
#pragma unroll
          for (int m = 0; m < 32; ++m) uo[m] = __ldcs(uu + g0 + 64 * (32 + m));
        }
#pragma unroll
        for (int mm = 0; mm < 32; ++mm) {
          const int m = 32 * h + mm;
          float K = r[m];
          if (ADJ) K *= w_t * wprod(T.w, m);
          bad |= !isfinite(K);
          const size_t g = g0 + 64 * m;
          // one FP64 add per value; everything else in FP32 / integer arithmetic
          const double un = uo[mm] + f32_to_f64(bf * K);
          __stcs(uu + g, un);
          // the next stage vector is streamed out (not read by this launch)
          if constexpr (sizeof(TW) == 4) {
            __stcs(dst + g, p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(uo[mm])));
          } else {
            __stcs(dst + g, p.last_stage ? un : uo[mm] + p.a_dt * f32_to_f64(K));
          }
        }
      }
    }
    fence_async_smem();
    __syncthreads();                             // Q is free; s_item was read by all threads
    if (!ok || !has_next) break;
    if (need_v3) mv.issue(Q, cellp(nbn[1]), t);  // x2 of the next cell
    else {
      const int tmp = P;                         // x1 landed in Q, x2 in P
      P = Q;
      Q = tmp;
    }
    if (next_item != item) {          // block-uniform
      item = next_item;
      base = next_base;
      fwd = next_fwd;
      if (t == 0) s_item = atomicAdd(p.work, 1u);
      __syncthreads();
    }
    i = next_i;
    cell = next;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      sp[j] = spn[j];
      nbr[j] = nbn[j];
    }
  }
  if (!ok && sizeof(TIN) == 4) {
    // a wait gave up: wait (bounded) for every copy that may still be in
    // flight before the block's shared memory is released
    for (int b = 0; b < kNumBuf; ++b) {
      const long long t0 = clock64();
      while (clock64() - t0 < kWaitCycles)
        if (mbar_try_wait(&pipe.bar[b], (mv.phase >> b) & 1u)) break;
    }
  }
  if (bad) atomicOr(p.err, 1);
}

template <typename TIN, typename TW, bool ADJ>
cudaError_t launch6(KParams& p, cudaStream_t s) {
  auto kern = k_cell6d4<TIN, TW, ADJ>;
  // three cell buffers and the carried v3 traces (17 floats per thread)
  const size_t smem = (static_cast<size_t>(kNumBuf) * kCellSmem + 64 * 17) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long npencils = p.cstride[5];
  const long long grid = std::min<long long>(npencils, static_cast<long long>(sms) * per_sm);
  // work items (v3 pencils) are handed out in order by an atomic counter
  e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  kern<<<static_cast<unsigned>(grid), 64, smem, s>>>(p);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Pair variant: 128 threads per cell, two threads per block of 64 values.
//
// Thread T (warp w, lane L) works on block t = 16 w + (L & 7) + 8 (L >> 4) and
// holds the 32 elements of that block whose middle digit has parity
// h = (L >> 3) & 1: local index k = a + 4 b + 8 c is element
// e = a + 4 (h + 2 b) + 16 c.  Lines along the first and last digit are
// thread-local (8 lines each); lines along the middle digit are split between
// the thread and its partner (lane L ^ 8, same t, other h), which exchange
// their halves by warp shuffles.  Half the registers per thread of the
// 64-thread variant give twice the warps per SM.
//
// Data movement: each cell arrives by one tensor copy (cp.async.bulk.tensor,
// two 8 KB boxes issued by a single thread, mbarrier completion) into an
// unpadded buffer with the 128-byte swizzle, instead of 64 per-thread bulk
// copies into padded rows: the per-lane copies serialise in the copy unit and
// cost the issuing warps more than their compute.  With the lane mapping
// above, each group of 8 lanes reads 8 rows with distinct swizzle phases
// (phase X, 16-byte reads) and the two halves of a warp read columns in rows
// 4 apart, whose chunks differ in the swizzle's top bit (phase V, 4-byte
// reads), so both views are free of bank conflicts.
constexpr unsigned kFull = 0xffffffffu;

// element offset (relative to the half's base, 4 h) of local index k
__device__ __forceinline__ constexpr int poff(int k) { return (k & 3) + 8 * ((k >> 2) & 1) + 16 * (k >> 3); }

// Cell buffers hold the 64 x 64 values of a cell (row = v node, column = x
// node) as the tensor copy writes them: two 8 KB halves (columns 0-31 and
// 32-63), each 64 lines of 128 bytes, the 16-byte chunks of line r stored at
// chunk index j ^ (r & 7) (128-byte swizzle).  Element (r, c) is at float
//   (c >> 5) * 2048 + 32 r + 4 ((((c >> 2) & 7) ^ (r & 7))) + (c & 3).
// The thread's offsets: phase X (row t) per (b, c & 1) for the four-value
// groups of the first digit, phase V (column t) per first digit a.
constexpr int kCellF = 4096;          // floats per cell buffer

__device__ __forceinline__ void offsets_x(int (&o)[4], int t, int h) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int b = i & 1, cc = i >> 1;
    o[i] = 32 * t + 4 * ((h + 2 * b + 4 * cc) ^ (t & 7));
  }
}
__device__ __forceinline__ void offsets_v(int (&o)[4], int t, int h) {
  const int jt = ((t >> 2) & 7) ^ (4 * h);
#pragma unroll
  for (int a = 0; a < 4; ++a) o[a] = (t >> 5) * 2048 + (t & 3) + 128 * h + 32 * a + 4 * (jt ^ a);
}
// the four values of group i = b + 2 c (first digit a = 0..3)
template <bool ROWS>
__device__ __forceinline__ void load4(float (&x)[4], const float* buf, const int (&o)[4], int i) {
  const int b = i & 1, cc = i >> 1;
  if constexpr (ROWS) {
    const float4 v = *reinterpret_cast<const float4*>(buf + o[b + 2 * (cc & 1)] + (cc >> 1) * 2048);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = buf[o[a] + 256 * b + 512 * cc];
  }
}
template <bool ROWS>
__device__ __forceinline__ void load_half(float (&x)[32], const float* buf, const int (&o)[4]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float v[4];
    load4<ROWS>(v, buf, o, i);
#pragma unroll
    for (int a = 0; a < 4; ++a) x[4 * i + a] = v[a];
  }
}

// weight product of element e = a + 4 (h + 2 b) + 16 c
__device__ __forceinline__ float wprod_p(const float* w, int k, int h) {
  return w[k & 3] * w[h + 2 * ((k >> 2) & 1)] * w[k >> 3];
}

// local index of point p on line l: J = 0 (first digit, lines (b, c)),
// J = 2 (last digit, lines (a, b)); J = 1 (middle digit): lines (a, c), the
// thread's own points b = 0, 1
template <int J>
__device__ __forceinline__ constexpr int pk(int l, int p) {
  return J == 0 ? p + 4 * (l & 1) + 8 * (l >> 1) : (J == 2 ? (l & 3) + 4 * (l >> 2) + 8 * p
                                                          : (l & 3) + 4 * p + 8 * (l >> 2));
}

// Upwind neighbour traces of the thread's lines along J from a landing
// buffer view (J = 0, 2: 8 lines; J = 1: 16 lines, partial sums over the two
// halves added across the pair).
template <int J, bool ROWS, bool ADJ>
__device__ __forceinline__ void nb_traces_p(float (&tr)[16], const float* nbv, const int (&o)[4], float c, int tb, int h,
                                            const Tab1D<float>& T) {
  const int side = tb + (signbit(c) ? 1 : 0);
  float lw[4];
  if constexpr (J == 1) {
    lw[0] = c_lw[side][h];
    lw[1] = c_lw[side][h + 2];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) lw[i] = c_lw[side][i];
  }
#pragma unroll
  for (int l = 0; l < 16; ++l) tr[l] = 0.f;
  // the neighbour's values arrive four at a time (first digit a = 0..3 at
  // fixed b, c) and are folded into the traces at once
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int b = i & 1, cc = i >> 1;
    float x[4];
    load4<ROWS>(x, nbv, o, i);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (ADJ) x[a] *= wprod_p(T.winv, 4 * i + a, h);
      if constexpr (J == 0) tr[b + 2 * cc] = fmaf(lw[a], x[a], tr[b + 2 * cc]);
      else if constexpr (J == 2) tr[a + 4 * b] = fmaf(lw[cc], x[a], tr[a + 4 * b]);
      else tr[a + 4 * cc] = fmaf(lw[b], x[a], tr[a + 4 * cc]);
    }
  }
  if constexpr (J == 1) {
#pragma unroll
    for (int l = 0; l < 16; ++l) tr[l] += __shfl_xor_sync(kFull, tr[l], 8);
  }
}

// The 16 split lines along the middle digit: the thread owns rows q = h and
// h + 2 and receives the partner's two values of each line by shuffles.  The
// rows depend on h, so their entries (scaled by c) are loaded into registers.
template <bool PACK>
__device__ __forceinline__ void lines_split(float (&r)[32], const float (&u)[32],
                                            const float (&tr)[16], float c, int tb, float tscale, int h) {
  const int side = tb + (signbit(c) ? 1 : 0);
  // columns ordered (own b = 0, own b = 1, partner b = 0, partner b = 1)
  float G[2][4], Ln[2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int q = h + 2 * b;
    G[b][0] = c * c_G[side][q * 4 + h];
    G[b][1] = c * c_G[side][q * 4 + h + 2];
    G[b][2] = c * c_G[side][q * 4 + 1 - h];
    G[b][3] = c * c_G[side][q * 4 + 3 - h];
    Ln[b] = c * c_Ln[side][q];
  }
  if constexpr (PACK) {
    // lines l and l + 1 (first digit a even and odd) hold adjacent values: they
    // go through the packed FP32 FMA together (per lane the same fmaf sequence)
#pragma unroll
    for (int l = 0; l < 16; l += 2) {
      const float2 u0 = make_float2(u[pk<1>(l, 0)], u[pk<1>(l + 1, 0)]);
      const float2 u1 = make_float2(u[pk<1>(l, 1)], u[pk<1>(l + 1, 1)]);
      const float2 v0 = make_float2(__shfl_xor_sync(kFull, u0.x, 8), __shfl_xor_sync(kFull, u0.y, 8));
      const float2 v1 = make_float2(__shfl_xor_sync(kFull, u1.x, 8), __shfl_xor_sync(kFull, u1.y, 8));
      const float2 t = make_float2(tscale * tr[l], tscale * tr[l + 1]);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int k = pk<1>(l, b);
        float2 acc = __ffma2_rn(make_float2(Ln[b], Ln[b]), t, make_float2(r[k], r[k + 1]));
        acc = __ffma2_rn(make_float2(G[b][0], G[b][0]), u0, acc);
        acc = __ffma2_rn(make_float2(G[b][1], G[b][1]), u1, acc);
        acc = __ffma2_rn(make_float2(G[b][2], G[b][2]), v0, acc);
        acc = __ffma2_rn(make_float2(G[b][3], G[b][3]), v1, acc);
        r[k] = acc.x;
        r[k + 1] = acc.y;
      }
    }
    return;
  }
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const float u0 = u[pk<1>(l, 0)], u1 = u[pk<1>(l, 1)];
    const float v0 = __shfl_xor_sync(kFull, u0, 8), v1 = __shfl_xor_sync(kFull, u1, 8);
    const float t = tscale * tr[l];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int k = pk<1>(l, b);
      float acc = fmaf(Ln[b], t, r[k]);
      acc = fmaf(G[b][0], u0, acc);
      acc = fmaf(G[b][1], u1, acc);
      acc = fmaf(G[b][2], v0, acc);
      acc = fmaf(G[b][3], v1, acc);
      r[k] = acc;
    }
  }
}

// PACK: the packed FP32 FMA for the pairs of lines that hold adjacent values
// (the operator application; the stage kernel keeps the scalar form, which
// needs fewer registers next to its FP64 state)
template <int J, bool PACK = false>
__device__ __forceinline__ void lines_p(float (&r)[32], const float (&u)[32], const float (&tr)[16],
                                        float c, int tb, float tscale, int h) {
  if constexpr (J == 1) {
    lines_split<PACK>(r, u, tr, c, tb, tscale, h);
  } else {
    // the 8 local lines along J = 0 or 2
    const int side = tb + (signbit(c) ? 1 : 0);
    float Ln[4], G[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) Ln[i] = c * c_Ln[side][i];
#pragma unroll
    for (int i = 0; i < 16; ++i) G[i] = c * c_G[side][i];
    if constexpr (J == 2 && PACK) {
      // lines (a, b) and (a + 1, b) hold adjacent values: packed FP32 FMA
      // over the pair (per lane the same fmaf sequence as below)
#pragma unroll
      for (int l = 0; l < 8; l += 2) {
        const float2 t = make_float2(tscale * tr[l], tscale * tr[l + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kq = pk<J>(l, q);
          float2 acc = __ffma2_rn(make_float2(Ln[q], Ln[q]), t, make_float2(r[kq], r[kq + 1]));
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const int kp = pk<J>(l, pp);
            acc = __ffma2_rn(make_float2(G[q * 4 + pp], G[q * 4 + pp]), make_float2(u[kp], u[kp + 1]), acc);
          }
          r[kq] = acc.x;
          r[kq + 1] = acc.y;
        }
      }
    } else {
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const float t = tscale * tr[l];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc = fmaf(Ln[q], t, r[pk<J>(l, q)]);
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) acc = fmaf(G[q * 4 + pp], u[pk<J>(l, pp)], acc);
          r[pk<J>(l, q)] = acc;
        }
      }
    }
  }
}

// own outflow traces along the last digit (8 local lines)
__device__ __forceinline__ void own_traces_p(float (&to)[8], const float (&u)[32], float c, int tb) {
  const int side = tb + (signbit(c) ? 1 : 0);
  float lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) lw[i] = c_lw[side][i];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p) s = fmaf(lw[p], u[pk<2>(l, p)], s);
    to[l] = s;
  }
}

template <int J, bool ROWS, bool ADJ, bool PACK>
__device__ __forceinline__ void direction_p(float (&r)[32], const float (&u)[32], const float* nbv,
                                            const int (&o)[4], float c, int tb, float wthread, int h,
                                            const Tab1D<float>& T) {
  float tr[16];
  nb_traces_p<J, ROWS, ADJ>(tr, nbv, o, c, tb, h, T);
  lines_p<J, PACK>(r, u, tr, c, tb, ADJ ? wthread : 1.f, h);
}

// Tensor copy of one cell into a swizzled buffer: two boxes of 32 x 1 x 64
// (the column halves of its 64 rows) of the 3D view (32, 2, rows) of the
// stage vector, counted on the buffer's mbarrier.
__device__ __forceinline__ void tma_cell(float* dst, const CUtensorMap* tm, unsigned cell,
                                         unsigned long long* bar, unsigned long long pol) {
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst + 2048 * h2)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(0), "r"(h2), "r"(static_cast<int>(cell * 64u)),
        "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Face layers of a cell for the Gauss-Lobatto collocation, whose neighbour
// traces are the neighbour's face nodes: the 16 rows (v nodes) with one v
// digit fixed, as two compact 32 x 16 boxes (column halves) of the 5D view
// (32, 2, 4 [q4], 4 [q5], 4 cells [q6]) of the stage vector.  dir 0, 1, 2 =
// v1, v2, v3; f = the face node (0 or 3).  Compact row m runs over the other
// two v digits (the lower one fastest).
struct FaceMaps {
  CUtensorMap m[3];
};
__device__ __forceinline__ void tma_face(float* dst, const FaceMaps* fm, int dir, unsigned cell, int f,
                                         unsigned long long* bar, unsigned long long pol) {
  const int c2 = dir == 0 ? f : 0, c3 = dir == 1 ? f : 0;
  const int c4 = static_cast<int>(cell * 4u) + (dir == 2 ? f : 0);
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(smem_u32(dst + 512 * h2)),
        "l"(reinterpret_cast<unsigned long long>(&fm->m[dir])), "r"(0), "r"(h2), "r"(c2), "r"(c3),
        "r"(c4), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Moves cells into the swizzled buffers.  FP32 input: one thread issues the
// tensor copy.  FP64 input: each row's thread loads, converts and stores it.
template <typename TIN>
struct Mover2 {
  float* sm;
  Pipe* pp;
  const CUtensorMap* tm;
  unsigned phase = 0;
  unsigned long long pol = l2_evict_last();

  __device__ __forceinline__ void issue(int b, unsigned cell, const TIN* src, int T_, int t, int h) {
    float* d = sm + b * kCellF;
    if constexpr (sizeof(TIN) == 4) {
      if (T_ == 0) {
        mbar_expect_tx(&pp->bar[b], 4096 * 4);
        tma_cell(d, tm, cell, &pp->bar[b], pol);
      }
    } else {
      if (h == 0) {
        const TIN* g = src + static_cast<size_t>(cell) * 4096 + t * 64;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          *reinterpret_cast<float4*>(d + (j >> 3) * 2048 + 32 * t + 4 * ((j & 7) ^ (t & 7))) =
              ld4(g + 4 * j);
      }
    }
  }
  // FP32 input only: the face layer of ``cell`` along v direction dir
  __device__ __forceinline__ void issue_face(int b, unsigned cell, const FaceMaps* fm, int dir, int f,
                                             int T_) {
    if (T_ == 0) {
      mbar_expect_tx(&pp->bar[b], 16 * 64 * 4);
      tma_face(sm + b * kCellF, fm, dir, cell, f, &pp->bar[b], pol);
    }
  }
  __device__ __forceinline__ bool wait(int b, int* err) {
    if constexpr (sizeof(TIN) == 4) {
      const unsigned par = (phase >> b) & 1u;
      phase ^= 1u << b;
      if (mbar_try_wait(&pp->bar[b], par)) return true;
      const long long t0 = clock64();
      while (clock64() - t0 < kWaitCycles)
        if (mbar_try_wait(&pp->bar[b], par)) return true;
      atomicOr(err, 2);
      return false;
    } else {
      __syncthreads();
      return true;
    }
  }
};

// Upwind traces from a compact face buffer (Gauss-Lobatto collocation: the
// trace of a line is its face node, the neighbour's face layer holds them).
// Thread (t, h) in phase V, local direction J of the v block:
//   J = 0 (v1): lines (b, c) -> row m = (h + 2 b) + 4 c
//   J = 1 (v2): lines (a, c) -> row m = a + 4 c      (16 lines, no shuffle)
//   J = 2 (v3): lines (a, b) -> row m = a + 4 (h + 2 b)
template <int J, bool ADJ>
__device__ __forceinline__ void face_traces(float (&tr)[16], const float* buf, int t, int h, int f,
                                            const Tab1D<float>& T) {
  const int base = (t >> 5) * 512 + (t & 3);
  const int tc = (t >> 2) & 7;
  constexpr int nl = J == 1 ? 16 : 8;
#pragma unroll
  for (int l = 0; l < nl; ++l) {
    int m, k;   // compact row, and the local element index (for the adjoint weights)
    if constexpr (J == 0) {
      m = (h + 2 * (l & 1)) + 4 * (l >> 1);
      k = f + 4 * (l & 1) + 8 * (l >> 1);
    } else if constexpr (J == 1) {
      m = l;
      k = (l & 3) + 8 * (l >> 2);
    } else {
      m = (l & 3) + 4 * (h + 2 * (l >> 2));
      k = (l & 3) + 4 * (l >> 2) + 8 * f;
    }
    float x = buf[base + 32 * m + 4 * (tc ^ (m & 7))];
    if (ADJ) {
      if constexpr (J == 1) x *= T.winv[l & 3] * T.winv[f] * T.winv[l >> 2];
      else x *= wprod_p(T.winv, k, h);
    }
    tr[l] = x;
  }
}

// Block-uniform description of a work item (a v3 pencil), kept in shared
// memory so that per-cell neighbour indices need no integer division.
struct PencilInfo {
  unsigned base;       // first cell (v3 = 0)
  unsigned cx, cvb;    // x cell, and v cell of the first cell
  unsigned coord[5];   // cell coordinates in x1, x2, x3, v1, v2
  unsigned fwd;        // walk direction along v3 (upwind first)
};

template <bool ADJ>
__device__ __forceinline__ void pencil_info(const KParams& p, unsigned item, PencilInfo& pi) {
  unsigned tsz = 1;
#pragma unroll
  for (int j = 0; j < 5; ++j) tsz *= (p.ncell[j] & 1) ? 1u : 2u;
  unsigned tile = item / tsz, r = item - (item / tsz) * tsz;
  unsigned base = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const unsigned bj = (p.ncell[j] & 1) ? 1u : 2u;
    const unsigned off = r % bj;
    r /= bj;
    const unsigned nt = static_cast<unsigned>(p.ncell[j]) / bj;
    const unsigned tj = tile % nt;
    tile /= nt;
    pi.coord[j] = tj * bj + off;
    base += pi.coord[j] * static_cast<unsigned>(p.cstride[j]);
  }
  const unsigned ncx = static_cast<unsigned>(p.ncx);
  pi.base = base;
  pi.cx = base % ncx;
  pi.cvb = base / ncx;
  float c5 = static_cast<const float*>(p.cv_tab)[(static_cast<size_t>(pi.cx) * 64) * 3 + 2];
  if (ADJ) c5 = -c5;
  pi.fwd = signbit(c5) ? 0u : 1u;
}

// upwind neighbour along j of a cell at coordinate cj (periodic wrap)
__device__ __forceinline__ unsigned nb_c(const KParams& p, unsigned cell, unsigned cj, int j,
                                         float c) {
  const unsigned st = static_cast<unsigned>(p.cstride[j]);
  const unsigned nj = static_cast<unsigned>(p.ncell[j]);
  if (!signbit(c)) return cj == 0 ? cell + (nj - 1) * st : cell - st;
  return cj == nj - 1 ? cell - (nj - 1) * st : cell + st;
}

// MODE 0: operator application (dst = K); MODE 1: fused LSRK stage.
// FACE: Gauss-Lobatto collocation with FP32 input; the v neighbours arrive
// as face layers only (a quarter of a cell each).
// TAB: constant-table set (0 Gauss-Legendre, 1 Gauss-Lobatto), a compile-time
// offset so that it costs no register.
template <typename TIN, typename TW, bool ADJ, int MODE, bool FACE, int TAB>
__device__ __forceinline__ void cell6d4p_body(const KParams& p, const CUtensorMap& tmap,
                                              const FaceMaps* fmaps) {
  extern __shared__ __align__(128) float sm_raw[];
  // swizzled buffers need 1024-byte alignment (one KB of slack is allocated)
  float* const sm6 = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u) / 4;
  __shared__ Pipe pipe;
  __shared__ unsigned s_item;
  __shared__ PencilInfo s_pi[2];      // current and next item
  const int T_ = threadIdx.x;
  const int lane = T_ & 31;
  const int h = (lane >> 3) & 1;
  const int t = 16 * (T_ >> 5) + (lane & 7) + 8 * (lane >> 4);
  const bool issuer = h == 0;          // one thread per block row issues its copies
  const Tab1D<float>& T = p.t32;
  constexpr int tb = 2 * TAB;            // constant-table set of the basis
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  const unsigned S3 = static_cast<unsigned>(p.cstride[5]);   // pencils along v3
  const unsigned SV3 = S3 / static_cast<unsigned>(p.ncx);    // v-cell stride of v3
  const int N3 = p.v3_n > 0 ? p.v3_n : p.ncell[5];            // cells walked per pencil
  const unsigned V3L = p.v3_n > 0 ? static_cast<unsigned>(p.v3_lo) : 0u;
  const unsigned npencils = S3;
  const float winv_t = ADJ ? wprod(T.winv, t) : 1.f;
  const float w_t = ADJ ? wprod(T.w, t) : 1.f;
  // the thread's outflow traces along v3, carried to the next cell of the pencil
  float* carried = sm6 + 3 * kCellF + T_ * 8;
  int bad = 0;

  if (T_ == 0) {
    for (int b = 0; b < kNumBuf; ++b) mbar_init(&pipe.bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const unsigned it = atomicAdd(p.work, 1u);
    s_item = it;
    if (it < npencils) pencil_info<ADJ>(p, it, s_pi[0]);
  }
  __syncthreads();
  unsigned item = s_item;
  if (item >= npencils) return;
  Mover2<TIN> mv{sm6, &pipe, &tmap};
  int slot = 0;
  auto issue = [&](int b, unsigned c) {
    DG_BOUND(p.err, c, p.ncells);
    mv.issue(b, c, src, T_, t, h);
  };
  auto v3c = [&](const PencilInfo& pi, int i) {
    unsigned c5 = V3L + (pi.fwd ? static_cast<unsigned>(i) : static_cast<unsigned>(N3 - 1 - i));
    DG_BOUND(p.err, c5, p.ncell[5]);
    return c5;
  };
  // speeds of the thread's nodes and the upwind neighbours of cell i of a pencil
  auto setup = [&](const PencilInfo& pi, int i, unsigned& cell, float (&sp)[6],
                   unsigned (&nbr)[6]) {
    const unsigned c5 = v3c(pi, i);
    cell = pi.base + c5 * S3;
    const unsigned cv = pi.cvb + c5 * SV3;
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * 64 + t) * 3;
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(pi.cx) * 64 + t) * 3;
    sp[0] = ctx[0];
    sp[1] = ctx[1];
    sp[2] = ctx[2];
    sp[3] = ctv[0];
    sp[4] = ctv[1];
    sp[5] = ctv[2];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (ADJ) sp[j] = -sp[j];
      nbr[j] = nb_c(p, cell, j < 5 ? pi.coord[j] : c5, j, sp[j]);
    }
  };

  constexpr int A = 0;
  int P = 1, Q = 2;
  int i = 0;
  unsigned cell;
  float sp[6];
  unsigned nbr[6];
  setup(s_pi[slot], 0, cell, sp, nbr);
  issue(A, cell);
  issue(P, nbr[0]);
  issue(Q, nbr[1]);
  bool ok = true;
  __syncthreads();
  if (T_ == 0) {                                 // the item after this pencil
    const unsigned it = atomicAdd(p.work, 1u);
    s_item = it;
    if (it < npencils) pencil_info<ADJ>(p, it, s_pi[1]);
  }
  __syncthreads();

  for (;;) {
    unsigned next_item = item;
    int next_slot = slot;
    int next_i = i + 1;
    if (next_i >= N3) {
      next_item = s_item;           // read by all threads before it changes (barriers below)
      next_slot = slot ^ 1;
      next_i = 0;
    }
    const bool has_next = next_item < npencils;
    const bool need_v3 = i == 0;    // the first cell's upwind v3 neighbour is not carried
    DG_BOUND(p.err, cell, p.ncells);
    DG_BOUND(p.err, nbr[3], p.ncells);
    DG_BOUND(p.err, nbr[4], p.ncells);
    DG_BOUND(p.err, nbr[5], p.ncells);
    // the next cell's upwind x1 and x2 neighbours (prefetched during phase V);
    // its full setup follows at the end of this iteration
    unsigned next = 0, nx0 = 0, nx1 = 0;
    if (has_next) {
      const PencilInfo& pn = s_pi[next_slot];
      const unsigned c5 = v3c(pn, next_i);
      next = pn.base + c5 * S3;
      const unsigned cv = pn.cvb + c5 * SV3;
      const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * 64 + t) * 3;
      float c0 = ctx[0], c1 = ctx[1];
      if (ADJ) {
        c0 = -c0;
        c1 = -c1;
      }
      nx0 = nb_c(p, next, pn.coord[0], 0, c0);
      nx1 = nb_c(p, next, pn.coord[1], 1, c1);
    }
    float u[32], r[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) r[e] = 0.f;

    // ---- phase X: rows, directions x1, x2 (split), x3
    int o[4];
    offsets_x(o, t, h);
    ok &= mv.wait(A, p.err);
    load_half<true>(u, sm6 + A * kCellF, o);
    if (ADJ) {
#pragma unroll
      for (int k = 0; k < 32; ++k) u[k] *= winv_t * wprod_p(T.winv, k, h);
    }
    ok &= mv.wait(P, p.err);
    direction_p<0, true, ADJ, MODE == 0>(r, u, sm6 + P * kCellF, o, sp[0], tb, winv_t, h, T);
    fence_async_smem();
    __syncthreads();
    issue(P, nbr[2]);                            // x3
    ok &= mv.wait(Q, p.err);
    direction_p<1, true, ADJ, MODE == 0>(r, u, sm6 + Q * kCellF, o, sp[1], tb, winv_t, h, T);
    fence_async_smem();
    __syncthreads();
    if constexpr (FACE)
      mv.issue_face(Q, nbr[3], fmaps, 0, signbit(sp[3]) ? 0 : 3, T_);   // v1 face layer
    else
      issue(Q, nbr[3]);                          // v1
    ok &= mv.wait(P, p.err);
    direction_p<2, true, ADJ, MODE == 0>(r, u, sm6 + P * kCellF, o, sp[2], tb, winv_t, h, T);
    __syncthreads();                             // P is free: it takes the phase X result
    {
      float* rb = sm6 + P * kCellF;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int b = i & 1, cc = i >> 1;
        *reinterpret_cast<float4*>(rb + o[b + 2 * (cc & 1)] + (cc >> 1) * 2048) =
            make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
      }
    }
    __syncthreads();

    // ---- phase V: columns, directions v1, v2 (split), v3
    offsets_v(o, t, h);
    load_half<false>(u, sm6 + A * kCellF, o);
    load_half<false>(r, sm6 + P * kCellF, o);
    if (ADJ) {
#pragma unroll
      for (int k = 0; k < 32; ++k) u[k] *= winv_t * wprod_p(T.winv, k, h);
    }
    fence_async_smem();
    __syncthreads();                             // A and P are free
    if (has_next) issue(A, next);                // the next cell
    if constexpr (FACE)
      mv.issue_face(P, nbr[4], fmaps, 1, signbit(sp[4]) ? 0 : 3, T_);   // v2 face layer
    else
      issue(P, nbr[4]);                          // v2
    ok &= mv.wait(Q, p.err);
    if constexpr (FACE) {
      float tr[16];
      face_traces<0, ADJ>(tr, sm6 + Q * kCellF, t, h, signbit(sp[3]) ? 0 : 3, T);
      lines_p<0, MODE == 0>(r, u, tr, sp[3], tb, ADJ ? winv_t : 1.f, h);
    } else {
      direction_p<0, false, ADJ, MODE == 0>(r, u, sm6 + Q * kCellF, o, sp[3], tb, winv_t, h, T);
    }
    fence_async_smem();
    __syncthreads();
    // the cell's FP64 state is needed only in the epilogue: ask L2 for it two
    // directions ahead (one 512-byte row per issuing thread).  Asked for at
    // the start of the cell, a fifth of it was evicted again before use.
    if (MODE >= 1 && issuer) prefetch_l2(p.u + static_cast<size_t>(cell) * 4096 + t * 64, 512);
    if (MODE == 2 && issuer) prefetch_l2(p.kref + static_cast<size_t>(cell) * 4096 + t * 64, 256);
    if (need_v3) {
      if constexpr (FACE)
        mv.issue_face(Q, nbr[5], fmaps, 2, signbit(sp[5]) ? 0 : 3, T_);  // v3 face layer
      else
        issue(Q, nbr[5]);                        // v3 (wrapped, not carried)
    }
    else if (has_next)
      issue(Q, nx0);                             // x1 of the next cell
    ok &= mv.wait(P, p.err);
    if constexpr (FACE) {
      float tr[16];
      face_traces<1, ADJ>(tr, sm6 + P * kCellF, t, h, signbit(sp[4]) ? 0 : 3, T);
      lines_p<1, MODE == 0>(r, u, tr, sp[4], tb, ADJ ? winv_t : 1.f, h);
    } else {
      direction_p<1, false, ADJ, MODE == 0>(r, u, sm6 + P * kCellF, o, sp[4], tb, winv_t, h, T);
    }
    fence_async_smem();
    __syncthreads();
    if (has_next) issue(P, need_v3 ? nx0 : nx1);        // x1 or x2 of the next cell
    float tr[16];
    if (need_v3) {
      ok &= mv.wait(Q, p.err);
      if constexpr (FACE)
        face_traces<2, ADJ>(tr, sm6 + Q * kCellF, t, h, signbit(sp[5]) ? 0 : 3, T);
      else
        nb_traces_p<2, false, ADJ>(tr, sm6 + Q * kCellF, o, sp[5], tb, h, T);
#pragma unroll
      for (int k = 0; k < 8; ++k) tr[k] *= ADJ ? winv_t : 1.f;
    } else {
      const float4 c0 = *reinterpret_cast<const float4*>(carried);
      const float4 c1 = *reinterpret_cast<const float4*>(carried + 4);
      tr[0] = c0.x; tr[1] = c0.y; tr[2] = c0.z; tr[3] = c0.w;
      tr[4] = c1.x; tr[5] = c1.y; tr[6] = c1.z; tr[7] = c1.w;
    }
    {
      float to[8];
      own_traces_p(to, u, sp[5], tb);
      *reinterpret_cast<float4*>(carried) = make_float4(to[0], to[1], to[2], to[3]);
      *reinterpret_cast<float4*>(carried + 4) = make_float4(to[4], to[5], to[6], to[7]);
    }

    // ---- last direction fused with step 5: scatter / LSRK stage update
    const size_t g0 = static_cast<size_t>(cell) * 4096 + t + 256 * h;
    if constexpr (MODE == 0) {
      lines_p<2, MODE == 0>(r, u, tr, sp[5], tb, 1.f, h);
      TW* dst = static_cast<TW*>(p.dst);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        float K = r[k];
        if (ADJ) K *= w_t * wprod_p(T.w, k, h);
        bad |= !isfinite(K);
        __stcs(dst + g0 + 64 * poff(k), cvt<TW>(K));
      }
    } else {
      // the FP64 state streams through in chunks of 8 values, each chunk's
      // loads issued while the previous one is used
      double* uu = p.u;
      double ua[8];
      float ka[8];   // MODE 2 (delta-f form): the reference operator K_ref
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ua[k] = __ldcs(uu + g0 + 64 * poff(k));
        ka[k] = MODE == 2 ? __ldcs(p.kref + g0 + 64 * poff(k)) : 0.f;
      }
      lines_p<2, MODE == 0>(r, u, tr, sp[5], tb, 1.f, h);
      TW* dst = static_cast<TW*>(p.dst);
      const float bf = static_cast<float>(p.b_dt);
      const float af = static_cast<float>(p.a_dt);
      float nanacc = 0.f;
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        double ub[8];
        float kb[8];
        if (ch < 3) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            ub[k] = __ldcs(uu + g0 + 64 * poff(8 * (ch + 1) + k));
            kb[k] = MODE == 2 ? __ldcs(p.kref + g0 + 64 * poff(8 * (ch + 1) + k)) : 0.f;
          }
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int k = 8 * ch + kk;
          float K = r[k];
          if (ADJ) K *= w_t * wprod_p(T.w, k, h);
          if (MODE == 2) K += ka[kk];
          nanacc = fmaf(K, 0.f, nanacc);   // stays 0 unless K is Inf or NaN
          const size_t g = g0 + 64 * poff(k);
          const double un = ua[kk] + f32_to_f64_finite(bf * K);
          __stcs(uu + g, un);
          if constexpr (sizeof(TW) == 4) {
            __stcs(dst + g, p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(ua[kk])));
          } else {
            __stcs(dst + g, p.last_stage ? un : ua[kk] + p.a_dt * f32_to_f64(K));
          }
        }
        if (ch < 3) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            ua[k] = ub[k];
            ka[k] = kb[k];
          }
        }
      }
      bad |= nanacc != 0.f;
    }
    fence_async_smem();
    __syncthreads();                             // Q is free; s_item was read by all threads
    if (!ok || !has_next) break;
    if (need_v3) issue(Q, nx1);                  // x2 of the next cell
    else {
      const int tmp = P;                         // x1 landed in Q, x2 in P
      P = Q;
      Q = tmp;
    }
    if (next_item != item) {          // block-uniform
      item = next_item;
      slot = next_slot;
      if (T_ == 0) {
        const unsigned it = atomicAdd(p.work, 1u);
        s_item = it;
        if (it < npencils) pencil_info<ADJ>(p, it, s_pi[slot ^ 1]);
      }
      __syncthreads();
    }
    i = next_i;
    setup(s_pi[slot], i, cell, sp, nbr);
  }
  if (!ok && sizeof(TIN) == 4) {
    for (int b = 0; b < kNumBuf; ++b) {
      const long long t0 = clock64();
      while (clock64() - t0 < kWaitCycles)
        if (mbar_try_wait(&pipe.bar[b], (mv.phase >> b) & 1u)) break;
    }
  }
  if (bad) atomicOr(p.err, 1);
}

template <typename TIN, typename TW, bool ADJ, int MODE, int TAB>
__global__ void __launch_bounds__(128, 4) k_cell6d4p(const KParams p,
                                                      const __grid_constant__ CUtensorMap tmap) {
  cell6d4p_body<TIN, TW, ADJ, MODE, false, TAB>(p, tmap, nullptr);
}

// Gauss-Lobatto collocation, FP32 input: the v neighbours as face layers.
template <typename TIN, typename TW, bool ADJ, int MODE>
__global__ void __launch_bounds__(128, 4) k_cell6d4p_face(const KParams p,
                                                           const __grid_constant__ CUtensorMap tmap,
                                                           const __grid_constant__ FaceMaps fmaps) {
  cell6d4p_body<TIN, TW, ADJ, MODE, true, 1>(p, tmap, &fmaps);
}

// 3D view (32 floats, 2 halves, 64 rows per cell) of an FP32 stage vector,
// box 32 x 1 x 64, 128-byte swizzle.
cudaError_t encode_cell_map(CUtensorMap* tm, const void* src, long long ncells) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {32, 2, static_cast<cuuint64_t>(ncells) * 64};
  const cuuint64_t strides[2] = {128, 256};
  const cuuint32_t box[3] = {32, 1, 64};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(src), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Face layers: 5D view (32 floats, 2 halves, 4 [q4], 4 [q5], 4 cells [q6])
// of an FP32 stage vector, boxes of 16 rows with one v digit fixed.
cudaError_t encode_face_maps(FaceMaps* fm, const void* src, long long ncells) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {32, 2, 4, 4, static_cast<cuuint64_t>(ncells) * 4};
  const cuuint64_t strides[4] = {128, 256, 1024, 4096};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const cuuint32_t boxes[3][5] = {{32, 1, 1, 4, 4}, {32, 1, 4, 1, 4}, {32, 1, 4, 4, 1}};
  for (int d = 0; d < 3; ++d) {
    CUresult r = enc(&fm->m[d], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(src), dims,
                     strides, boxes[d], estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// FP64 vectors, FP32 sweeps, Gauss-Legendre: the cells come from p.src32 (the
// input rounded to FP32 beforehand) by tensor copies; the output or the stage
// vector is written in FP64 exactly as by the FP64-input kernel.
template <bool ADJ>
cudaError_t launch6p_in32(const KParams& p0, cudaStream_t s) {
  KParams p = p0;
  p.src = p0.src32;
  if (p.ncells * 64 >= (1LL << 31)) return cudaErrorNotSupported;
  const void* kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell6d4p<float, double, ADJ, 0, 0>)
                                 : reinterpret_cast<const void*>(k_cell6d4p<float, double, ADJ, 1, 0>);
  alignas(64) CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  cudaError_t e;
  if ((e = encode_cell_map(&tm, p.src, p.ncells)) != cudaSuccess) return e;
  const size_t smem = 1024 + (static_cast<size_t>(kNumBuf) * kCellF + 128 * 8) * sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long grid = std::min<long long>(p.cstride[5], static_cast<long long>(sms) * per_sm);
  if ((e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  (p.mode == 0 ? k_cell6d4p<float, double, ADJ, 0, 0> : k_cell6d4p<float, double, ADJ, 1, 0>)
      <<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm);
  return cudaGetLastError();
}

template <typename TIN, typename TW, bool ADJ>
cudaError_t launch6p(KParams& p, cudaStream_t s) {
  constexpr bool kF32 = sizeof(TIN) == 4;
  const bool face = kF32 && p.tab == 1;
  // delta-f stages: only the Gauss-Legendre FP32 kernel (else the generic one)
  if (p.kref && (!kF32 || face || p.tab != 0 || ADJ || p.mode != 1)) return cudaErrorNotSupported;
  const bool df = p.kref != nullptr;
  if constexpr (!kF32) {
    // FP64 input with an FP32 copy of it: the FP32-input kernel, FP64 output
    if (p.src32 != nullptr && p.tab == 0 && !df) return launch6p_in32<ADJ>(p, s);
  }
  // kernels: Gauss-Legendre tables; Gauss-Lobatto with FP32 input (face
  // layers); Gauss-Lobatto with FP64 input (full cells)
  const void* kern = nullptr;
  if constexpr (kF32) {
    if (df) {
      if constexpr (!ADJ) kern = reinterpret_cast<const void*>(k_cell6d4p<float, float, false, 2, 0>);
    } else if (face) {
      kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell6d4p_face<float, float, ADJ, 0>)
                         : reinterpret_cast<const void*>(k_cell6d4p_face<float, float, ADJ, 1>);
    } else {
      kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 0, 0>)
                         : reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 1, 0>);
    }
  } else {
    if (p.tab == 1)
      kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 0, 1>)
                         : reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 1, 1>);
    else
      kern = p.mode == 0 ? reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 0, 0>)
                         : reinterpret_cast<const void*>(k_cell6d4p<TIN, TW, ADJ, 1, 0>);
  }
  if (kern == nullptr) return cudaErrorNotSupported;
  // cell coordinates of the tensor copies are 32-bit signed rows
  if (p.ncells * 64 >= (1LL << 31)) return cudaErrorNotSupported;
  alignas(64) CUtensorMap tm;
  alignas(64) FaceMaps fm;
  std::memset(&tm, 0, sizeof(tm));
  std::memset(&fm, 0, sizeof(fm));
  cudaError_t e;
  if constexpr (kF32) {
    if ((e = encode_cell_map(&tm, p.src, p.ncells)) != cudaSuccess) return e;
    if (face && (e = encode_face_maps(&fm, p.src, p.ncells)) != cudaSuccess) return e;
  }
  // 1 KB alignment slack, three cell buffers, the carried v3 traces (8 floats per thread)
  const size_t smem = 1024 + (static_cast<size_t>(kNumBuf) * kCellF + 128 * 8) * sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long npencils = p.cstride[5];
  const long long grid = std::min<long long>(npencils, static_cast<long long>(sms) * per_sm);
  e = cudaMemsetAsync(p.work, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if constexpr (kF32 && !ADJ) {
    if (df) {
      k_cell6d4p<float, float, false, 2, 0><<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm);
      return cudaGetLastError();
    }
  }
  if constexpr (kF32) {
    if (face)
      (p.mode == 0 ? k_cell6d4p_face<float, float, ADJ, 0> : k_cell6d4p_face<float, float, ADJ, 1>)
          <<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm, fm);
    else
      (p.mode == 0 ? k_cell6d4p<TIN, TW, ADJ, 0, 0> : k_cell6d4p<TIN, TW, ADJ, 1, 0>)
          <<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm);
  } else {
    if (p.tab == 1)
      (p.mode == 0 ? k_cell6d4p<TIN, TW, ADJ, 0, 1> : k_cell6d4p<TIN, TW, ADJ, 1, 1>)
          <<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm);
    else
      (p.mode == 0 ? k_cell6d4p<TIN, TW, ADJ, 0, 0> : k_cell6d4p<TIN, TW, ADJ, 1, 0>)
          <<<static_cast<unsigned>(grid), 128, smem, s>>>(p, tm);
  }
  return cudaGetLastError();
}

}  // namespace

// Self-test of the bounded waits: one block arrives on an mbarrier that
// expects 16 bytes no copy will ever deliver, waits with the same bounded
// loop as the cell kernels (a short limit here), gives up and latches the
// timeout bit.  Nothing is in flight when it returns.
__global__ void k_wait_probe(int* err, long long limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, 16);
  }
  __syncthreads();
  const long long t0 = clock64();
  bool done = false;
  while (!done && clock64() - t0 < limit) done = mbar_try_wait(&bar, 0);
  if (!done && threadIdx.x == 0) atomicOr(err, 2);
}

cudaError_t launch_wait_probe(int* err, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(err, 2000000LL);   // about 1 ms of SM clock
  return cudaGetLastError();
}

cudaError_t init_cell6d_tables(const Tab1D<float>& t, int tab) {
  float G[2][16], Ln[2][4], lw[2][4];
  for (int i = 0; i < 16; ++i) {
    G[0][i] = t.Gp[(i / 4) * 4 + i % 4];
    G[1][i] = t.Gn[(i / 4) * 4 + i % 4];
  }
  for (int i = 0; i < 4; ++i) {
    Ln[0][i] = t.Lm[i];
    Ln[1][i] = -t.Lp[i];
    lw[0][i] = t.lp[i];
    lw[1][i] = t.lm[i];
  }
  // table set ``tab`` (0: Gauss-Legendre, 1: Gauss-Lobatto collocation)
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_G, G, sizeof(G), tab * sizeof(G))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_Ln, Ln, sizeof(Ln), tab * sizeof(Ln))) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_lw, lw, sizeof(lw), tab * sizeof(lw));
}

cudaError_t launch_cell_6d4(int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.dx != 3 || p.dv != 3 || p.ncells >= (1LL << 31)) return cudaErrorNotSupported;
  if (p.v3_n > 0 && (cfg.variant != 2 || p.v3_lo < 0 || p.v3_lo + p.v3_n > p.ncell[5]))
    return cudaErrorInvalidValue;                                   // v3 ranges: pair kernel only
  if (p.kref && cfg.variant != 2) return cudaErrorNotSupported;   // delta-f: pair kernel or generic
  if (cfg.variant == 2) {
    if (combo == kFFF)
      return p.adjoint ? launch6p<float, float, true>(p, s) : launch6p<float, float, false>(p, s);
    if (combo == kFDD)
      return p.adjoint ? launch6p<double, double, true>(p, s) : launch6p<double, double, false>(p, s);
    return cudaErrorNotSupported;
  }
  if (combo == kFFF)
    return p.adjoint ? launch6<float, float, true>(p, s) : launch6<float, float, false>(p, s);
  if (combo == kFDD)
    return p.adjoint ? launch6<double, double, true>(p, s) : launch6<double, double, false>(p, s);
  return cudaErrorNotSupported;
}

}  // namespace dg
