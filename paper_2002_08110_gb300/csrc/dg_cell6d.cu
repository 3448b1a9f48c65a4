// Specialised element-centric cell kernel for d = 6 (3 x + 3 v), n = 4 (k = 3),
// FP32 sweeps and fluxes.
//
// A cell has 4096 values, q = q_x + 64 q_v with q_x = (q1,q2,q3), q_v = (q4,q5,q6)
// (x_1 fastest).  64 threads (one "group") process one cell in two phases,
// mirroring Algorithm 2's split of the cell work into the x-space part and the
// v-space part (which reduces the working set):
//   phase X: thread t owns the v node q_v = t and holds the 4x4x4 x-block
//            {q_x} of that node in registers, so every line along x1, x2, x3
//            is thread-local; the contravariant speeds c_1..c_3 depend on q_v
//            only (a_x = v), so they are thread constants;
//   phase V: thread t owns the x node q_x = t and holds the 4x4x4 v-block,
//            lines along v1, v2, v3 thread-local; c_4..c_6 = 2 E(x)/h_v depend
//            on q_x only.
// Per direction and line: du_q += c (sum_p G[q][p] u_p + L_nb[q] t_nb) with the
// collocated 1D operator of dg_internal.h; t_nb is the upwind neighbour's trace
// on the shared face, computed from the neighbour's line, read from global
// memory (periodic wrap; phase X reads the neighbour's contiguous 256-byte
// x-block, phase V reads stride-64 values that are coalesced across the warp).
// Shared memory holds the cell's input (for the phase V transpose) and the
// phase X partial result; blocks of 64 floats are padded to 68 so that the
// 16-byte accesses of phase X and the 4-byte accesses of phase V are free of
// bank conflicts.
//
// Modes: operator application (dst = K) or fused LSRK stage
// (u += b dt K in FP64; w_out = u + a dt K).  Adjoint: L^T = M L(-a) M^{-1}.
#include "dg_convert.cuh"
#include "dg_generic.cuh"

namespace dg {
namespace {

constexpr int kPad = 68;              // padded floats per 64-value block
constexpr int kCellSmem = 64 * kPad;  // floats per cell buffer

__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(64) : "memory");
}

template <typename TIN>
struct Ld;
template <>
struct Ld<float> {
  static __device__ __forceinline__ float4 ld4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
};
template <>
struct Ld<double> {
  static __device__ __forceinline__ float4 ld4(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    return make_float4(f64_to_f32(a.x), f64_to_f32(a.y), f64_to_f32(b.x), f64_to_f32(b.y));
  }
  static __device__ __forceinline__ float ld1(const double* p) {
    return f64_to_f32(__ldg(p));
  }
};

// Element index inside a 4x4x4 block of the point p on line (l1, l2) along
// local direction J.
template <int J>
__device__ __forceinline__ constexpr int eidx(int l1, int l2, int p) {
  return J == 0 ? p + 4 * l1 + 16 * l2 : (J == 1 ? l1 + 4 * p + 16 * l2 : l1 + 4 * l2 + 16 * p);
}

// Row (b, c) of the neighbour's block: the four values a = 0..3 at element
// a + 4 b + 16 c.  STRIDE is the distance between consecutive elements in
// memory (1 in phase X, 64 in phase V).
template <typename TIN, int STRIDE>
__device__ __forceinline__ float4 nb_row(const TIN* base, int b, int c) {
  const TIN* p = base + (4 * b + 16 * c) * STRIDE;
  if constexpr (STRIDE == 1) {
    return Ld<TIN>::ld4(p);
  } else {
    return make_float4(Ld<TIN>::ld1(p), Ld<TIN>::ld1(p + STRIDE), Ld<TIN>::ld1(p + 2 * STRIDE),
                       Ld<TIN>::ld1(p + 3 * STRIDE));
  }
}

__device__ __forceinline__ float comp(const float4& v, int a) {
  return a == 0 ? v.x : (a == 1 ? v.y : (a == 2 ? v.z : v.w));
}

// Block weights for the adjoint's M^{-1} scaling of the neighbour values:
// product of the inverse 1D weights over the three block digits.
__device__ __forceinline__ float wprod(const float* w, int e) {
  return w[e & 3] * w[(e >> 2) & 3] * w[e >> 4];
}

// Contribution of local direction J (0..2) of the thread's block: all 16
// lines along J.  POS: c > 0 (inflow through the lower face, neighbour below).
template <int J, bool POS, bool ADJ, typename TIN, int STRIDE>
__device__ __forceinline__ void sweep(const float (&u)[64], float (&r)[64], float c,
                                      const Tab1D<float>& T, const TIN* nb, float wnb) {
  // traces of the 16 neighbour lines on the shared face
  float tr[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) tr[i] = 0.f;
#pragma unroll
  for (int cc = 0; cc < 4; ++cc)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float4 v = nb_row<TIN, STRIDE>(nb, b, cc);
      if (ADJ) {
        v.x *= wprod(T.winv, 0 + 4 * b + 16 * cc);
        v.y *= wprod(T.winv, 1 + 4 * b + 16 * cc);
        v.z *= wprod(T.winv, 2 + 4 * b + 16 * cc);
        v.w *= wprod(T.winv, 3 + 4 * b + 16 * cc);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        // element (a, b, cc): line and position along J
        const int l1 = J == 0 ? b : a;
        const int l2 = J == 2 ? b : cc;
        const int pp = J == 0 ? a : (J == 1 ? b : cc);
        const float lw = POS ? T.lp[pp] : T.lm[pp];
        tr[l1 + 4 * l2] = fmaf(lw, comp(v, a), tr[l1 + 4 * l2]);
      }
    }
#pragma unroll
  for (int l2 = 0; l2 < 4; ++l2)
#pragma unroll
    for (int l1 = 0; l1 < 4; ++l1) {
      const float t = (ADJ ? wnb : 1.f) * tr[l1 + 4 * l2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float acc = (POS ? T.Lm[q] : -T.Lp[q]) * t;
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
          acc = fmaf(POS ? T.Gp[q * 4 + pp] : T.Gn[q * 4 + pp], u[eidx<J>(l1, l2, pp)], acc);
        r[eidx<J>(l1, l2, q)] = fmaf(c, acc, r[eidx<J>(l1, l2, q)]);
      }
    }
}

template <int J, bool ADJ, typename TIN, int STRIDE>
__device__ __forceinline__ void direction(const KParams& p, long long cell, int gdim, int off,
                                          const float (&u)[64], float (&r)[64], float c,
                                          const Tab1D<float>& T, float wnb) {
  if (ADJ) c = -c;
  if (c == 0.f) return;
  const TIN* src = static_cast<const TIN*>(p.src);
  if (c > 0.f) {
    const long long nb = neighbour_cell(p, cell, gdim, -1);
    sweep<J, true, ADJ, TIN, STRIDE>(u, r, c, T, src + nb * 4096 + off, wnb);
  } else {
    const long long nb = neighbour_cell(p, cell, gdim, 1);
    sweep<J, false, ADJ, TIN, STRIDE>(u, r, c, T, src + nb * 4096 + off, wnb);
  }
}

template <typename TIN, typename TW, int CPB, bool ADJ>
__global__ void __launch_bounds__(64 * CPB) k_cell6d4(const KParams p) {
  extern __shared__ __align__(16) float sm6[];
  const int grp = threadIdx.x >> 6;
  const int t = threadIdx.x & 63;
  float* su = sm6 + grp * 2 * kCellSmem;
  float* sr = su + kCellSmem;
  const Tab1D<float>& T = p.t32;
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  // thread-constant weight factors of the adjoint scaling
  const float wv_inv = ADJ ? wprod(T.winv, t) : 1.f;   // phase X: v node t
  int bad = 0;

  for (long long cell = static_cast<long long>(blockIdx.x) * CPB + grp; cell < p.ncells;
       cell += static_cast<long long>(gridDim.x) * CPB) {
    // ---- step 1: gather the cell into shared memory (coalesced, padded)
    const TIN* cs = src + cell * 4096;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int f = i * 64 + t;                 // float4 index within the cell
      const int m = f >> 4, ch = f & 15;        // block (v node) and chunk
      float4 v = Ld<TIN>::ld4(cs + 4 * f);
      if (ADJ) {
        const float wm = wprod(T.winv, m);
        v.x *= wm * wprod(T.winv, 4 * ch + 0);
        v.y *= wm * wprod(T.winv, 4 * ch + 1);
        v.z *= wm * wprod(T.winv, 4 * ch + 2);
        v.w *= wm * wprod(T.winv, 4 * ch + 3);
      }
      *reinterpret_cast<float4*>(su + m * kPad + 4 * ch) = v;
    }
    group_sync(grp);

    // ---- phase X: directions x1, x2, x3 on the x-block of v node t
    float u[64], r[64];
    {
      const float* ub = su + t * kPad;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(ub + 4 * i);
        u[4 * i] = v.x;
        u[4 * i + 1] = v.y;
        u[4 * i + 2] = v.z;
        u[4 * i + 3] = v.w;
      }
#pragma unroll
      for (int e = 0; e < 64; ++e) r[e] = 0.f;
      const long long cv = cell / p.ncx;
      const float* ct = static_cast<const float*>(p.cx_tab) + (cv * 64 + t) * 3;
      const float c0 = ct[0], c1 = ct[1], c2 = ct[2];
      direction<0, ADJ, TIN, 1>(p, cell, 0, t * 64, u, r, c0, T, wv_inv);
      direction<1, ADJ, TIN, 1>(p, cell, 1, t * 64, u, r, c1, T, wv_inv);
      direction<2, ADJ, TIN, 1>(p, cell, 2, t * 64, u, r, c2, T, wv_inv);
      float* rb = sr + t * kPad;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        *reinterpret_cast<float4*>(rb + 4 * i) =
            make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
    }
    group_sync(grp);

    // ---- phase V: directions v1, v2, v3 on the v-block of x node t
    {
#pragma unroll
      for (int m = 0; m < 64; ++m) {
        u[m] = su[m * kPad + t];
        r[m] = sr[m * kPad + t];
      }
      const long long cx = cell % p.ncx;
      const float* ct = static_cast<const float*>(p.cv_tab) + (cx * 64 + t) * 3;
      const float c3 = ct[0], c4 = ct[1], c5 = ct[2];
      const float wx_inv = ADJ ? wprod(T.winv, t) : 1.f;
      direction<0, ADJ, TIN, 64>(p, cell, 3, t, u, r, c3, T, wx_inv);
      direction<1, ADJ, TIN, 64>(p, cell, 4, t, u, r, c4, T, wx_inv);
      direction<2, ADJ, TIN, 64>(p, cell, 5, t, u, r, c5, T, wx_inv);
    }

    // ---- step 5: scatter / fused LSRK stage update (coalesced across x nodes)
    const float wx = ADJ ? wprod(T.w, t) : 1.f;
    const long long g0 = cell * 4096 + t;
    if (p.mode == 0) {
      TW* dst = static_cast<TW*>(p.dst);
#pragma unroll
      for (int m = 0; m < 64; ++m) {
        float K = r[m];
        if (ADJ) K *= wx * wprod(T.w, m);
        bad |= !isfinite(K);
        dst[g0 + 64 * m] = cvt<TW>(K);
      }
    } else {
      TW* dst = static_cast<TW*>(p.dst);
      double* uu = p.u;
      const float bf = static_cast<float>(p.b_dt);
      const float af = static_cast<float>(p.a_dt);
#pragma unroll
      for (int m = 0; m < 64; ++m) {
        float K = r[m];
        if (ADJ) K *= wx * wprod(T.w, m);
        bad |= !isfinite(K);
        const long long g = g0 + 64 * m;
        const double uo = __ldcs(uu + g);
        // one FP64 add per value; everything else in FP32 / integer arithmetic
        const double un = uo + f32_to_f64(bf * K);
        __stcs(uu + g, un);
        if constexpr (sizeof(TW) == 4) {
          dst[g] = p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(uo));
        } else {
          dst[g] = p.last_stage ? un : uo + p.a_dt * f32_to_f64(K);
        }
      }
    }
    group_sync(grp);  // shared buffers are reused by the next cell
  }
  if (bad) atomicOr(p.err, 1);
}

template <typename TIN, typename TW, int CPB, bool ADJ>
cudaError_t launch6(KParams& p, cudaStream_t s) {
  auto kern = k_cell6d4<TIN, TW, CPB, ADJ>;
  const size_t smem = static_cast<size_t>(CPB) * 2 * kCellSmem * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * CPB, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long chunks = (p.ncells + CPB - 1) / CPB;
  const long long grid = std::min<long long>(chunks, static_cast<long long>(sms) * per_sm);
  kern<<<static_cast<unsigned>(grid), 64 * CPB, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename TIN, typename TW, bool ADJ>
cudaError_t launch6_cpb(int cpb, KParams& p, cudaStream_t s) {
  switch (cpb) {
    case 1: return launch6<TIN, TW, 1, ADJ>(p, s);
    case 2: return launch6<TIN, TW, 2, ADJ>(p, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_cell_6d4(int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.dx != 3 || p.dv != 3) return cudaErrorNotSupported;
  const int cpb = cfg.cells_per_block;
  if (combo == kFFF) {
    return p.adjoint ? launch6_cpb<float, float, true>(cpb, p, s)
                     : launch6_cpb<float, float, false>(cpb, p, s);
  }
  if (combo == kFDD) {
    return p.adjoint ? launch6_cpb<double, double, true>(cpb, p, s)
                     : launch6_cpb<double, double, false>(cpb, p, s);
  }
  return cudaErrorNotSupported;
}

}  // namespace dg
