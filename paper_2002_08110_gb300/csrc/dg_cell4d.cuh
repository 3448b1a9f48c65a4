// Building blocks of the 4D (dim_x = dim_v = 2) register kernels with FP32
// sweeps, shared by the single-problem kernel (dg_cell4d.cu) and the batched
// one (dg_batch.cu).  A cell's n^4 values are an (n^2) x (n^2) matrix: a
// column is the n^2 x values at one v node (contiguous in memory), a row the
// n^2 v values at one x node; a thread holds a column (phase X) or a row
// (phase V) in registers and does both directions of that phase on it.
#pragma once

#include "dg_convert.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

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
template <int N, int ST>
__device__ __forceinline__ void dir4(float (&r)[N * N], const float (&u)[N * N],
                                     const float (&nb)[N * N], float c, const Tab1D<float>& T) {
  const bool pos = c > 0.f;
  float G[N * N], L[N], l[N];
#pragma unroll
  for (int k = 0; k < N * N; ++k) G[k] = pos ? T.Gp[k] : T.Gn[k];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    L[q] = pos ? T.Lm[q] : -T.Lp[q];
    l[q] = pos ? T.lp[q] : T.lm[q];
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
