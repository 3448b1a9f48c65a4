// Specialised 4D cell kernel (dim_x = 2, dim_v = 2) with FP32 sweeps, n = 2..6.
//
// It computes the same operator as the generic kernel (Algorithm 2: per
// direction the collocated 1D operator with the upwind flux and the inverse
// mass folded in, Gp / Gn and the lifts Lm / Lp of the tables; the weak form
// and its upwind flux are those of Sec. 1.3, Eq. into:adv:ref) but keeps
// every value a thread works on in registers.
// In phase space a cell's n^4 values form an (n^2) x (n^2) matrix: a column
// is the n^2 x values at one v node (contiguous in memory, DoF index
// q = x1 + n x2 + n^2 (v1 + n v2)), a row the n^2 v values at one x node.
// The x speeds depend on the v node only and the v speeds on the x node only
// (the phase-space field of the Vlasov equation, Sec. 1.2 and Sec. 6), so
//   phase X: thread k holds column k: both x directions are line operations
//            on its registers with one speed each; the upwind neighbour's
//            column (a per-thread choice, so speeds may change sign inside a
//            cell) is read from global memory, contiguous;
//   phase V: after an exchange through shared memory, thread k holds row k
//            and the phase X residual of it; both v directions likewise,
//            then the scatter or the fused LSRK stage update.
// A block takes CPB consecutive cells, n^2 threads each.  Shared memory
// holds the cells (padded columns: conflict-free in both phases) and the
// phase X residuals.
#include "dg_cell4d.cuh"

namespace dg {
namespace {

// MODE 0: operator application (dst = K); MODE 1: fused LSRK stage.
// ADJ: the transpose L^T = M L(-a) M^{-1} (input and neighbours scaled by the
// inverse node weights, speeds negated, output scaled by the node weights).
// Every global read is issued as early as its address is known, so that a
// thread has several in flight: the upwind neighbours' columns before the
// barrier that completes the gather, their rows before the exchange, the
// FP64 state in chunks of 8 ahead of its use.  With FP32 input the gather
// and the neighbours' rows are asynchronous copies into shared memory issued
// together at the start (the rows land during phase X; sn holds the
// thread's two rows at sn[m * THREADS + tid]).
template <int N, typename TIN, typename TW, int MODE, bool ADJ>
__global__ void __launch_bounds__(Cell4<N>::THREADS, Cell4<N>::MINB) k_cell4d(const KParams p) {
  using C = Cell4<N>;
  constexpr int S = C::S, NP = C::NP, PAD = C::PAD, CPB = C::CPB;
  constexpr int NCH = (S + 7) / 8;       // chunks of the FP64 state of a row
  extern __shared__ __align__(16) float sm4[];
  float* const su = sm4;
  float* const sr = sm4 + C::BUF;
  float* const sn = sr + C::BUF;
  constexpr bool kAsync = sizeof(TIN) == 4;
  const TIN* __restrict__ src = static_cast<const TIN*>(p.src);
  const Tab1D<float>& T = p.t32;
  const unsigned ncells = static_cast<unsigned>(p.ncells);
  const unsigned cell0 = blockIdx.x * static_cast<unsigned>(CPB);
  const int nc = static_cast<int>(min(static_cast<unsigned>(CPB), ncells - cell0));
  const int c = threadIdx.x / S;
  const int k = threadIdx.x - c * S;     // the thread's column (phase X) and row (phase V)
  const bool active = c < nc;
  const unsigned cell = cell0 + static_cast<unsigned>(c);
  unsigned co[4];                        // cell coordinates, x1 fastest
  {
    unsigned rem = cell;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned nj = static_cast<unsigned>(p.ncell[j]);
      co[j] = rem % nj;
      rem /= nj;
    }
  }
  // upwind neighbour along j (periodic): below for a positive speed
  auto upwind = [&](int j, bool pos) -> unsigned {
    const unsigned st = static_cast<unsigned>(p.cstride[j]);
    const unsigned nj = static_cast<unsigned>(p.ncell[j]);
    unsigned nb;
    if (pos) nb = co[j] == 0 ? cell + (nj - 1) * st : cell - st;
    else nb = co[j] == nj - 1 ? cell - (nj - 1) * st : cell + st;
    DG_BOUND(p.err, nb, ncells);
    return nb;
  };
  // speeds: x directions at the v node k of the cell, v directions at its x node k
  float c0 = 0.f, c1 = 0.f, e0 = 0.f, e1 = 0.f;
  if (active) {
    const unsigned cx = co[0] + static_cast<unsigned>(p.ncell[0]) * co[1];
    const unsigned cv = co[2] + static_cast<unsigned>(p.ncell[2]) * co[3];
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * S + k) * 2;
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(cx) * S + k) * 2;
    c0 = ADJ ? -ctx[0] : ctx[0];
    c1 = ADJ ? -ctx[1] : ctx[1];
    e0 = ADJ ? -ctv[0] : ctv[0];
    e1 = ADJ ? -ctv[1] : ctv[1];
  }

  // gather the block's cells, each column padded to S + 1 floats
  if constexpr (kAsync) {
#pragma unroll 4
    for (int i = threadIdx.x; i < nc * NP; i += C::THREADS) {
      const int cc = i / NP, rem = i - cc * NP, t = rem / S, q = rem - t * S;
      cp_async4(su + (cc * S + t) * PAD + q, reinterpret_cast<const float*>(src) + static_cast<size_t>(cell0) * NP + i);
    }
    cp_async_commit();
    if (active) {
      const float* s32 = reinterpret_cast<const float*>(src);
      if (e0 != 0.f) {
        const float* row = s32 + static_cast<size_t>(upwind(2, e0 > 0.f)) * NP + k;
#pragma unroll
        for (int m = 0; m < S; ++m) cp_async4(sn + m * C::THREADS + threadIdx.x, row + S * m);
      }
      if (e1 != 0.f) {
        const float* row = s32 + static_cast<size_t>(upwind(3, e1 > 0.f)) * NP + k;
#pragma unroll
        for (int m = 0; m < S; ++m) cp_async4(sn + (S + m) * C::THREADS + threadIdx.x, row + S * m);
      }
    }
    cp_async_commit();
  } else {
#pragma unroll 4
    for (int i = threadIdx.x; i < nc * NP; i += C::THREADS) {
      const int cc = i / NP, rem = i - cc * NP, t = rem / S, q = rem - t * S;
      float v = cvt<float>(src[static_cast<size_t>(cell0) * NP + i]);
      if (ADJ) v *= w2<N>(T.winv, q) * w2<N>(T.winv, t);
      su[(cc * S + t) * PAD + q] = v;
    }
  }
  float u[S], r[S], nbA[S], nbB[S];
  if (active) {
    if (c0 != 0.f) load_col<N>(nbA, src, upwind(0, c0 > 0.f), k);
    if (c1 != 0.f) load_col<N>(nbB, src, upwind(1, c1 > 0.f), k);
  }
  if constexpr (kAsync) {
    cp_async_wait<1>();
    if (ADJ) {                           // each thread scales the values it copied
#pragma unroll 4
      for (int i = threadIdx.x; i < nc * NP; i += C::THREADS) {
        const int cc = i / NP, rem = i - cc * NP, t = rem / S, q = rem - t * S;
        su[(cc * S + t) * PAD + q] *= w2<N>(T.winv, q) * w2<N>(T.winv, t);
      }
    }
  }
  __syncthreads();

  // ---- phase X: column k, directions x1, x2
  if (active) {
#pragma unroll
    for (int q = 0; q < S; ++q) {
      u[q] = su[(c * S + k) * PAD + q];
      r[q] = 0.f;
    }
    if (ADJ) {                           // the neighbours' columns at the same nodes
      const float wk = w2<N>(T.winv, k);
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const float wq = w2<N>(T.winv, q) * wk;
        nbA[q] = c0 != 0.f ? nbA[q] * wq : 0.f;
        nbB[q] = c1 != 0.f ? nbB[q] * wq : 0.f;
      }
    }
    if (c0 != 0.f) dir4<N, 1>(r, u, nbA, c0, T);
    if (c1 != 0.f) dir4<N, N>(r, u, nbB, c1, T);
#pragma unroll
    for (int q = 0; q < S; ++q) sr[(c * S + k) * PAD + q] = r[q];
    if constexpr (!kAsync) {
      if (e0 != 0.f) load_row<N>(nbA, src, upwind(2, e0 > 0.f), k);
      if (e1 != 0.f) load_row<N>(nbB, src, upwind(3, e1 > 0.f), k);
    }
  }
  if constexpr (kAsync) cp_async_wait<0>();
  __syncthreads();
  if (!active) return;
  if constexpr (kAsync) {
#pragma unroll
    for (int m = 0; m < S; ++m) {
      nbA[m] = sn[m * C::THREADS + threadIdx.x];
      nbB[m] = sn[(S + m) * C::THREADS + threadIdx.x];
    }
  }

  // ---- phase V: row k, directions v1, v2
  const size_t g0 = static_cast<size_t>(cell) * NP + k;
  const double* __restrict__ uin = p.u;
  double ua[8];
  if constexpr (MODE == 1) {
#pragma unroll
    for (int m = 0; m < 8; ++m)
      if (m < S) ua[m] = __ldcs(uin + g0 + static_cast<size_t>(S) * m);
  }
#pragma unroll
  for (int m = 0; m < S; ++m) {
    u[m] = su[(c * S + m) * PAD + k];
    r[m] = sr[(c * S + m) * PAD + k];
  }
  if (ADJ) {                             // the neighbours' rows at the same nodes
    const float wk = w2<N>(T.winv, k);
#pragma unroll
    for (int m = 0; m < S; ++m) {
      const float wm = w2<N>(T.winv, m) * wk;
      nbA[m] = e0 != 0.f ? nbA[m] * wm : 0.f;
      nbB[m] = e1 != 0.f ? nbB[m] * wm : 0.f;
    }
  }
  if (e0 != 0.f) dir4<N, 1>(r, u, nbA, e0, T);
  if (e1 != 0.f) dir4<N, N>(r, u, nbB, e1, T);
  if (ADJ) {
    const float wk = w2<N>(T.w, k);
#pragma unroll
    for (int m = 0; m < S; ++m) r[m] *= w2<N>(T.w, m) * wk;
  }

  // ---- scatter / fused LSRK stage update (consecutive threads, consecutive DoFs)
  TW* __restrict__ dst = static_cast<TW*>(p.dst);
  float nanacc = 0.f;
  if constexpr (MODE == 0) {
#pragma unroll
    for (int m = 0; m < S; ++m) {
      nanacc = fmaf(r[m], 0.f, nanacc);    // stays 0 unless a value is Inf or NaN
      __stcs(dst + g0 + static_cast<size_t>(S) * m, cvt<TW>(r[m]));
    }
  } else {
    double* __restrict__ uout = p.u;
    const float bf = static_cast<float>(p.b_dt), af = static_cast<float>(p.a_dt);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      double ub[8];
      if (ch + 1 < NCH) {                // the next chunk's loads go out first
#pragma unroll
        for (int m = 0; m < 8; ++m)
          if (8 * (ch + 1) + m < S) ub[m] = __ldcs(uin + g0 + static_cast<size_t>(S) * (8 * (ch + 1) + m));
      }
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
        const int m = 8 * ch + mm;
        if (m >= S) break;
        const size_t g = g0 + static_cast<size_t>(S) * m;
        const float K = r[m];
        nanacc = fmaf(K, 0.f, nanacc);
        const double un = ua[mm] + f32_to_f64_finite(bf * K);
        __stcs(uout + g, un);
        if constexpr (sizeof(TW) == 4)
          __stcs(dst + g, p.last_stage ? f64_to_f32(un) : fmaf(af, K, f64_to_f32(ua[mm])));
        else
          __stcs(dst + g, p.last_stage ? un : ua[mm] + p.a_dt * f32_to_f64(K));
      }
      if (ch + 1 < NCH) {
#pragma unroll
        for (int m = 0; m < 8; ++m) ua[m] = ub[m];
      }
    }
  }
  if (nanacc != 0.f) atomicOr(p.err, 1);
}

template <int N, typename TIN, typename TW>
cudaError_t launch4(KParams& p, cudaStream_t s) {
  using C = Cell4<N>;
  // cell and residual buffers; FP32 input: the staged neighbour rows
  const size_t smem = (2 * static_cast<size_t>(C::BUF) + (sizeof(TIN) == 4 ? 2 * C::S * C::THREADS : 0)) * sizeof(float);
  auto kern = p.adjoint ? (p.mode == 0 ? k_cell4d<N, TIN, TW, 0, true> : k_cell4d<N, TIN, TW, 1, true>)
                        : (p.mode == 0 ? k_cell4d<N, TIN, TW, 0, false> : k_cell4d<N, TIN, TW, 1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long grid = (p.ncells + C::CPB - 1) / C::CPB;
  kern<<<static_cast<unsigned>(grid), C::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

// n = 6: the pair-split kernel (two threads per column and row, 18 values
// each; 3 cells per 224-thread block).
constexpr int kCpb6 = 3, kThreads6 = 224;

template <typename TIN, typename TW, int MODE, bool ADJ>
__global__ void __launch_bounds__(kThreads6, 2) k_cell4p(const KParams p) {
  extern __shared__ __align__(16) float sm4p[];
  float* const su = sm4p;
  float* const sr = sm4p + kCpb6 * kPS * kPad6;
  float* const sn = sm4p + 2 * kCpb6 * kPS * kPad6;   // staged neighbour values, 72 per thread
  const unsigned ncells = static_cast<unsigned>(p.ncells);
  const unsigned cell0 = blockIdx.x * static_cast<unsigned>(kCpb6);
  const int nc = static_cast<int>(min(static_cast<unsigned>(kCpb6), ncells - cell0));
  int ncell[4];
  unsigned cst[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ncell[j] = p.ncell[j];
    cst[j] = static_cast<unsigned>(p.cstride[j]);
  }
  // x speeds at v node k of the cell, v speeds at its x node k (tables)
  auto speeds = [&](unsigned, const unsigned (&co)[4], int k, float& c0, float& c1, float& e0,
                    float& e1) {
    const unsigned cx = co[0] + static_cast<unsigned>(ncell[0]) * co[1];
    const unsigned cv = co[2] + static_cast<unsigned>(ncell[2]) * co[3];
    const float* ctx = static_cast<const float*>(p.cx_tab) + (static_cast<size_t>(cv) * kPS + k) * 2;
    const float* ctv = static_cast<const float*>(p.cv_tab) + (static_cast<size_t>(cx) * kPS + k) * 2;
    c0 = ADJ ? -ctx[0] : ctx[0];
    c1 = ADJ ? -ctx[1] : ctx[1];
    e0 = ADJ ? -ctv[0] : ctv[0];
    e1 = ADJ ? -ctv[1] : ctv[1];
  };
  const bool bad = cell4p_block<TIN, TW, MODE, ADJ, kCpb6, kThreads6>(
      static_cast<const TIN*>(p.src), static_cast<TW*>(p.dst), p.u, cell0, nc, ncells, ncell, cst,
      static_cast<float>(p.b_dt), static_cast<float>(p.a_dt), p.a_dt, p.last_stage != 0, speeds, p.t32,
      su, sr, sn, p.err);
  if (bad) atomicOr(p.err, 1);
}

template <typename TIN, typename TW>
cudaError_t launch4p(KParams& p, cudaStream_t s) {
  const size_t smem = (2 * static_cast<size_t>(kCpb6) * kPS * kPad6 + 72 * kThreads6 + kSplitTab) * sizeof(float);
  auto kern = p.adjoint ? (p.mode == 0 ? k_cell4p<TIN, TW, 0, true> : k_cell4p<TIN, TW, 1, true>)
                        : (p.mode == 0 ? k_cell4p<TIN, TW, 0, false> : k_cell4p<TIN, TW, 1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const long long grid = (p.ncells + kCpb6 - 1) / kCpb6;
  kern<<<static_cast<unsigned>(grid), kThreads6, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename TIN, typename TW>
cudaError_t launch4_n(int n, KParams& p, cudaStream_t s) {
  switch (n) {
    case 2: return launch4<2, TIN, TW>(p, s);
    case 3: return launch4<3, TIN, TW>(p, s);
    case 4: return launch4<4, TIN, TW>(p, s);
    case 5: return launch4<5, TIN, TW>(p, s);
    case 6: return launch4p<TIN, TW>(p, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_cell_4d(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s) {
  if (p.dx != 2 || p.dv != 2 || cfg.variant != 2) return cudaErrorNotSupported;
  // not covered: the delta-f stage, curved meshes, partial pencils
  if (p.kref != nullptr || p.geo_c != nullptr || p.v3_n > 0) return cudaErrorNotSupported;
  if (p.ncells >= (1LL << 31)) return cudaErrorNotSupported;   // 32-bit cell indices
  if (combo == kFFF) return launch4_n<float, float>(n, p, s);
  if (combo == kFDD) return launch4_n<double, double>(n, p, s);
  return cudaErrorNotSupported;
}

}  // namespace dg
