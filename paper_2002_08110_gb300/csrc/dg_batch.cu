// Batched execution of many independent advection problems.
//
// Every member is a constant-velocity problem (Sec. 5.1 setting) of its own
// dimension (dim_x = 2, dim_v = 1 or 2 here: d = 3 or 4), degree and mesh.
// Each LSRK(5,4) stage of all members is ONE persistent launch: blocks take
// work tiles (a member and a run of its cells) from a device queue with an
// atomic counter, and process each tile with the element-centric cell
// algorithm specialised at compile time for the tile's (d, n) (a switch over
// the supported pairs).  Tiles of one member are consecutive in the queue so
// that neighbouring cells are processed close in time (L2 reuse), and the
// queue interleaves nothing else, so load balance comes from the dynamic
// assignment.  One step = 5 stage launches (+ a counter reset), replayed from
// a CUDA graph.  The tile size (DoFs per tile) and the block size are chosen
// by dg_batch_autotune.
//
// Per member and stage: K = M^{-1} A(w_in); u += b_s dt K (FP64);
// w_out = u_old + a_s dt K (s < 4) or u_new (s = 4), exactly as the
// single-problem fused stage; stage vectors ping-pong between w0 and w1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

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
  int mode;        // 0: convert u -> w0, 1: stage
  int stage, parity;
  int nbt_off;     // byte offset of the per-cell neighbour table in shared memory
  double a, b;     // a_s (or b_4 at the last stage), b_s
  int last_stage;
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

__device__ __forceinline__ int nb_cell(const BInst& I, int cell, int j, int s) {
  const int st = I.cstride[j], nj = I.ncell[j];
  const int cj = (cell / st) % nj;
  if (s < 0) return cj == 0 ? cell + (nj - 1) * st : cell - st;
  return cj == nj - 1 ? cell - (nj - 1) * st : cell + st;
}

// One tile of member I: cells [c0, c0 + nc), d = D, n = N, compute type TC,
// stage vectors of type TW (TC == TW here).
template <int D, int N, typename TC, typename TW>
__device__ void process_tile(const BInst& I, const BParams& bp, int c0, int nc, TC* su, TC* sr,
                             int* nbt, int& bad) {
  constexpr int NP = Pow<N, D>::v;
  constexpr int NL = NP / N;
  const Tab1D<TC>& T = btab<TC>(N);
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
      nbt[c * 2 * kBatchMaxDim + 2 * j] = nb_cell(I, c0 + c, j, -1);
      nbt[c * 2 * kBatchMaxDim + 2 * j + 1] = nb_cell(I, c0 + c, j, 1);
    }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int sj = 1;
    for (int m = 0; m < j; ++m) sj *= N;
    const TC cj = speed<TC>(I, j);
    if (cj != TC(0)) {
      const bool pos = cj > TC(0);
      for (int it = threadIdx.x; it < nc * NL; it += blockDim.x) {
        const int c = it / NL;
        const int l = it - c * NL;
        const int base = (l % sj) + (l / sj) * sj * N;
        TC uu[N];
#pragma unroll
        for (int q = 0; q < N; ++q) uu[q] = su[c * NP + base + q * sj];
        const int nb = nbt[c * 2 * kBatchMaxDim + 2 * j + (pos ? 0 : 1)];
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
    __syncthreads();
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
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(bp.counter, 1);
    __syncthreads();
    const int tix = s_tile;
    __syncthreads();
    if (tix >= bp.ntiles) break;
    const Tile tl = bp.tiles[tix];
    const BInst I = bp.inst[tl.inst];
    if (bp.mode == 0) {
      TW* w0 = static_cast<TW*>(const_cast<void*>(I.w[bp.parity & 1]));
      const size_t b0 = static_cast<size_t>(tl.cell0) * I.npc;
      const size_t cnt = static_cast<size_t>(tl.ncells) * I.npc;
      for (size_t i = threadIdx.x; i < cnt; i += blockDim.x)
        w0[b0 + i] = cvt<TW>(I.u[b0 + i]);
      continue;
    }
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
  }
  if (bad) atomicOr(bp.err, 1);
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
  int tile_dofs = 4096;
  int threads = 256;
  std::vector<Tile> tiles;
  size_t smem64 = 0, smem32 = 0;  // bytes of dynamic shared memory
  int nbt_off64 = 0, nbt_off32 = 0;  // offset of the neighbour table in it
  BInst* inst_d = nullptr;
  Tile* tiles_d = nullptr;
  int* counters_d = nullptr;      // one per stage (+ the conversion pass)
  int* err_d = nullptr;
  cudaStream_t capture_stream = nullptr;
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

void free_batch(dg_batch b) {
  if (!b) return;
  for (int i = 0; i < 2; ++i)
    if (b->gexec[i]) cudaGraphExecDestroy(b->gexec[i]);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  cudaFree(b->inst_d);
  cudaFree(b->tiles_d);
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

// Tiles of `tile_dofs` DoFs (whole cells, at least one), member by member.
dg_status build_tiles(dg_batch b) {
  b->tiles.clear();
  size_t max_cells_dofs = 0, max_cells = 0;
  for (int m = 0; m < b->count; ++m) {
    const int npc = static_cast<int>(b->npc[m]);
    const int per = std::max(1, b->tile_dofs / npc);
    const int nc = b->inst[m].ncells;
    for (int c = 0; c < nc; c += per) {
      Tile t{m, c, std::min(per, nc - c)};
      b->tiles.push_back(t);
    }
    max_cells_dofs = std::max(max_cells_dofs, static_cast<size_t>(per) * npc);
    max_cells = std::max(max_cells, static_cast<size_t>(per));
  }
  // the tile's values and residuals, then its cells' neighbour table
  b->nbt_off64 = static_cast<int>(max_cells_dofs * 2 * sizeof(double));
  b->nbt_off32 = static_cast<int>(max_cells_dofs * 2 * sizeof(float));
  const size_t nbt_bytes = max_cells * 2 * kBatchMaxDim * sizeof(int);
  b->smem64 = b->nbt_off64 + nbt_bytes;
  b->smem32 = b->nbt_off32 + nbt_bytes;
  if (b->smem64 > 200 * 1024) b->smem64 = 0;  // FP64 not possible at this tile size
  if (b->smem32 > 200 * 1024) return report(DG_ERR_INVALID_ARG, "tile too large for shared memory");
  cudaFree(b->tiles_d);
  b->tiles_d = nullptr;
  cudaError_t e = cudaMalloc(&b->tiles_d, b->tiles.size() * sizeof(Tile));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->tiles_d, b->tiles.data(), b->tiles.size() * sizeof(Tile),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
  drop_graphs(b);
  return DG_OK;
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
  const int grid = std::max(1, sms * std::max(1, per_sm));
  kern<<<grid, b->threads, smem, s>>>(bp);
  return cudaGetLastError();
}

dg_status enqueue_step(dg_batch b, int prec, int parity, cudaStream_t s) {
  double A[4], B[5];
  lsrk_coefficients(A, B);
  cudaError_t e = cudaMemsetAsync(b->counters_d, 0, 5 * sizeof(int), s);
  if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
  for (int st = 0; st < 5; ++st) {
    BParams bp{};
    bp.inst = b->inst_d;
    bp.tiles = b->tiles_d;
    bp.ntiles = static_cast<int>(b->tiles.size());
    bp.counter = b->counters_d + st;
    bp.err = b->err_d;
    bp.mode = 1;
    bp.stage = st;
    bp.parity = parity;
    bp.a = st < 4 ? A[st] : B[4];
    bp.b = B[st];
    bp.last_stage = st == 4;
    bp.nbt_off = prec == DG_PREC_FP64 ? b->nbt_off64 : b->nbt_off32;
    e = prec == DG_PREC_FP64 ? launch_batch<double, double>(b, bp, b->smem64, s)
                             : launch_batch<float, float>(b, bp, b->smem32, s);
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
      (e = cudaMalloc(&b->counters_d, 8 * sizeof(int))) != cudaSuccess ||
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
  if (tiles) *tiles = static_cast<long long>(b->tiles.size());
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
  if (prec == DG_PREC_FP64 && b->smem64 == 0)
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
  // w0 = u for every member (one persistent pass over all tiles)
  {
    BParams bp{};
    bp.inst = b->inst_d;
    bp.tiles = b->tiles_d;
    bp.ntiles = static_cast<int>(b->tiles.size());
    bp.counter = b->counters_d + 5;
    bp.err = b->err_d;
    bp.mode = 0;
    bp.parity = 0;
    if ((e = cudaMemsetAsync(b->counters_d + 5, 0, sizeof(int), s)) != cudaSuccess)
      return report(DG_ERR_CUDA, cudaGetErrorString(e));
    e = prec == DG_PREC_FP64 ? launch_batch<double, double>(b, bp, 0, s)
                             : launch_batch<float, float>(b, bp, 0, s);
    if (e != cudaSuccess) return report(DG_ERR_CUDA, cudaGetErrorString(e));
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
  if (flag & 1) return report(DG_ERR_NONFINITE, "a batched kernel produced a non-finite value");
  return DG_OK;
}

dg_status dg_batch_set_launch(dg_batch b, int tile_dofs, int threads) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  if (tile_dofs < 64 || tile_dofs > (1 << 16) || threads < 32 || threads > 512 || threads % 32)
    return report(DG_ERR_INVALID_ARG, "tile_dofs in [64, 65536], threads a multiple of 32 <= 512");
  const int old_tile = b->tile_dofs, old_threads = b->threads;
  b->tile_dofs = tile_dofs;
  b->threads = threads;
  dg_status st = build_tiles(b);
  if (st != DG_OK) {
    b->tile_dofs = old_tile;
    b->threads = old_threads;
    build_tiles(b);
  }
  return st;
}

dg_status dg_batch_autotune(dg_batch b, double* const* u, void* const* w0, void* const* w1,
                            const double* dt, int prec, void* stream, double* best_ms) {
  if (b == nullptr) return report(DG_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tiles_c[] = {1024, 2048, 4096, 8192};
  const int threads_c[] = {128, 256, 512};
  double best = 1e300;
  int bt = b->tile_dofs, bth = b->threads;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time two steps per candidate (after one untimed step that captures its
  // graphs) on the caller's buffers: their contents are advanced, as the
  // header states
  for (int tdofs : tiles_c)
    for (int th : threads_c) {
      if (dg_batch_set_launch(b, tdofs, th) != DG_OK) continue;
      if (prec == DG_PREC_FP64 && b->smem64 == 0) continue;
      if (dg_batch_rk_step(b, u, w0, w1, dt, 1, prec, stream) != DG_OK) continue;  // warm-up / capture
      cudaEventRecord(e0, s);
      if (dg_batch_rk_step(b, u, w0, w1, dt, 2, prec, stream) != DG_OK) continue;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 2 < best) {
        best = ms / 2;
        bt = tdofs;
        bth = th;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dg_status st = dg_batch_set_launch(b, bt, bth);
  if (best_ms) *best_ms = best;
  return st;
}

}  // extern "C"
