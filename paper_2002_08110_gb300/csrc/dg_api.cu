// C ABI of the DG advection library: handle set-up, validation, dispatch of
// the cell kernels, fused LSRK stages replayed from CUDA graphs, integrals,
// error latch and the launch-configuration autotuner.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.h"

using namespace dg;

namespace {

thread_local std::string g_err;

dg_status fail(dg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

dg_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(DG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(DG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// LSRK(5,4), 2R form: Kennedy, Carpenter & Lewis (2000), the scheme cited in
// Sec. 5.4 of the paper.
const double kRkA[4] = {970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
                        2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0};
const double kRkB[5] = {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
                        -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
                        5198255086312.0 / 14908931495163.0};

int combo_of(int prec) {
  switch (prec) {
    case DG_PREC_FP64: return kDDD;
    case DG_PREC_FP32: return kFFF;
    case DG_PREC_MIXED: return kFDD;
    default: return -1;
  }
}

size_t elem_bytes(int prec) { return prec == DG_PREC_FP32 ? 4 : 8; }
size_t compute_bytes(int prec) { return prec == DG_PREC_FP64 ? 8 : 4; }

int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cached <= 0)
      cached = 1;
  }
  return cached;
}

bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bbytes && y < x + abytes;
}

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  return ranges_overlap(a, bytes, b, bytes);
}

dg_status check_vec(const void* ptr, const char* name) {
  if (ptr == nullptr) return fail(DG_ERR_INVALID_ARG, "%s is NULL", name);
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0)
    return fail(DG_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  return DG_OK;
}

// Captured LSRK graphs hold kernel choices and scratch pointers: dropped
// whenever either changes.
void drop_graphs(dg_ctx* h) {
  for (int i = 0; i < dg_ctx::kGraphSlots; ++i)
    if (h->gexec[i]) {
      cudaGraphExecDestroy(h->gexec[i]);
      h->gexec[i] = nullptr;
    }
}

KParams base_params(const dg_ctx* h, int prec) {
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.dx = h->dx;
  p.dv = h->dv;
  for (int j = 0; j < kMaxDim; ++j) {
    p.ncell[j] = j < h->d ? h->ncell[j] : 1;
    p.cstride[j] = j < h->d ? h->cstride[j] : 1;
  }
  p.ncells = h->ncells;
  p.ncx = h->ncx;
  const LaunchCfg& c = h->cfg[prec];
  for (int j = 0; j < kMaxDim; ++j) p.order[j] = c.order[j];
  p.cells_per_block = c.cells_per_block;
  const bool f = prec != DG_PREC_FP64;
  p.cx_tab = f ? static_cast<const void*>(h->cx_d32) : static_cast<const void*>(h->cx_d64);
  p.cv_tab = f ? static_cast<const void*>(h->cv_d32) : static_cast<const void*>(h->cv_d64);
  p.scratch = h->scratch;
  p.err = h->err_d;
  p.work = h->work_d;
  p.t64 = h->tables.t64;
  p.t32 = h->tables.t32;
  p.tab = h->basis == DG_BASIS_GLL ? 1 : 0;
  p.kref = h->kref_active;
  if (h->curved) {
    const bool f64 = prec == DG_PREC_FP64;   // compute type of the sweeps
    p.geo_c = f64 ? static_cast<const void*>(h->geo_c64) : static_cast<const void*>(h->geo_c32);
    p.geo_f = f64 ? static_cast<const void*>(h->geo_f64) : static_cast<const void*>(h->geo_f32);
    p.ax_tab = f64 ? static_cast<const void*>(h->ax64) : static_cast<const void*>(h->ax32);
  }
  return p;
}

// FP32 compute with FP64 vectors on the 128-thread 6D kernel (Gauss-Legendre):
// the input is first rounded to FP32 into the handle's in32 buffer and the
// kernel takes its cells from there with tensor copies (the FP64-input
// kernel loads them with plain loads, which do not overlap the sweeps).
bool use_in32(const dg_ctx* h, int prec) {
  return prec == DG_PREC_MIXED && h->d == 6 && h->dx == 3 && h->n == 4 && h->uniform_sides &&
         !h->curved && h->cfg[prec].variant == 2 && h->basis != DG_BASIS_GLL &&
         h->kref_active == nullptr && h->ncells * 64 < (1LL << 31);
}

// Scratch needed by the global-memory variant of the generic kernel, and the
// FP32 input copy of use_in32 (both allocated outside any graph capture).
dg_status ensure_scratch(dg_ctx* h, int prec) {
  if (use_in32(h, prec) && h->in32 == nullptr) {
    cudaError_t e = cudaMalloc(&h->in32, static_cast<size_t>(h->n_dofs) * sizeof(float));
    if (e != cudaSuccess) {
      h->in32 = nullptr;
      return cuda_fail(e, "FP32 input buffer");
    }
  }

  const int combo = combo_of(prec);
  if (generic_smem_bytes(h->d, h->n, combo, 1) != 0) return DG_OK;
  const int blocks = generic_grid_blocks(h->d, h->n, h->ncells, 1, h->cfg[prec].threads);
  const size_t need = static_cast<size_t>(blocks) * generic_scratch_elems(h->d, h->n) *
                      compute_bytes(prec);
  if (h->scratch_bytes >= need) return DG_OK;
  // captured graphs hold the old scratch pointer
  drop_graphs(h);
  if (h->scratch) cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&h->scratch, need);
  if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
  h->scratch_bytes = need;
  return DG_OK;
}

cudaError_t launch_generic_any(const dg_ctx* h, int combo, KParams& p, const LaunchCfg& cfg,
                               cudaStream_t s) {
  if (p.v3_n > 0) return cudaErrorInvalidValue;     // the generic kernels walk whole cells only
  switch (h->d) {
    case 2: return launch_cell_d2(h->n, combo, p, cfg, s);
    case 3: return launch_cell_d3(h->n, combo, p, cfg, s);
    case 4: return launch_cell_d4(h->n, combo, p, cfg, s);
    case 5: return launch_cell_d5(h->n, combo, p, cfg, s);
    case 6: return launch_cell_d6(h->n, combo, p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cell(const dg_ctx* h, int combo, KParams& p, const LaunchCfg& cfg,
                        cudaStream_t s) {
  if (cfg.variant == 2 && h->d == 5 && h->dx == 2 && !h->curved) {
    cudaError_t e = launch_cell_5d(h->n, combo, p, cfg, s);
    if (e != cudaErrorNotSupported) return e;
  }
  // the negated-field forward operator: the generic and the 5D kernels only
  if (p.negate) return launch_generic_any(h, combo, p, cfg, s);
  if (cfg.variant >= 1 && h->d == 6 && h->n == 4 && h->uniform_sides && !h->curved) {
    cudaError_t e = launch_cell_6d4(combo, p, cfg, s);
    if (e != cudaErrorNotSupported) return e;
  }
  if (cfg.variant == 2 && h->d == 4 && h->dx == 2 && !h->curved) {
    cudaError_t e = launch_cell_4d(h->n, combo, p, cfg, s);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_generic_any(h, combo, p, cfg, s);
}

// Do the adjoint steps for this precision run as forward steps of the
// negated field on weight-scaled states?  Yes where the kernel that runs has
// no transpose of its own: the generic kernel and the 5D kernel (the 6D and
// 4D kernels apply the node weights inside).
bool generic_runs(const dg_ctx* h, int prec) {
  if (prec == DG_PREC_FP64 || h->curved) return true;
  const LaunchCfg& c = h->cfg[prec];
  if (c.variant >= 1 && h->d == 6 && h->n == 4 && h->uniform_sides && h->ncells < (1LL << 31))
    return false;
  if (c.variant == 2 && h->d == 4 && h->dx == 2 && h->ncells < (1LL << 31)) return false;
  return true;
}

// Node weights W_q = prod_i w_{q_i} of the handle's basis and their inverses
// (device, 2 npc doubles), for the adjoint steps of the generic path.
dg_status ensure_wnode(dg_ctx* h) {
  if (h->wnode_d) return DG_OK;
  std::vector<double> w(2 * static_cast<size_t>(h->npc));
  for (int q = 0; q < h->npc; ++q) {
    double f = 1.0;
    int r = q;
    for (int j = 0; j < h->d; ++j) {
      f *= h->tables.t64.w[r % h->n];
      r /= h->n;
    }
    w[q] = f;
    w[h->npc + q] = 1.0 / f;
  }
  cudaError_t e = cudaMalloc(&h->wnode_d, w.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(h->wnode_d, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(h->wnode_d);
    h->wnode_d = nullptr;
    return cuda_fail(e, "node weights");
  }
  return DG_OK;
}

// DG_BASIS_GLL_GAUSS: four FP64 temporaries of n_dofs values (two vectors
// at the Gauss points, the state there, and one for multi-pass basis
// changes of cells too large for shared memory), allocated on first use.
dg_status ensure_bc_tmp(dg_ctx* h) {
  for (int i = 0; i < 4; ++i) {
    if (h->bc_tmp[i]) continue;
    cudaError_t e = cudaMalloc(&h->bc_tmp[i], static_cast<size_t>(h->n_dofs) * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "basis-change temporaries");
  }
  return DG_OK;
}

// y = M x on every cell, M = V (which 0), V^{-1} (1), V^T (2) or V^{-T} (3)
// in every direction; x and y FP32 when the flags say so.
dg_status change_basis(dg_ctx* h, int which, const void* x, int xf, void* y, int yf,
                       cudaStream_t s) {
  BasisMat M;
  std::memset(&M, 0, sizeof(M));
  for (int q = 0; q < h->n; ++q)
    for (int i = 0; i < h->n; ++i) {
      const int r = which >= 2 ? i : q, c = which >= 2 ? q : i;   // transposes read (i, q)
      M.m[q * kMaxN + i] = (which % 2 == 0) ? h->tables.V[r][c] : h->tables.Vinv[r][c];
    }
  cudaError_t e = launch_basis_change(x, xf, y, yf, h->bc_tmp[3], h->ncells, h->d, h->n, M, s);
  if (e == cudaErrorNotSupported)
    return fail(DG_ERR_UNSUPPORTED, "FP32 basis change of cells this large");
  if (e != cudaSuccess) return cuda_fail(e, "basis change");
  return DG_OK;
}

dg_status apply_core(dg_handle h, const void* src, void* dst, int prec, cudaStream_t s,
                     int adjoint) {
  dg_status st;
  if ((st = ensure_scratch(h, prec)) != DG_OK) return st;
  KParams p = base_params(h, prec);
  p.src = src;
  p.dst = dst;
  p.mode = 0;
  p.adjoint = adjoint;
  cudaError_t e;
  if (use_in32(h, prec) && h->in32 != nullptr) {
    if ((e = launch_convert(static_cast<const double*>(src), h->in32, 1, h->n_dofs, s)) != cudaSuccess)
      return cuda_fail(e, "FP32 input copy");
    p.src32 = h->in32;
  }
  e = launch_cell(h, combo_of(prec), p, h->cfg[prec], s);
  if (e != cudaSuccess) return cuda_fail(e, "cell kernel launch");
  return DG_OK;
}

dg_status do_apply(dg_handle h, const void* src, void* dst, int prec, void* stream, int adjoint) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (adjoint && h->curved)
    return fail(DG_ERR_UNSUPPORTED, "the transposed operator is not available on a curved mesh");
  const int combo = combo_of(prec);
  if (combo < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  dg_status st;
  if ((st = check_vec(src, "src")) != DG_OK) return st;
  if ((st = check_vec(dst, "dst")) != DG_OK) return st;
  const size_t bytes = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  if (ranges_overlap(src, dst, bytes)) return fail(DG_ERR_INVALID_ARG, "src and dst overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->basis != DG_BASIS_GLL_GAUSS) return apply_core(h, src, dst, prec, s, adjoint);
  // L = V^{-1} L_GL V;  L^T = V^T L_GL^T V^{-T}
  if ((st = ensure_bc_tmp(h)) != DG_OK) return st;
  const int f = prec == DG_PREC_FP32;
  if ((st = change_basis(h, adjoint ? 3 : 0, src, f, h->bc_tmp[0], f, s)) != DG_OK ||
      (st = apply_core(h, h->bc_tmp[0], h->bc_tmp[1], prec, s, adjoint)) != DG_OK ||
      (st = change_basis(h, adjoint ? 2 : 1, h->bc_tmp[1], f, dst, f, s)) != DG_OK)
    return st;
  return DG_OK;
}

dg_status enqueue_stage(dg_handle h, const void* w_in, void* w_out, double* u, int stage, double dt,
                        int prec, int adjoint, cudaStream_t s) {
  KParams p = base_params(h, prec);
  p.src = w_in;
  p.dst = w_out;
  p.u = u;
  p.mode = 1;
  p.adjoint = adjoint == 1 ? 1 : 0;
  p.negate = adjoint == 2 ? 1 : 0;     // 2: L(-a) on weight-scaled states (rk_step_core)
  p.last_stage = stage == 4;
  p.a_dt = stage < 4 ? kRkA[stage] * dt : kRkB[4] * dt;
  p.b_dt = kRkB[stage] * dt;
  cudaError_t e;
  if (use_in32(h, prec) && h->in32 != nullptr) {
    if ((e = launch_convert(static_cast<const double*>(w_in), h->in32, 1, h->n_dofs, s)) != cudaSuccess)
      return cuda_fail(e, "FP32 input copy");
    p.src32 = h->in32;
  }
  e = launch_cell(h, combo_of(prec), p, h->cfg[prec], s);
  if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
  return DG_OK;
}

// One LSRK step: stage s reads w[s % 2 ^ parity] and writes the other buffer.
dg_status enqueue_step(dg_handle h, double* u, void* w0, void* w1, double dt, int prec,
                       int adjoint, int parity, cudaStream_t s) {
  void* w[2] = {parity ? w1 : w0, parity ? w0 : w1};
  for (int st = 0; st < 5; ++st) {
    dg_status r = enqueue_stage(h, w[st % 2], w[(st + 1) % 2], u, st, dt, prec, adjoint, s);
    if (r != DG_OK) return r;
  }
  return DG_OK;
}

void default_cfg(dg_ctx* h) {
  for (int prec = 0; prec < 3; ++prec) {
    LaunchCfg& c = h->cfg[prec];
    c.threads = 256;
    c.variant = 0;
    for (int j = 0; j < kMaxDim; ++j) c.order[j] = j;
    int cpb = std::max(1, 2048 / h->npc);
    while (cpb > 1 && generic_smem_bytes(h->d, h->n, combo_of(prec), cpb) == 0) --cpb;
    c.cells_per_block = cpb;
    if (h->npc >= 1024) c.threads = 512;
    if (h->d == 6 && h->n == 4 && prec != DG_PREC_FP64) c.variant = 2;
    if (h->d == 4 && h->dx == 2 && prec != DG_PREC_FP64) c.variant = 2;
    if (h->d == 5 && h->dx == 2 && h->n == 4 && prec != DG_PREC_FP64) c.variant = 2;
  }
}

dg_status validate_cfg(const dg_ctx* h, int prec, const LaunchCfg& c) {
  if (c.threads < 32 || c.threads > 512 || c.threads % 32 != 0)
    return fail(DG_ERR_INVALID_ARG, "threads must be a multiple of 32 in [32, 512]");
  if (c.cells_per_block < 1 || c.cells_per_block > 4096)
    return fail(DG_ERR_INVALID_ARG, "cells_per_block out of range");
  if (c.variant < 0 || c.variant > 2) return fail(DG_ERR_INVALID_ARG, "unknown variant");
  bool seen[kMaxDim] = {false};
  for (int j = 0; j < h->d; ++j) {
    if (c.order[j] < 0 || c.order[j] >= h->d || seen[c.order[j]])
      return fail(DG_ERR_INVALID_ARG, "order must be a permutation of 0..d-1");
    seen[c.order[j]] = true;
  }
  (void)prec;
  return DG_OK;
}

void free_ctx(dg_ctx* h) {
  if (!h) return;
  for (int i = 0; i < dg_ctx::kGraphSlots; ++i)
    if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  cudaFree(h->cx_d64);
  cudaFree(h->cx_d32);
  cudaFree(h->cv_d64);
  cudaFree(h->cv_d32);
  cudaFree(h->err_d);
  cudaFree(h->work_d);
  cudaFree(h->scratch);
  cudaFree(h->wnode_d);
  cudaFree(h->partial);
  cudaFree(h->field_flags_d);
  cudaFree(h->vp_rho);
  cudaFree(h->vp_e);
  cudaFree(h->vpa);
  cudaFree(h->host_stage);
  cudaFree(h->in32);
  if (h->xfer_in) cudaStreamDestroy(h->xfer_in);
  if (h->xfer_out) cudaStreamDestroy(h->xfer_out);
  for (cudaEvent_t ev : h->xev)
    if (ev) cudaEventDestroy(ev);
  for (int i = 0; i < 4; ++i) cudaFree(h->bc_tmp[i]);
  cudaFree(h->geo_c64);
  cudaFree(h->geo_c32);
  cudaFree(h->geo_f64);
  cudaFree(h->geo_f32);
  cudaFree(h->ax64);
  cudaFree(h->ax32);
  cudaFree(h->jx_d);
  cudaFree(h->df_u);
  cudaFree(h->df_k64);
  cudaFree(h->df_k32);
  cudaFree(h->df_tmp);
  delete h;
}

cudaError_t upload32(const std::vector<float>& src, float** dst) {
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(float), cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t upload(const std::vector<double>& src, T** dst) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = static_cast<T>(src[i]);
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, tmp.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Contravariant speeds c = J^{-1} a at the x and v nodes (Sec. 3: only the
// low-dimensional parts are stored and combined on the fly, Sec. 6).
// Curved x-mesh (dg_geometry.deform): x = Phi(y), Phi_i(y) = y_i +
// delta_i L_m / (2 pi) sin(2 pi (y_m - lo_m) / L_m), m = (i+1) mod dx.  At
// every x quadrature point and every x face point: J_x = (dPhi/dy) diag(h/2),
// its determinant and |J_x| J_x^{-1} (the contravariant flux rows; Nanson's
// formula for the faces).
void jacobian_x(const dg_ctx* h, const double* y, double* det, double* R) {
  const int dx = h->dx;
  double J[3][3];
  for (int i = 0; i < dx; ++i)
    for (int m = 0; m < dx; ++m) J[i][m] = (i == m ? 1.0 : 0.0);
  for (int i = 0; i < dx; ++i) {
    const int m = (i + 1) % dx;
    const double L = h->h[m] * h->ncell[m];
    J[i][m] += h->deform[i] * std::cos(2.0 * 3.14159265358979323846 * (y[m] - h->lo[m]) / L);
  }
  for (int i = 0; i < dx; ++i)
    for (int m = 0; m < dx; ++m) J[i][m] *= h->h[m] / 2.0;
  // adjugate / determinant for dx <= 3
  double A[3][3] = {{0}};
  double dt;
  if (dx == 1) {
    dt = J[0][0];
    A[0][0] = 1.0;
  } else if (dx == 2) {
    dt = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    A[0][0] = J[1][1];
    A[0][1] = -J[0][1];
    A[1][0] = -J[1][0];
    A[1][1] = J[0][0];
  } else {
    for (int i = 0; i < 3; ++i)
      for (int m = 0; m < 3; ++m) {
        const int i1 = (m + 1) % 3, i2 = (m + 2) % 3, m1 = (i + 1) % 3, m2 = (i + 2) % 3;
        A[i][m] = J[i1][m1] * J[i2][m2] - J[i1][m2] * J[i2][m1];   // adj = cofactor^T
      }
    dt = J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
  }
  *det = dt;
  // |J| J^{-1} = sign(det) adj(J)
  const double sg = dt < 0.0 ? -1.0 : 1.0;
  for (int i = 0; i < dx; ++i)
    for (int m = 0; m < dx; ++m) R[i * dx + m] = sg * A[i][m];
  *det = std::fabs(dt);
}

dg_status compute_geometry(dg_ctx* h) {
  const int dx = h->dx, n = h->n, nqx = h->nqx;
  const double* z = h->tables.zeta;
  int nf = 1;
  for (int m = 1; m < dx; ++m) nf *= n;
  const int sc = 1 + dx * dx;
  h->geo_c_host.assign(static_cast<size_t>(h->ncx) * nqx * sc, 0.0);
  h->geo_f_host.assign(static_cast<size_t>(h->ncx) * dx * 2 * nf * dx, 0.0);
  for (long long cx = 0; cx < h->ncx; ++cx) {
    int cc[3] = {0, 0, 0};
    long long c = cx;
    for (int m = 0; m < dx; ++m) {
      cc[m] = static_cast<int>(c % h->ncell[m]);
      c /= h->ncell[m];
    }
    // cell points
    for (int q = 0; q < nqx; ++q) {
      double y[3];
      int qq = q;
      for (int m = 0; m < dx; ++m) {
        y[m] = h->lo[m] + h->h[m] * (cc[m] + (z[qq % n] + 1.0) / 2.0);
        qq /= n;
      }
      double det, R[9];
      jacobian_x(h, y, &det, R);
      if (!(det > 0.0)) return fail(DG_ERR_INVALID_ARG, "deformation folds the mesh");
      double* o = &h->geo_c_host[(static_cast<size_t>(cx) * nqx + q) * sc];
      o[0] = det;
      for (int i = 0; i < dx * dx; ++i) o[1 + i] = R[i];
    }
    // face points: direction j, side (0: xi_j = -1, 1: +1), the other digits
    for (int j = 0; j < dx; ++j)
      for (int sd = 0; sd < 2; ++sd)
        for (int f = 0; f < nf; ++f) {
          double y[3];
          int ff = f;
          for (int m = 0; m < dx; ++m) {
            double xi;
            if (m == j) {
              xi = sd ? 1.0 : -1.0;
            } else {
              xi = z[ff % n];
              ff /= n;
            }
            y[m] = h->lo[m] + h->h[m] * (cc[m] + (xi + 1.0) / 2.0);
          }
          double det, R[9];
          jacobian_x(h, y, &det, R);
          if (!(det > 0.0)) return fail(DG_ERR_INVALID_ARG, "deformation folds the mesh");
          double* o = &h->geo_f_host[((((static_cast<size_t>(cx) * dx + j) * 2 + sd) * nf) + f) * dx];
          for (int m = 0; m < dx; ++m) o[m] = R[j * dx + m];
        }
  }
  return DG_OK;
}

dg_status compute_speeds(dg_ctx* h, const double* e_nodes) {
  const int n = h->n, dx = h->dx, dv = h->dv;
  h->cx_host.assign(static_cast<size_t>(h->ncv) * h->nqv * dx, 0.0);
  h->cv_host.assign(static_cast<size_t>(h->ncx) * h->nqx * dv, 0.0);
  h->ax_host.assign(static_cast<size_t>(h->ncv) * h->nqv * dx, 0.0);
  const double* z = h->tables.zeta;
  for (long long cv = 0; cv < h->ncv; ++cv)
    for (int q = 0; q < h->nqv; ++q) {
      double a[3] = {0, 0, 0};
      if (h->field_kind == DG_FIELD_CONSTANT) {
        for (int i = 0; i < dx; ++i) a[i] = h->a_const[i];
      } else {
        long long c = cv;
        int qq = q;
        double v[3] = {0, 0, 0};
        for (int m = 0; m < dv; ++m) {
          const int j = dx + m;
          const long long cm = c % h->ncell[j];
          c /= h->ncell[j];
          v[m] = h->lo[j] + h->h[j] * (static_cast<double>(cm) + (z[qq % n] + 1.0) / 2.0);
          qq /= n;
        }
        for (int i = 0; i < dx; ++i) a[i] = v[i];
      }
      for (int i = 0; i < dx; ++i) {
        double s = 0.0;
        for (int m = 0; m < dx; ++m) s += h->Sinv[i * dx + m] * a[m];
        h->cx_host[(cv * h->nqv + q) * dx + i] = 2.0 / h->h[i] * s;
        h->ax_host[(cv * h->nqv + q) * dx + i] = a[i];   // physical, for the curved mesh
      }
    }
  for (long long cx = 0; cx < h->ncx; ++cx)
    for (int q = 0; q < h->nqx; ++q)
      for (int i = 0; i < dv; ++i) {
        double a = 0.0;
        if (h->field_kind == DG_FIELD_CONSTANT)
          a = h->a_const[dx + i];
        else if (e_nodes)
          a = e_nodes[(cx * h->nqx + q) * dv + i];
        if (!std::isfinite(a)) return fail(DG_ERR_INVALID_ARG, "E is not finite");
        h->cv_host[(cx * h->nqx + q) * dv + i] = 2.0 / h->h[dx + i] * a;
      }
  // Upwind side per cell and direction, and the FP32 tables of the FP32-sweep
  // kernels.  A cell's side is the sign of its largest speed; speeds of at
  // most 1e-12 of that (zeros of the field that fall on nodes, e.g. v = 0 on
  // a Gauss-Lobatto face node, up to rounding) carry no flux at FP32
  // precision and are stored as a zero with the cell's sign, so every node of
  // the cell reads the same side; the cell is uniform if no larger speed has
  // the other sign.  The FP64 tables keep the exact values.
  auto sides = [](const std::vector<double>& tab, std::vector<float>& f32, long long ncellsub,
                  int nq, int dims) {
    f32.assign(tab.size(), 0.f);
    bool ok = true;
    for (long long c = 0; c < ncellsub; ++c)
      for (int j = 0; j < dims; ++j) {
        double big = 0.0;
        for (int q = 0; q < nq; ++q) {
          const double v = tab[(c * nq + q) * dims + j];
          if (std::fabs(v) > std::fabs(big)) big = v;
        }
        const double thr = 1e-12 * std::fabs(big);
        for (int q = 0; q < nq; ++q) {
          const size_t r = (c * nq + q) * dims + j;
          const double v = tab[r];
          if (std::fabs(v) <= thr) {
            f32[r] = big < 0.0 ? -0.0f : 0.0f;
          } else {
            f32[r] = static_cast<float>(v);
            ok = ok && ((v > 0.0) == (big > 0.0));
          }
        }
      }
    return ok;
  };
  h->cx_uniform = sides(h->cx_host, h->cx32_host, h->ncv, h->nqv, dx);
  const bool cv_uniform = sides(h->cv_host, h->cv32_host, h->ncx, h->nqx, dv);   // always built
  h->uniform_sides = h->cx_uniform && cv_uniform;
  double sum = 0.0;
  for (int j = 0; j < h->d; ++j) {
    double mx = 0.0;
    if (j < dx) {
      for (size_t r = j; r < h->cx_host.size(); r += dx) mx = std::max(mx, std::fabs(h->cx_host[r]));
    } else {
      for (size_t r = j - dx; r < h->cv_host.size(); r += dv)
        mx = std::max(mx, std::fabs(h->cv_host[r]));
    }
    sum += 0.5 * mx;  // |c_j| / 2 = |a_j| / h_j (without shear)
  }
  h->speed_sum = sum;
  return DG_OK;
}

}  // namespace

namespace dg {

dg_status report(dg_status s, const char* msg) { return fail(s, "%s", msg); }

void lsrk_coefficients(double* a4, double* b5) {
  for (int i = 0; i < 4; ++i) a4[i] = kRkA[i];
  for (int i = 0; i < 5; ++i) b5[i] = kRkB[i];
}

size_t generic_smem_bytes(int d, int n, int combo, int cells_per_block) {
  // per cell: input and residual in the compute type, and the cell's
  // bookkeeping (x cell, v cell, two neighbours per direction)
  const size_t tb = combo == kDDD ? 8 : 4;
  const size_t b = (static_cast<size_t>(ipow(n, d)) * tb * 2 + (2 + 2 * d) * 8) * cells_per_block;
  return b <= 200 * 1024 ? b : 0;
}

long long generic_scratch_elems(int d, int n) { return ipow(n, d); }

int generic_grid_blocks(int d, int n, long long ncells, int cells_per_block, int threads) {
  (void)d;
  (void)n;
  (void)threads;
  long long want = 2LL * sm_count();
  const long long chunks = (ncells + cells_per_block - 1) / cells_per_block;
  return static_cast<int>(std::max<long long>(1, std::min(want, chunks)));
}

}  // namespace dg

extern "C" {

int dg_version(void) { return DG_ABI_VERSION; }

const char* dg_last_error(void) { return g_err.c_str(); }

dg_status dg_reference_nodes(int degree, double* nodes, double* weights) {
  if (nodes == nullptr) return fail(DG_ERR_INVALID_ARG, "nodes is NULL");
  if (degree < 0 || degree > 5) return fail(DG_ERR_INVALID_ARG, "degree must be in [0, 5]");
  double x[kMaxN], w[kMaxN];
  gauss_legendre(degree + 1, x, w);
  for (int i = 0; i <= degree; ++i) {
    nodes[i] = x[i];
    if (weights) weights[i] = w[i];
  }
  return DG_OK;
}

dg_status dg_basis_nodes(int basis, int degree, double* nodes, double* qpoints, double* qweights) {
  if (basis < DG_BASIS_GL || basis > DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_INVALID_ARG, "unknown basis %d", basis);
  if (degree < 0 || degree > 5) return fail(DG_ERR_INVALID_ARG, "degree must be in [0, 5]");
  if (basis != DG_BASIS_GL && degree < 1)
    return fail(DG_ERR_INVALID_ARG, "Gauss-Lobatto bases need degree >= 1");
  if (!basis_points(basis, degree + 1, nodes, qpoints, qweights))
    return fail(DG_ERR_INVALID_ARG, "no points for this degree");
  return DG_OK;
}

dg_status dg_create(int dim_x, int dim_v, int degree, const int* cells_x, const int* cells_v,
                    const dg_geometry* geometry, dg_handle* out) {
  if (out == nullptr) return fail(DG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (cells_x == nullptr || cells_v == nullptr || geometry == nullptr)
    return fail(DG_ERR_INVALID_ARG, "cells_x, cells_v and geometry must not be NULL");
  if (dim_x < 1 || dim_x > 3 || dim_v < 1 || dim_v > 3)
    return fail(DG_ERR_UNSUPPORTED, "dim_x and dim_v must be in [1, 3] (got %d, %d)", dim_x, dim_v);
  if (dim_x + dim_v > 6) return fail(DG_ERR_UNSUPPORTED, "d = dim_x + dim_v must be <= 6");
  if (degree < 1 || degree > 5) return fail(DG_ERR_UNSUPPORTED, "degree must be in [1, 5]");
  const dg_geometry& g = *geometry;
  if (g.field_kind != DG_FIELD_CONSTANT && g.field_kind != DG_FIELD_PHASE_SPACE)
    return fail(DG_ERR_INVALID_ARG, "unknown field_kind %d", g.field_kind);
  if (g.basis < DG_BASIS_GL || g.basis > DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_INVALID_ARG, "unknown basis %d", g.basis);
  if (g.field_kind == DG_FIELD_PHASE_SPACE && dim_v < dim_x)
    return fail(DG_ERR_UNSUPPORTED, "phase-space field needs dim_v >= dim_x");

  dg_ctx* h = new (std::nothrow) dg_ctx();
  if (!h) return fail(DG_ERR_OOM, "host allocation failed");
  h->dx = dim_x;
  h->dv = dim_v;
  h->d = dim_x + dim_v;
  h->k = degree;
  h->n = degree + 1;
  h->field_kind = g.field_kind;
  h->basis = g.basis;
  long long ncx = 1, ncv = 1;
  for (int j = 0; j < h->d; ++j) {
    const int c = j < dim_x ? cells_x[j] : cells_v[j - dim_x];
    if (c < 1 || c > (1 << 24)) {
      delete h;
      return fail(DG_ERR_INVALID_ARG, "cells per direction must be in [1, 2^24]");
    }
    h->ncell[j] = c;
    const double lo = j < dim_x ? g.x_lo[j] : g.v_lo[j - dim_x];
    const double hi = j < dim_x ? g.x_hi[j] : g.v_hi[j - dim_x];
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) {
      delete h;
      return fail(DG_ERR_INVALID_ARG, "box of direction %d is empty or not finite", j);
    }
    h->lo[j] = lo;
    h->h[j] = (hi - lo) / c;
    if (j < dim_x) ncx *= c; else ncv *= c;
  }
  h->ncx = ncx;
  h->ncv = ncv;
  h->ncells = ncx * ncv;
  long long st = 1;
  for (int j = 0; j < h->d; ++j) {
    h->cstride[j] = st;
    st *= h->ncell[j];
  }
  h->npc = ipow(h->n, h->d);
  h->nqx = ipow(h->n, dim_x);
  h->nqv = ipow(h->n, dim_v);
  if (h->ncells > (1LL << 40) / h->npc) {
    delete h;
    return fail(DG_ERR_INVALID_ARG, "mesh too large");
  }
  h->n_dofs = h->ncells * h->npc;
  // shear S (row-major), identity if all zero
  bool zero = true;
  for (int i = 0; i < 9; ++i) zero = zero && g.shear_x[i] == 0.0;
  for (int i = 0; i < dim_x; ++i)
    for (int m = 0; m < dim_x; ++m)
      h->S[i * dim_x + m] = zero ? (i == m ? 1.0 : 0.0) : g.shear_x[i * dim_x + m];
  {
    // invert the dx-by-dx shear by Gauss-Jordan elimination with pivoting
    double a[3][6];
    const int m = dim_x;
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < 2 * m; ++c) a[i][c] = c < m ? h->S[i * m + c] : (c - m == i ? 1.0 : 0.0);
    double det = 1.0;
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
      if (!(std::fabs(a[piv][c]) > 1e-300) || !std::isfinite(a[piv][c])) {
        delete h;
        return fail(DG_ERR_INVALID_ARG, "shear matrix is singular or not finite");
      }
      if (piv != c) {
        for (int k2 = 0; k2 < 2 * m; ++k2) std::swap(a[c][k2], a[piv][k2]);
        det = -det;
      }
      det *= a[c][c];
      const double inv = 1.0 / a[c][c];
      for (int k2 = 0; k2 < 2 * m; ++k2) a[c][k2] *= inv;
      for (int r = 0; r < m; ++r) {
        if (r == c) continue;
        const double f = a[r][c];
        for (int k2 = 0; k2 < 2 * m; ++k2) a[r][k2] -= f * a[c][k2];
      }
    }
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < m; ++c) h->Sinv[i * m + c] = a[i][m + c];
    double dj = std::fabs(det);
    for (int j = 0; j < h->d; ++j) dj *= h->h[j] / 2.0;
    h->detJ = dj;
  }
  for (int j = 0; j < h->d; ++j) {
    h->a_const[j] = g.a_const[j];
    if (!std::isfinite(g.a_const[j])) {
      delete h;
      return fail(DG_ERR_INVALID_ARG, "a_const is not finite");
    }
  }
  build_tables(h->n, h->basis, &h->tables);
  dg_status s = compute_speeds(h, g.e_nodes);
  if (s != DG_OK) {
    delete h;
    return s;
  }
  for (int i = 0; i < 3; ++i) {
    const double dl = i < dim_x ? g.deform[i] : 0.0;
    if (!std::isfinite(dl) || std::fabs(dl) >= 0.5) {
      delete h;
      return fail(DG_ERR_INVALID_ARG, "deform amplitudes must be finite and below 0.5 in size");
    }
    h->deform[i] = dl;
    h->curved = h->curved || dl != 0.0;
  }
  if (h->curved) {
    if (!zero) {
      delete h;
      return fail(DG_ERR_UNSUPPORTED, "a curved mesh cannot also be sheared");
    }
    if (h->basis == DG_BASIS_GLL_GAUSS) {
      delete h;
      return fail(DG_ERR_UNSUPPORTED, "the curved mesh needs a collocated basis");
    }
    if (static_cast<size_t>(h->npc) * 16 > 200 * 1024) {
      delete h;
      return fail(DG_ERR_UNSUPPORTED, "curved meshes support cells of at most 12800 DoFs");
    }
    if ((s = compute_geometry(h)) != DG_OK) {
      delete h;
      return s;
    }
    h->uniform_sides = false;   // the specialised kernels assume an affine mesh
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess ||
      (e = upload(h->cx_host, &h->cx_d64)) != cudaSuccess ||
      (e = upload32(h->cx32_host, &h->cx_d32)) != cudaSuccess ||
      (e = upload(h->cv_host, &h->cv_d64)) != cudaSuccess ||
      (e = upload32(h->cv32_host, &h->cv_d32)) != cudaSuccess ||
      (e = cudaMalloc(&h->err_d, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(h->err_d, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&h->work_d, 16 * sizeof(unsigned))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    free_ctx(h);
    return cuda_fail(e, "dg_create");
  }
  if (h->curved) {
    std::vector<double> jx(static_cast<size_t>(h->ncx) * h->nqx);
    for (size_t i = 0; i < jx.size(); ++i) jx[i] = h->geo_c_host[i * (1 + dim_x * dim_x)];
    // the kernels divide by |J_x| at every point: the device table holds its
    // reciprocal (computed here in FP64)
    std::vector<double> gc(h->geo_c_host);
    for (size_t i = 0; i < jx.size(); ++i) gc[i * (1 + dim_x * dim_x)] = 1.0 / jx[i];
    if ((e = upload(gc, &h->geo_c64)) != cudaSuccess ||
        (e = upload(gc, &h->geo_c32)) != cudaSuccess ||
        (e = upload(h->geo_f_host, &h->geo_f64)) != cudaSuccess ||
        (e = upload(h->geo_f_host, &h->geo_f32)) != cudaSuccess ||
        (e = upload(h->ax_host, &h->ax64)) != cudaSuccess ||
        (e = upload(h->ax_host, &h->ax32)) != cudaSuccess ||
        (e = upload(jx, &h->jx_d)) != cudaSuccess) {
      free_ctx(h);
      return cuda_fail(e, "dg_create");
    }
  }
  h->partial_blocks = std::min<long long>(4 * sm_count(), std::max<long long>(1, h->n_dofs / 256));
  if ((e = cudaMalloc(&h->partial, sizeof(double) * 3 * h->partial_blocks)) != cudaSuccess) {
    free_ctx(h);
    return cuda_fail(e, "dg_create");
  }
  if (h->d == 6 && h->n == 4 &&
      (e = init_cell6d_tables(h->tables.t32, h->basis == DG_BASIS_GLL ? 1 : 0)) != cudaSuccess) {
    free_ctx(h);
    return cuda_fail(e, "dg_create");
  }
  default_cfg(h);
  *out = h;
  return DG_OK;
}

dg_status dg_destroy(dg_handle h) {
  free_ctx(h);
  return DG_OK;
}

dg_status dg_info(dg_handle h, dg_info_t* info) {
  if (h == nullptr || info == nullptr) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->n_dofs = h->n_dofs;
  info->n_cells = h->ncells;
  info->n_xcells = h->ncx;
  info->n_vcells = h->ncv;
  info->dofs_per_cell = h->npc;
  info->dim_x = h->dx;
  info->dim_v = h->dv;
  info->degree = h->k;
  info->speed_sum = h->speed_sum;
  info->det_jacobian = h->detJ;
  for (int j = 0; j < h->d; ++j) info->h[j] = h->h[j];
  info->uniform_sides = h->uniform_sides ? 1 : 0;
  info->basis = h->basis;
  return DG_OK;
}

dg_status dg_node_coordinates(dg_handle h, int space, double* out) {
  if (h == nullptr || out == nullptr) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  if (space < 0 || space > 4)
    return fail(DG_ERR_INVALID_ARG,
                "space must be 0 (x nodes), 1 (v nodes), 2 or 3 (points), 4 (physical x nodes)");
  if (space == 4) {
    dg_status st = dg_node_coordinates(h, 0, out);
    if (st != DG_OK) return st;
    const int dx = h->dx;
    const long long rows = h->ncx * h->nqx;
    for (long long r = 0; r < rows; ++r) {
      double y[3], x[3];
      for (int m = 0; m < dx; ++m) y[m] = out[r * dx + m];
      for (int i = 0; i < dx; ++i) {
        double v = 0.0;
        if (h->curved) {
          const int m = (i + 1) % dx;
          const double L = h->h[m] * h->ncell[m];
          v = y[i] + h->deform[i] * L / (2.0 * 3.14159265358979323846) *
                         std::sin(2.0 * 3.14159265358979323846 * (y[m] - h->lo[m]) / L);
        } else {
          for (int m = 0; m < dx; ++m) v += h->S[i * dx + m] * y[m];
        }
        x[i] = v;
      }
      for (int m = 0; m < dx; ++m) out[r * dx + m] = x[m];
    }
    return DG_OK;
  }
  const bool xs = space % 2 == 0;
  const int dims = xs ? h->dx : h->dv;
  const int off = xs ? 0 : h->dx;
  const long long nc = xs ? h->ncx : h->ncv;
  const int nq = xs ? h->nqx : h->nqv;
  const double* z = space < 2 ? h->tables.dofz : h->tables.zeta;
  for (long long c = 0; c < nc; ++c)
    for (int q = 0; q < nq; ++q) {
      long long cc = c;
      int qq = q;
      for (int m = 0; m < dims; ++m) {
        const int j = off + m;
        const long long cm = cc % h->ncell[j];
        cc /= h->ncell[j];
        out[(c * nq + q) * dims + m] =
            h->lo[j] + h->h[j] * (static_cast<double>(cm) + (z[qq % h->n] + 1.0) / 2.0);
        qq /= h->n;
      }
    }
  return DG_OK;
}

dg_status dg_set_field(dg_handle h, const double* e_nodes, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->field_kind != DG_FIELD_PHASE_SPACE)
    return fail(DG_ERR_INVALID_ARG, "dg_set_field needs a phase-space handle");
  const bool was_uniform = h->uniform_sides;
  dg_status s = compute_speeds(h, e_nodes);
  if (s != DG_OK) return s;
  if (h->uniform_sides != was_uniform) drop_graphs(h);   // they hold the other kernel
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // synchronous with respect to the host buffers (pageable copies)
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess ||
      (e = cudaMemcpy(h->cv_d64, h->cv_host.data(), h->cv_host.size() * 8, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(h->cv_d32, h->cv32_host.data(), h->cv32_host.size() * 4,
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "dg_set_field");
  // graphs captured with the same kernel stay valid (tables are read at run time)
  return DG_OK;
}

// The specialised 6D kernel is chosen on the host from uniform_sides; a field
// set on the device records its sign pattern in field_flags_d.  Only where
// that kernel could run is the flag read back (a synchronisation).
dg_status set_field_device(dg_ctx* h, const double* e, int comps, double scale, cudaStream_t s) {
  cudaError_t err;
  if (h->field_flags_d == nullptr && (err = cudaMalloc(&h->field_flags_d, sizeof(int))) != cudaSuccess)
    return cuda_fail(err, "field flag allocation");
  double two_over_h[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < h->dv; ++j) two_over_h[j] = 2.0 / h->h[h->dx + j];
  if ((err = cudaMemsetAsync(h->field_flags_d, 0, sizeof(int), s)) != cudaSuccess ||
      (err = launch_field_speeds(e, comps, scale, h->ncx, h->nqx, h->dv, two_over_h, h->cv_d64,
                                 h->cv_d32, h->field_flags_d, h->err_d, s)) != cudaSuccess)
    return cuda_fail(err, "field speeds");
  const bool was_uniform = h->uniform_sides;
  if (h->d == 6 && h->n == 4) {
    int flags = 0;
    if ((err = cudaMemcpyAsync(&flags, h->field_flags_d, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(err, "field flag read-back");
    h->uniform_sides = h->cx_uniform && !(flags & 1);
  } else {
    h->uniform_sides = false;   // not inspected; no specialised kernel for this (d, k)
  }
  if (h->uniform_sides != was_uniform) drop_graphs(h);
  return DG_OK;
}

dg_status dg_set_field_device(dg_handle h, const double* e, int components, double scale,
                              void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->field_kind != DG_FIELD_PHASE_SPACE)
    return fail(DG_ERR_INVALID_ARG, "dg_set_field_device needs a phase-space handle");
  if (e == nullptr || reinterpret_cast<uintptr_t>(e) % 8 != 0)
    return fail(DG_ERR_INVALID_ARG, "e is NULL or not 8-byte aligned");
  if (components < 1 || components > h->dv)
    return fail(DG_ERR_INVALID_ARG, "components must be in [1, dim_v]");
  if (!std::isfinite(scale)) return fail(DG_ERR_INVALID_ARG, "scale is not finite");
  return set_field_device(h, e, components, scale, static_cast<cudaStream_t>(stream));
}

dg_status dg_poisson_periodic_1d(dg_handle h, const double* rho, double* e, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "the Poisson solve needs a collocated basis (DG_BASIS_GL or DG_BASIS_GLL)");
  if (h->dx != 1) return fail(DG_ERR_UNSUPPORTED, "the Poisson solve needs dim_x = 1");
  if (h->curved) return fail(DG_ERR_UNSUPPORTED, "the Poisson solve needs an affine mesh");
  if (rho == nullptr || e == nullptr || reinterpret_cast<uintptr_t>(rho) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(e) % 8 != 0)
    return fail(DG_ERR_INVALID_ARG, "rho and e must be non-NULL and 8-byte aligned");
  const size_t bytes = static_cast<size_t>(h->ncx) * h->n * sizeof(double);
  if (ranges_overlap(rho, e, bytes)) return fail(DG_ERR_INVALID_ARG, "rho and e overlap");
  PoissonTab t;
  std::memset(&t, 0, sizeof(t));
  for (int q = 0; q < h->n; ++q) {
    t.w[q] = h->tables.w[q];
    for (int p = 0; p < h->n; ++p) t.Iq[q * kMaxN + p] = h->tables.Iq[q][p];
  }
  const double hphys = h->S[0] * h->h[0];   // x = S y (1 x 1 shear)
  cudaError_t err = launch_poisson_1d(rho, e, h->ncx, h->n, t, hphys,
                                      static_cast<cudaStream_t>(stream));
  if (err != cudaSuccess) return cuda_fail(err, "Poisson kernel");
  return DG_OK;
}

dg_status dg_vp_rk_step(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps, int prec,
                        void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need a collocated basis (DG_BASIS_GL or DG_BASIS_GLL)");
  if (h->dx != 1) return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need dim_x = 1");
  if (h->field_kind != DG_FIELD_PHASE_SPACE)
    return fail(DG_ERR_INVALID_ARG, "Vlasov-Poisson steps need a phase-space handle");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  if (h->curved) return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need an affine mesh");
  dg_status st;
  if ((st = check_vec(u, "u")) != DG_OK || (st = check_vec(w0, "w0")) != DG_OK ||
      (st = check_vec(w1, "w1")) != DG_OK)
    return st;
  const size_t wb = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  const size_t ub = static_cast<size_t>(h->n_dofs) * 8;
  if (ranges_overlap(w0, w1, wb) || ranges_overlap(w0, wb, u, ub) ||
      ranges_overlap(w1, wb, u, ub))
    return fail(DG_ERR_INVALID_ARG, "u, w0 and w1 must not overlap");
  if (nsteps == 0) return DG_OK;
  if ((st = ensure_scratch(h, prec)) != DG_OK) return st;
  cudaError_t err;
  const size_t xb = static_cast<size_t>(h->ncx) * h->nqx * sizeof(double);
  if (h->vp_rho == nullptr && ((err = cudaMalloc(&h->vp_rho, xb)) != cudaSuccess ||
                               (err = cudaMalloc(&h->vp_e, xb)) != cudaSuccess))
    return cuda_fail(err, "Vlasov-Poisson scratch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((err = launch_convert(u, w0, prec == DG_PREC_FP32, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(err, "stage-vector initialisation");
  const int fprec = prec == DG_PREC_FP32 ? DG_PREC_FP32 : DG_PREC_FP64;
  for (int i = 0; i < nsteps; ++i) {
    void* w[2] = {i % 2 ? w1 : w0, i % 2 ? w0 : w1};
    for (int sg = 0; sg < 5; ++sg) {
      const void* w_in = w[sg % 2];
      // Sec. 6, steps 1-4 on the stage's input, then the advection stage
      if ((st = dg_charge_density(h, w_in, fprec, h->vp_rho, s)) != DG_OK) return st;
      if ((st = dg_poisson_periodic_1d(h, h->vp_rho, h->vp_e, s)) != DG_OK) return st;
      if ((st = set_field_device(h, h->vp_e, 1, -1.0, s)) != DG_OK) return st;   // a_v = -E
      if ((st = enqueue_stage(h, w_in, w[(sg + 1) % 2], u, sg, dt, prec, 0, s)) != DG_OK)
        return st;
    }
  }
  return DG_OK;
}

// The tables of the 1D Poisson kernels.
static PoissonTab poisson_tab(const dg_ctx* h) {
  PoissonTab t;
  std::memset(&t, 0, sizeof(t));
  for (int q = 0; q < h->n; ++q) {
    t.w[q] = h->tables.w[q];
    for (int p = 0; p < h->n; ++p) t.Iq[q * kMaxN + p] = h->tables.Iq[q][p];
  }
  return t;
}

// One Vlasov-Poisson stage transposed (FP64): out = J(w)^T lam with
// J(w) = L(a(w)) + B(w) P R (dg_vp_adjoint.cu); the field of w is set as the
// forward stage sets it.  g, m: x-node scratch.
static dg_status vp_stage_adjoint(dg_handle h, const double* w, const double* lam, double* out,
                                  double* g, double* m, cudaStream_t s) {
  dg_status st;
  if ((st = dg_charge_density(h, w, DG_PREC_FP64, h->vp_rho, s)) != DG_OK) return st;
  if ((st = dg_poisson_periodic_1d(h, h->vp_rho, h->vp_e, s)) != DG_OK) return st;
  if ((st = set_field_device(h, h->vp_e, 1, -1.0, s)) != DG_OK) return st;   // a_v = -E
  if ((st = apply_core(h, lam, out, DG_PREC_FP64, s, 1)) != DG_OK) return st;  // L(a)^T lam
  double detJv = 1.0;
  for (int j = h->dx; j < h->d; ++j) detJv *= h->h[j] / 2.0;
  const double hphys = h->S[0] * h->h[0];
  const PoissonTab pt = poisson_tab(h);
  cudaError_t e;
  if ((e = launch_field_adjoint(w, lam, h->cv_d64, h->ncx, h->ncv, h->npc, h->nqx, h->nqv, h->n, h->dv,
                                h->ncell[h->dx], h->tables.t64, 2.0 / h->h[h->dx], g, s)) != cudaSuccess ||
      (e = launch_poisson_1d_adjoint(g, m, h->ncx, h->n, pt, hphys, s)) != cudaSuccess ||
      (e = launch_charge_adjoint_add(out, m, h->ncx, h->ncells, h->npc, h->nqx, h->n, h->dv,
                                     h->tables.t64, detJv, s)) != cudaSuccess)
    return cuda_fail(e, "Vlasov-Poisson adjoint kernels");
  return DG_OK;
}

dg_status dg_vp_step_adjoint(dg_handle h, const double* u, double* ubar, double dt, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need a collocated basis (DG_BASIS_GL or DG_BASIS_GLL)");
  if (h->dx != 1) return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need dim_x = 1");
  if (h->field_kind != DG_FIELD_PHASE_SPACE)
    return fail(DG_ERR_INVALID_ARG, "Vlasov-Poisson steps need a phase-space handle");
  if (h->curved) return fail(DG_ERR_UNSUPPORTED, "Vlasov-Poisson steps need an affine mesh");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  dg_status st;
  if ((st = check_vec(u, "u")) != DG_OK || (st = check_vec(ubar, "ubar")) != DG_OK) return st;
  const size_t nb = static_cast<size_t>(h->n_dofs) * sizeof(double);
  if (ranges_overlap(u, ubar, nb)) return fail(DG_ERR_INVALID_ARG, "u and ubar overlap");
  if ((st = ensure_scratch(h, DG_PREC_FP64)) != DG_OK) return st;
  cudaError_t err;
  const size_t xb = static_cast<size_t>(h->ncx) * h->nqx * sizeof(double);
  if (h->vp_rho == nullptr && ((err = cudaMalloc(&h->vp_rho, xb)) != cudaSuccess ||
                               (err = cudaMalloc(&h->vp_e, xb)) != cudaSuccess))
    return cuda_fail(err, "Vlasov-Poisson scratch");
  if (h->vpa == nullptr && (err = cudaMalloc(&h->vpa, 9 * nb + 2 * xb)) != cudaSuccess) {
    h->vpa = nullptr;
    return cuda_fail(err, "adjoint Vlasov-Poisson scratch");
  }
  const long long n = h->n_dofs;
  double* W[5];                          // the stage inputs w_0 .. w_4 of the step
  for (int i = 0; i < 5; ++i) W[i] = h->vpa + i * n;
  double* uc = h->vpa + 5 * n;           // the running state of the recomputation
  double* wbar = h->vpa + 6 * n;
  double* kbar = h->vpa + 7 * n;
  double* tmp = h->vpa + 8 * n;
  double* g = h->vpa + 9 * n;
  double* m = g + h->ncx * h->nqx;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // recompute the step's stage inputs (the forward stages of dg_vp_rk_step)
  if ((err = cudaMemcpyAsync(W[0], u, nb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(uc, u, nb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_fail(err, "adjoint stage copies");
  for (int sg = 0; sg < 4; ++sg) {
    if ((st = dg_charge_density(h, W[sg], DG_PREC_FP64, h->vp_rho, s)) != DG_OK) return st;
    if ((st = dg_poisson_periodic_1d(h, h->vp_rho, h->vp_e, s)) != DG_OK) return st;
    if ((st = set_field_device(h, h->vp_e, 1, -1.0, s)) != DG_OK) return st;
    if ((st = enqueue_stage(h, W[sg], W[sg + 1], uc, sg, dt, DG_PREC_FP64, 0, s)) != DG_OK) return st;
  }
  // reverse through the stages: u_{s+1} = u_s + B_s dt K_s, w_{s+1} = u_s +
  // A_s dt K_s, K_s = F(w_s); the last stage's w output is not an output of
  // the step, so wbar starts at zero
  if ((err = cudaMemsetAsync(wbar, 0, nb, s)) != cudaSuccess) return cuda_fail(err, "adjoint init");
  for (int sg = 4; sg >= 0; --sg) {
    const double a = sg < 4 ? kRkA[sg] * dt : 0.0;
    if ((err = launch_lincomb(kbar, kRkB[sg] * dt, ubar, a, wbar, n, s)) != cudaSuccess ||
        (err = launch_axpy(ubar, 1.0, wbar, n, s)) != cudaSuccess)
      return cuda_fail(err, "adjoint stage combination");
    if ((st = vp_stage_adjoint(h, W[sg], kbar, tmp, g, m, s)) != DG_OK) return st;
    std::swap(wbar, tmp);
  }
  if ((err = launch_axpy(ubar, 1.0, wbar, n, s)) != cudaSuccess)   // w_0 = u
    return cuda_fail(err, "adjoint stage combination");
  return DG_OK;
}

dg_status dg_apply(dg_handle h, const void* src, void* dst, int prec, void* stream) {
  return do_apply(h, src, dst, prec, stream, 0);
}

dg_status dg_apply_adjoint(dg_handle h, const void* src, void* dst, int prec, void* stream) {
  return do_apply(h, src, dst, prec, stream, 1);
}

dg_status dg_rk_stage(dg_handle h, const void* w_in, void* w_out, double* u, int stage, double dt,
                      int prec, int adjoint, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  if (stage < 0 || stage > 4) return fail(DG_ERR_INVALID_ARG, "stage must be in [0, 4]");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  if (adjoint && h->curved)
    return fail(DG_ERR_UNSUPPORTED, "adjoint stages are not available on a curved mesh");
  dg_status st;
  if ((st = check_vec(w_in, "w_in")) != DG_OK || (st = check_vec(w_out, "w_out")) != DG_OK ||
      (st = check_vec(u, "u")) != DG_OK)
    return st;
  const size_t wb = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  const size_t ub = static_cast<size_t>(h->n_dofs) * 8;
  if (ranges_overlap(w_in, w_out, wb) || ranges_overlap(w_in, wb, u, ub) ||
      ranges_overlap(w_out, wb, u, ub))
    return fail(DG_ERR_INVALID_ARG, "w_in, w_out and u must not overlap");
  if ((st = ensure_scratch(h, prec)) != DG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->basis != DG_BASIS_GLL_GAUSS)
    return enqueue_stage(h, w_in, w_out, u, stage, dt, prec, adjoint ? 1 : 0, s);
  // the stage at the Gauss points: w_in and u changed there, w_out and u back
  if ((st = ensure_bc_tmp(h)) != DG_OK) return st;
  const int f = prec == DG_PREC_FP32;
  const int to = adjoint ? 3 : 0, back = adjoint ? 2 : 1;
  if ((st = change_basis(h, to, w_in, f, h->bc_tmp[0], f, s)) != DG_OK ||
      (st = change_basis(h, to, u, 0, h->bc_tmp[2], 0, s)) != DG_OK ||
      (st = enqueue_stage(h, h->bc_tmp[0], h->bc_tmp[1], h->bc_tmp[2], stage, dt, prec,
                          adjoint ? 1 : 0, s)) != DG_OK ||
      (st = change_basis(h, back, h->bc_tmp[1], f, w_out, f, s)) != DG_OK ||
      (st = change_basis(h, back, h->bc_tmp[2], 0, u, 0, s)) != DG_OK)
    return st;
  return DG_OK;
}

// Can the host-buffer stage run slab by slab?  Only the 128-thread 6D kernel
// walks part of a pencil (KParams::v3_lo/v3_n), and it needs 2+ v3 cells.
bool stage_pipelines(const dg_ctx* h, int prec) {
  return h->d == 6 && h->dx == 3 && h->n == 4 && h->uniform_sides && !h->curved &&
         prec != DG_PREC_FP64 && h->cfg[prec].variant == 2 && h->ncell[5] >= 2 &&
         h->kref_active == nullptr && h->ncells * 64 < (1LL << 31);
}

// The host-buffer stage as a pipeline over slabs of v3 cells (contiguous in
// memory): slab c's copies in, its stage kernel and its copies out run on
// three streams, so that the two copy directions and the kernels overlap.
// Kernel c reads the stage vector of slab c and of both v3-neighbour slabs
// (either may be upwind, the sign of the v3 speed varies with x), so the
// stage vector's slabs are sent in the order last, 0, 1, 2, ...
dg_status stage_host_pipelined(dg_handle h, const void* w_in, void* w_out, double* u, int stage,
                               double dt, int prec, double* du, void* dw_in, void* dw_out,
                               cudaStream_t s) {
  constexpr int kC = dg_ctx::kMaxChunks;
  cudaError_t e;
  if (!h->xfer_in && (e = cudaStreamCreateWithFlags(&h->xfer_in, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream");
  if (!h->xfer_out && (e = cudaStreamCreateWithFlags(&h->xfer_out, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream");
  for (cudaEvent_t& ev : h->xev)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "copy event");
  const int n3 = h->ncell[5];
  const int nch = std::min(n3, kC);
  int lo[kC + 1];
  for (int c = 0; c <= nch; ++c) lo[c] = static_cast<int>(static_cast<long long>(c) * n3 / nch);
  const size_t slab_dofs = static_cast<size_t>(h->cstride[5]) * h->npc;   // DoFs per v3 cell
  const size_t we = elem_bytes(prec);
  cudaEvent_t ev_start = h->xev[2 * kC], ev_done = h->xev[2 * kC + 1];
  cudaEvent_t* ev_in = h->xev;
  cudaEvent_t* ev_k = h->xev + kC;
  auto copy = [&](void* dst, const void* src, size_t elem, int c, cudaMemcpyKind kind,
                  cudaStream_t st) {
    const size_t off = static_cast<size_t>(lo[c]) * slab_dofs * elem;
    const size_t len = static_cast<size_t>(lo[c + 1] - lo[c]) * slab_dofs * elem;
    return cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, len,
                           kind, st);
  };
  if ((e = cudaEventRecord(ev_start, s)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(h->xfer_in, ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(h->xfer_out, ev_start, 0)) != cudaSuccess)
    return cuda_fail(e, "pipeline start");
  bool sent[kC] = {false};
  for (int c = 0; c < nch; ++c) {
    for (int nb : {(c + nch - 1) % nch, c, (c + 1) % nch}) {
      if (sent[nb]) continue;
      if ((e = copy(dw_in, w_in, we, nb, cudaMemcpyHostToDevice, h->xfer_in)) != cudaSuccess)
        return cuda_fail(e, "host-to-device copy");
      sent[nb] = true;
    }
    if ((e = copy(du, u, 8, c, cudaMemcpyHostToDevice, h->xfer_in)) != cudaSuccess ||
        (e = cudaEventRecord(ev_in[c], h->xfer_in)) != cudaSuccess)
      return cuda_fail(e, "host-to-device copy");
  }
  KParams p = base_params(h, prec);
  p.src = dw_in;
  p.dst = dw_out;
  p.u = du;
  p.mode = 1;
  p.last_stage = stage == 4;
  p.a_dt = stage < 4 ? kRkA[stage] * dt : kRkB[4] * dt;
  p.b_dt = kRkB[stage] * dt;
  for (int c = 0; c < nch; ++c) {
    p.v3_lo = lo[c];
    p.v3_n = lo[c + 1] - lo[c];
    if ((e = cudaStreamWaitEvent(s, ev_in[c], 0)) != cudaSuccess)
      return cuda_fail(e, "pipeline wait");
    if ((e = launch_cell(h, combo_of(prec), p, h->cfg[prec], s)) != cudaSuccess)
      return cuda_fail(e, "stage kernel launch");
    if ((e = cudaEventRecord(ev_k[c], s)) != cudaSuccess) return cuda_fail(e, "pipeline event");
  }
  for (int c = 0; c < nch; ++c) {
    if ((e = cudaStreamWaitEvent(h->xfer_out, ev_k[c], 0)) != cudaSuccess ||
        (e = copy(u, du, 8, c, cudaMemcpyDeviceToHost, h->xfer_out)) != cudaSuccess ||
        (e = copy(w_out, dw_out, we, c, cudaMemcpyDeviceToHost, h->xfer_out)) != cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
  }
  if ((e = cudaEventRecord(ev_done, h->xfer_out)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(s, ev_done, 0)) != cudaSuccess)
    return cuda_fail(e, "pipeline end");
  return DG_OK;
}

dg_status dg_rk_stage_host(dg_handle h, const void* w_in, void* w_out, double* u, int stage,
                           double dt, int prec, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "the host-buffer stage needs a collocated basis (DG_BASIS_GL or DG_BASIS_GLL)");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  if (stage < 0 || stage > 4) return fail(DG_ERR_INVALID_ARG, "stage must be in [0, 4]");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  if (w_in == nullptr || w_out == nullptr || u == nullptr)
    return fail(DG_ERR_INVALID_ARG, "w_in, w_out and u must not be NULL");
  const size_t wb = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  const size_t ub = static_cast<size_t>(h->n_dofs) * 8;
  if (ranges_overlap(w_in, w_out, wb) || ranges_overlap(w_in, wb, u, ub) ||
      ranges_overlap(w_out, wb, u, ub))
    return fail(DG_ERR_INVALID_ARG, "w_in, w_out and u must not overlap");
  dg_status st;
  if ((st = ensure_scratch(h, prec)) != DG_OK) return st;
  // staging: u, then two stage vectors, each 256-byte aligned
  auto round_up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t need = round_up(ub) + 2 * round_up(wb);
  cudaError_t e;
  if (h->host_stage_bytes < need) {
    cudaFree(h->host_stage);
    h->host_stage = nullptr;
    h->host_stage_bytes = 0;
    if ((e = cudaMalloc(&h->host_stage, need)) != cudaSuccess) return cuda_fail(e, "staging");
    h->host_stage_bytes = need;
  }
  char* base = static_cast<char*>(h->host_stage);
  double* du = reinterpret_cast<double*>(base);
  void* dw_in = base + round_up(ub);
  void* dw_out = base + round_up(ub) + round_up(wb);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (stage_pipelines(h, prec))
    return stage_host_pipelined(h, w_in, w_out, u, stage, dt, prec, du, dw_in, dw_out, s);
  if ((e = cudaMemcpyAsync(dw_in, w_in, wb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(du, u, ub, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "host-to-device copy");
  if ((st = enqueue_stage(h, dw_in, dw_out, du, stage, dt, prec, 0, s)) != DG_OK) return st;
  if ((e = cudaMemcpyAsync(u, du, ub, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w_out, dw_out, wb, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "device-to-host copy");
  return DG_OK;
}

dg_status rk_step_core(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps, int prec,
                       int adjoint, cudaStream_t s);

dg_status dg_rk_step(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps, int prec,
                     int adjoint, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  if (adjoint && h->curved)
    return fail(DG_ERR_UNSUPPORTED, "adjoint steps are not available on a curved mesh");
  dg_status st;
  if ((st = check_vec(u, "u")) != DG_OK || (st = check_vec(w0, "w0")) != DG_OK ||
      (st = check_vec(w1, "w1")) != DG_OK)
    return st;
  const size_t wb = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  const size_t ub = static_cast<size_t>(h->n_dofs) * 8;
  if (ranges_overlap(w0, w1, wb) || ranges_overlap(w0, wb, u, ub) ||
      ranges_overlap(w1, wb, u, ub))
    return fail(DG_ERR_INVALID_ARG, "u, w0 and w1 must not overlap");
  if (nsteps == 0) return DG_OK;
  adjoint = adjoint ? 1 : 0;
  if ((st = ensure_scratch(h, prec)) != DG_OK) return st;
  if (adjoint && (st = ensure_wnode(h)) != DG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->basis != DG_BASIS_GLL_GAUSS) return rk_step_core(h, u, w0, w1, dt, nsteps, prec, adjoint, s);
  // R(dt L) = V^{-1} R(dt L_GL) V: the steps run on the state at the Gauss points
  if ((st = ensure_bc_tmp(h)) != DG_OK) return st;
  if ((st = change_basis(h, adjoint ? 3 : 0, u, 0, h->bc_tmp[2], 0, s)) != DG_OK ||
      (st = rk_step_core(h, h->bc_tmp[2], w0, w1, dt, nsteps, prec, adjoint, s)) != DG_OK ||
      (st = change_basis(h, adjoint ? 2 : 1, h->bc_tmp[2], 0, u, 0, s)) != DG_OK)
    return st;
  return DG_OK;
}

dg_status rk_step_core(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps, int prec,
                       int adjoint, cudaStream_t s) {
  dg_status st;
  cudaError_t e;
  if (adjoint == 1 && generic_runs(h, prec) && h->wnode_d != nullptr) {
    // L^T = M L(-a) M^{-1} with M = |J| diag(W) on an affine mesh, so the
    // adjoint steps R(dt L^T) = W R(dt L(-a)) W^{-1}: scale the state by the
    // inverse node weights, step with the negated field (no per-value weights
    // inside the generic kernel), scale back
    if ((e = launch_scale_nodes(u, h->ncells, h->npc, h->wnode_d + h->npc, s)) != cudaSuccess)
      return cuda_fail(e, "adjoint scaling");
    if ((st = rk_step_core(h, u, w0, w1, dt, nsteps, prec, 2, s)) != DG_OK) return st;
    if ((e = launch_scale_nodes(u, h->ncells, h->npc, h->wnode_d, s)) != cudaSuccess)
      return cuda_fail(e, "adjoint scaling");
    return DG_OK;
  }
  e = launch_convert(u, w0, prec == DG_PREC_FP32, h->n_dofs, s);
  if (e != cudaSuccess) return cuda_fail(e, "stage-vector initialisation");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return cuda_fail(e, "capture query");
  if (cap != cudaStreamCaptureStatusNone) {
    for (int i = 0; i < nsteps; ++i)
      if ((st = enqueue_step(h, u, w0, w1, dt, prec, adjoint, i % 2, s)) != DG_OK) return st;
    return DG_OK;
  }
  int slot_of[2] = {-1, -1};
  for (int parity = 0; parity < 2 && parity < nsteps; ++parity) {
    dg_ctx::GraphKey key;
    key.u = u;
    key.w0 = w0;
    key.w1 = w1;
    key.dt = dt;
    key.prec = prec;
    key.adjoint = adjoint;
    key.parity = parity;
    key.kref = h->kref_active;
    int slot = -1;
    for (int i = 0; i < dg_ctx::kGraphSlots; ++i)
      if (h->gexec[i] && h->gkey[i] == key) slot = i;
    if (slot >= 0) {
      h->gused[slot] = ++h->gclock;
      slot_of[parity] = slot;
      continue;
    }
    // a free slot, else the least recently used one other than this call's
    for (int i = 0; i < dg_ctx::kGraphSlots && slot < 0; ++i)
      if (!h->gexec[i]) slot = i;
    if (slot < 0) {
      for (int i = 0; i < dg_ctx::kGraphSlots; ++i)
        if (i != slot_of[0] && (slot < 0 || h->gused[i] < h->gused[slot])) slot = i;
      cudaGraphExecDestroy(h->gexec[slot]);
      h->gexec[slot] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return cuda_fail(e, "graph capture");
    st = enqueue_step(h, u, w0, w1, dt, prec, adjoint, parity, h->capture_stream);
    e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&h->gexec[slot], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->gexec[slot] = nullptr;
      return cuda_fail(e, "graph instantiation");
    }
    h->gkey[slot] = key;
    h->gused[slot] = ++h->gclock;
    slot_of[parity] = slot;
  }
  for (int i = 0; i < nsteps; ++i)
    if ((e = cudaGraphLaunch(h->gexec[slot_of[i % 2]], s)) != cudaSuccess)
      return cuda_fail(e, "graph launch");
  return DG_OK;
}

dg_status dg_integrals(dg_handle h, const double* u, double* out, void* stream) {
  if (h == nullptr || out == nullptr) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  dg_status st;
  if ((st = check_vec(u, "u")) != DG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->basis == DG_BASIS_GLL_GAUSS) {
    // the quadrature acts on the interpolant's values at the Gauss points
    if ((st = ensure_bc_tmp(h)) != DG_OK ||
        (st = change_basis(h, 0, u, 0, h->bc_tmp[2], 0, s)) != DG_OK)
      return st;
    u = h->bc_tmp[2];
  }
  KParams p = base_params(h, DG_PREC_FP64);
  double detJv = 1.0;
  for (int j = h->dx; j < h->d; ++j) detJv *= h->h[j] / 2.0;
  cudaError_t e = launch_integrals(p, h->n, u, h->partial, h->partial_blocks,
                                   h->curved ? detJv : h->detJ, h->curved ? h->jx_d : nullptr,
                                   h->nqx, s);
  if (e != cudaSuccess) return cuda_fail(e, "integrals kernel");
  std::vector<double> host(3 * h->partial_blocks);
  if ((e = cudaMemcpyAsync(host.data(), h->partial, host.size() * 8, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "integrals readback");
  double m = 0.0, l = 0.0, x = 0.0;
  for (int b = 0; b < h->partial_blocks; ++b) {
    m += host[3 * b];
    l += host[3 * b + 1];
    x = std::max(x, host[3 * b + 2]);
  }
  out[0] = m;
  out[1] = l;
  out[2] = x;
  return DG_OK;
}

dg_status dg_charge_density(dg_handle h, const void* f, int prec, double* rho, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "the charge density needs a collocated basis (DG_BASIS_GL or DG_BASIS_GLL)");
  if (prec != DG_PREC_FP64 && prec != DG_PREC_FP32)
    return fail(DG_ERR_INVALID_ARG, "f must be FP64 (DG_PREC_FP64) or FP32 (DG_PREC_FP32)");
  dg_status st;
  if ((st = check_vec(f, "f")) != DG_OK) return st;
  if (rho == nullptr) return fail(DG_ERR_INVALID_ARG, "rho is NULL");
  if (ranges_overlap(f, static_cast<size_t>(h->n_dofs) * elem_bytes(prec), rho,
                     static_cast<size_t>(h->ncx) * h->nqx * sizeof(double)))
    return fail(DG_ERR_INVALID_ARG, "f and rho overlap");
  if (h->ncx > 0x7fffffffLL) return fail(DG_ERR_INVALID_ARG, "too many x cells");
  double detJv = 1.0;
  for (int j = h->dx; j < h->d; ++j) detJv *= h->h[j] / 2.0;
  cudaError_t e = launch_charge_density(f, prec == DG_PREC_FP32, h->ncx, h->ncv, h->npc, h->nqx,
                                        h->nqv, h->dv, h->n, h->tables.t64, detJv, rho,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "charge density kernel");
  return DG_OK;
}

dg_status dg_check(dg_handle h, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flag = 0;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
      (e = cudaMemcpy(&flag, h->err_d, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemset(h->err_d, 0, sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "dg_check");
  if (flag & 4) return fail(DG_ERR_BOUNDS, "a kernel computed an index out of its range");
  if (flag & 2) return fail(DG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
  if (flag & 1) return fail(DG_ERR_NONFINITE, "a kernel produced a non-finite value");
  return DG_OK;
}

dg_status dg_get_launch(dg_handle h, int prec, dg_launch* cfg) {
  if (h == nullptr || cfg == nullptr) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  const LaunchCfg& c = h->cfg[prec];
  cfg->threads = c.threads;
  cfg->cells_per_block = c.cells_per_block;
  for (int j = 0; j < 6; ++j) cfg->order[j] = c.order[j];
  cfg->variant = c.variant;
  return DG_OK;
}

dg_status dg_set_launch(dg_handle h, int prec, const dg_launch* cfg) {
  if (h == nullptr || cfg == nullptr) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  if (combo_of(prec) < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  LaunchCfg c;
  c.threads = cfg->threads;
  c.cells_per_block = cfg->cells_per_block;
  for (int j = 0; j < 6; ++j) c.order[j] = j < h->d ? cfg->order[j] : j;
  c.variant = cfg->variant;
  dg_status s = validate_cfg(h, prec, c);
  if (s != DG_OK) return s;
  h->cfg[prec] = c;
  drop_graphs(h);
  return DG_OK;
}

dg_status dg_autotune(dg_handle h, const void* src, void* dst, int prec, void* stream,
                      double* best_ms) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  const int combo = combo_of(prec);
  if (combo < 0) return fail(DG_ERR_INVALID_ARG, "unknown precision %d", prec);
  dg_status st;
  if ((st = check_vec(src, "src")) != DG_OK || (st = check_vec(dst, "dst")) != DG_OK) return st;
  const size_t bytes = static_cast<size_t>(h->n_dofs) * elem_bytes(prec);
  if (ranges_overlap(src, dst, bytes)) return fail(DG_ERR_INVALID_ARG, "src and dst overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // candidate set: threads x cells-per-block x sweep order x variant
  std::vector<LaunchCfg> cands;
  const int threads_c[] = {128, 256, 512};
  std::vector<int> cpbs;
  for (int c = 1; c <= 4096; c *= 2)
    if (static_cast<long long>(c) * h->npc <= 8192 &&
        (generic_smem_bytes(h->d, h->n, combo, c) != 0 || c == 1))
      cpbs.push_back(c);
  for (int variant = 0; variant < 3; ++variant) {
    const bool spec6 = h->d == 6 && h->n == 4 && prec != DG_PREC_FP64;
    const bool spec4 = h->d == 4 && h->dx == 2 && prec != DG_PREC_FP64 && !h->curved;
    const bool spec5 = h->d == 5 && h->dx == 2 && h->n == 4 && prec != DG_PREC_FP64 && !h->curved;
    if (variant >= 1 && !spec6 && !(variant == 2 && (spec4 || spec5))) continue;
    for (int rev = 0; rev < 2; ++rev)
      for (int t : threads_c)
        for (int c : cpbs) {
          LaunchCfg cfg;
          cfg.threads = t;
          cfg.cells_per_block = c;
          cfg.variant = variant;
          for (int j = 0; j < kMaxDim; ++j) cfg.order[j] = j;
          if (rev)
            for (int j = 0; j < h->d; ++j) cfg.order[j] = h->d - 1 - j;
          // the specialised kernels fix their block shape and sweep order
          if (variant >= 1 && (c > 2 || rev || t != 128)) continue;
          cands.push_back(cfg);
        }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const LaunchCfg saved = h->cfg[prec];
  double best = 1e300;
  LaunchCfg best_cfg = saved;
  for (const LaunchCfg& cfg : cands) {
    h->cfg[prec] = cfg;
    if ((st = ensure_scratch(h, prec)) != DG_OK) break;
    KParams p = base_params(h, prec);
    p.src = src;
    p.dst = dst;
    cudaError_t e = launch_cell(h, combo, p, cfg, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int reps = 3;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) {
      KParams q = base_params(h, prec);
      q.src = src;
      q.dst = dst;
      launch_cell(h, combo, q, cfg, s);
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / reps < best) {
      best = ms / reps;
      best_cfg = cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->cfg[prec] = best_cfg;
  drop_graphs(h);
  if (best_ms) *best_ms = best;
  if (st != DG_OK) return st;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// delta-f form: K = L(u_ref) + L(u - u_ref)
// ---------------------------------------------------------------------------
dg_status dg_set_reference(dg_handle h, const double* u_ref, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (h->basis == DG_BASIS_GLL_GAUSS)
    return fail(DG_ERR_UNSUPPORTED, "the delta-f form needs a collocated basis");
  dg_status st;
  if ((st = check_vec(u_ref, "u_ref")) != DG_OK) return st;
  const size_t n = static_cast<size_t>(h->n_dofs);
  cudaError_t e;
  if (h->df_u == nullptr &&
      ((e = cudaMalloc(&h->df_u, n * sizeof(double))) != cudaSuccess ||
       (e = cudaMalloc(&h->df_k64, n * sizeof(double))) != cudaSuccess ||
       (e = cudaMalloc(&h->df_k32, n * sizeof(float))) != cudaSuccess ||
       (e = cudaMalloc(&h->df_tmp, (n + 64) * sizeof(double))) != cudaSuccess))
    return cuda_fail(e, "delta-f storage");
  if (ranges_overlap(u_ref, n * 8, h->df_u, n * 8))
    return fail(DG_ERR_INVALID_ARG, "u_ref overlaps the handle's storage");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((e = cudaMemcpyAsync(h->df_u, u_ref, n * sizeof(double), cudaMemcpyDeviceToDevice, s)) !=
      cudaSuccess)
    return cuda_fail(e, "reference copy");
  if ((st = apply_core(h, h->df_u, h->df_k64, DG_PREC_FP64, s, 0)) != DG_OK) return st;
  if ((e = launch_convert(h->df_k64, h->df_k32, 1, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(e, "reference operator conversion");
  h->df_ready = true;
  return DG_OK;
}

dg_status dg_apply_df(dg_handle h, const double* src, double* dst, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (!h->df_ready) return fail(DG_ERR_INVALID_ARG, "no reference state (dg_set_reference)");
  dg_status st;
  if ((st = check_vec(src, "src")) != DG_OK || (st = check_vec(dst, "dst")) != DG_OK) return st;
  const size_t n = static_cast<size_t>(h->n_dofs);
  if (ranges_overlap(src, dst, n * 8)) return fail(DG_ERR_INVALID_ARG, "src and dst overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* t1 = reinterpret_cast<float*>(h->df_tmp);
  float* t2 = t1 + ((n + 63) / 64) * 64;          // two FP32 vectors in the FP64 scratch
  cudaError_t e;
  if ((e = launch_sub_to_f32(src, h->df_u, t1, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(e, "delta-f input");
  if ((st = apply_core(h, t1, t2, DG_PREC_FP32, s, 0)) != DG_OK) return st;
  if ((e = launch_add_f32(h->df_k64, t2, dst, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(e, "delta-f output");
  return DG_OK;
}

dg_status dg_rk_step_df(dg_handle h, double* u, float* w0, float* w1, double dt, int nsteps,
                        void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  if (!h->df_ready) return fail(DG_ERR_INVALID_ARG, "no reference state (dg_set_reference)");
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt is not finite");
  dg_status st;
  if ((st = check_vec(u, "u")) != DG_OK || (st = check_vec(w0, "w0")) != DG_OK ||
      (st = check_vec(w1, "w1")) != DG_OK)
    return st;
  const size_t wb = static_cast<size_t>(h->n_dofs) * 4, ub = static_cast<size_t>(h->n_dofs) * 8;
  if (ranges_overlap(w0, w1, wb) || ranges_overlap(w0, wb, u, ub) || ranges_overlap(w1, wb, u, ub))
    return fail(DG_ERR_INVALID_ARG, "u, w0 and w1 must not overlap");
  if (nsteps == 0) return DG_OK;
  if ((st = ensure_scratch(h, DG_PREC_FP32)) != DG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // the steps advance du = u - u_ref with K = K_ref + L(dw)
  if ((e = launch_axpy(u, -1.0, h->df_u, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(e, "delta-f state");
  h->kref_active = h->df_k32;
  st = rk_step_core(h, u, w0, w1, dt, nsteps, DG_PREC_FP32, 0, s);
  h->kref_active = nullptr;
  if (st != DG_OK) return st;
  if ((e = launch_axpy(u, 1.0, h->df_u, h->n_dofs, s)) != cudaSuccess)
    return cuda_fail(e, "delta-f state");
  return DG_OK;
}

dg_status dg_selftest_wait(dg_handle h, void* stream) {
  if (h == nullptr) return fail(DG_ERR_INVALID_ARG, "handle is NULL");
  cudaError_t e = launch_wait_probe(h->err_d, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  return DG_OK;
}
