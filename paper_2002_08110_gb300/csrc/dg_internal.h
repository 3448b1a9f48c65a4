// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dg.h"

// Bounds-check build (compiled with -DDG_BOUNDS_CHECK, library
// libdg_bounds.so): every computed cell, neighbour, tile and slab index is
// checked against its range before it is used; a violation latches bit 2 (4)
// of the device error word, which dg_check reports as DG_ERR_BOUNDS, and the
// index is replaced by 0 so that nothing traps and nothing is read or
// written out of range.  In the normal build the check compiles to nothing.
#ifdef DG_BOUNDS_CHECK
#define DG_BOUND(err, idx, n)                                                          \
  do {                                                                                 \
    if (static_cast<unsigned long long>(idx) >= static_cast<unsigned long long>(n)) { \
      atomicOr((err), 4);                                                              \
      (idx) = 0;                                                                       \
    }                                                                                  \
  } while (0)
#else
#define DG_BOUND(err, idx, n) \
  do {                        \
  } while (0)
#endif

namespace dg {

constexpr int kMaxDim = 6;
constexpr int kMaxN = 6;

// 1D tables of the collocated Gauss-Legendre element, precomputed in FP64 on
// the host (Sec. 2.3, Sec. 2.5).  With nodal basis phi_i at the GL points
// zeta_i, weights w_i, D[p][i] = phi_i'(zeta_p), and face values
// l_i(+-1) = phi_i(+-1), the collocated weak form of one direction j of
// Algorithm 2 (cell term, both faces, inverse mass) reduces, for a line of
// n values u along j with contravariant speed c (constant along the line),
// to
//   c > 0:  du_q = c ( sum_p Gp[q][p] u_p + Lm[q] t ),  t = sum_p lp[p] u^-_p
//   c < 0:  du_q = c ( sum_p Gn[q][p] u_p - Lp[q] t ),  t = sum_p lm[p] u^+_p
// with u^- / u^+ the line of the upwind neighbour below / above, and
//   Dt[q][p] = D[p][q] w_p / w_q,  Lp = lp / w,  Lm = lm / w,
//   Gp = Dt - Lp lp^T,  Gn = Dt + Lm lm^T.
// (The transverse weights and |J| of the cell and face integrals cancel
// against the diagonal mass matrix.)
template <typename T>
struct Tab1D {
  T Dt[kMaxN * kMaxN];      // Dt[q][p] = D[p][q] w_p / w_q (the curved-mesh line operator)
  T Gp[kMaxN * kMaxN];
  T Gn[kMaxN * kMaxN];
  T Lp[kMaxN];
  T Lm[kMaxN];
  T lp[kMaxN];
  T lm[kMaxN];
  T w[kMaxN];
  T winv[kMaxN];
};

// Host-side FP64 tables (dg_tables.cpp).  zeta/w: the quadrature points
// and weights at which the operator is collocated; dofz: the DoF nodes
// (equal to zeta except for DG_BASIS_GLL_GAUSS); V[q][i] = phi_i(zeta_q)
// maps DoF values to values at zeta (identity for the collocated bases).
struct HostTables {
  int n, basis;
  double zeta[kMaxN], w[kMaxN];
  double dofz[kMaxN];
  double V[kMaxN][kMaxN], Vinv[kMaxN][kMaxN];
  double D[kMaxN][kMaxN];  // D[p][i] = phi_i'(zeta_p)
  double lp[kMaxN], lm[kMaxN];
  double Iq[kMaxN][kMaxN];  // Iq[q][i] = int_{-1}^{zeta_q} phi_i (1D Poisson solve)
  Tab1D<double> t64;
  Tab1D<float> t32;
};
bool gauss_legendre(int n, double* x, double* w);
bool gauss_lobatto(int n, double* x, double* w);
// DoF nodes, quadrature points and weights of a basis (any may be NULL).
bool basis_points(int basis, int n, double* dof_nodes, double* qpoints, double* qweights);
void build_tables(int n, int basis, HostTables* t);

// Kernel parameters (passed by value; lives in the constant bank).
struct KParams {
  int dx, dv;
  int ncell[kMaxDim];
  long long cstride[kMaxDim];
  long long ncells;
  long long ncx;            // cells of the x mesh (cell = c_x + ncx * c_v)
  int order[kMaxDim];       // sweep order of the directions
  int cells_per_block;
  const void* cx_tab;       // contravariant speeds of the x directions at v nodes: [ncv][n^dv][dx]
  const void* cv_tab;       // contravariant speeds of the v directions at x nodes: [ncx][n^dx][dv]
  const void* src;          // operator input (apply) / stage vector w_in
  void* dst;                // operator output (apply) / stage vector w_out
  double* u;                // FP64 state (stage mode)
  void* scratch;            // per-block accumulators (large cells)
  int* err;                 // device error latch
  unsigned* work;           // work-queue counter of the persistent kernels
  int mode;                 // 0 = apply, 1 = LSRK stage
  int adjoint;              // 1: L^T = M L(-a) M^{-1}
  int negate;               // 1: L(-a), the forward operator of the negated field
                            // (generic kernel only; the adjoint steps of the generic
                            // path run it on states scaled by the node weights)
  int last_stage;           // stage mode: w_out = u_new
  double a_dt, b_dt;        // stage mode coefficients (a_s dt, b_s dt)
  int tab;                  // constant-table set of the 6D kernels (0 GL, 1 GLL)
  const float* kref;        // stage mode, delta-f form: K = kref + L(w) (nullptr: plain)
  // 128-thread 6D kernel only: walk the v3 cells [v3_lo, v3_lo + v3_n) of
  // every pencil (v3_n = 0: all of them); the upwind v3 neighbour of the
  // first cell is read from the stage vector
  int v3_lo, v3_n;
  // 128-thread 6D kernel with FP64 input (Gauss-Legendre): an FP32 copy of
  // src (same rounding as its own loads), read by tensor copies instead
  const float* src32;
  // curved x-mesh (nullptr: affine), in the compute type: per x cell and x
  // point [ncx][n^dx][1 + dx*dx] = (1/|J_x|, |J_x| J_x^{-1} row-major); per x
  // cell, direction j, side (0: -1, 1: +1) and face point (the other x
  // digits) [ncx][dx][2][n^(dx-1)][dx] = |J_x| (J_x^{-1})_{j,:}; and the
  // physical a_x at the v points [ncv][n^dv][dx]
  const void* geo_c;
  const void* geo_f;
  const void* ax_tab;
  Tab1D<double> t64;
  Tab1D<float> t32;
};

// Precision combinations of the cell kernels: compute type / input / output.
enum Combo { kDDD = 0, kFFF = 1, kFDD = 2, kNumCombo = 3 };

struct LaunchCfg {
  int threads = 256;
  int cells_per_block = 1;
  int order[kMaxDim] = {0, 1, 2, 3, 4, 5};
  int variant = 0;
};

// Launch entry points, one per dimension (dg_inst_d*.cu).  Return a CUDA
// error code (cudaSuccess on success).
cudaError_t launch_cell_d2(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_cell_d3(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_cell_d4(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_cell_d5(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_cell_d6(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);

// Bytes of dynamic shared memory of the generic kernel, or 0 if the cell does
// not fit (then the global-memory variant with per-block scratch is used).
size_t generic_smem_bytes(int d, int n, int combo, int cells_per_block);
// Scratch elements (of the compute type) per block for the global variant.
long long generic_scratch_elems(int d, int n);
int generic_grid_blocks(int d, int n, long long ncells, int cells_per_block, int threads);

// Specialised 6D, n = 4, FP32-sweep kernel (dg_cell6d.cu).  Returns
// cudaErrorNotSupported if the configuration is not covered.
cudaError_t launch_cell_6d4(int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
// Specialised 5D (dim_x = 2, dim_v = 3), n = 4 FP32-sweep kernel (dg_cell5d.cu):
// forward operator (also of the negated field), apply and stage;
// cudaErrorNotSupported if the configuration is not covered.
cudaError_t launch_cell_5d(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
// Specialised 4D (dim_x = dim_v = 2) FP32-sweep kernel, n = 2..6 (dg_cell4d.cu);
// cudaErrorNotSupported if the configuration is not covered.
cudaError_t launch_cell_4d(int n, int combo, KParams& p, const LaunchCfg& cfg, cudaStream_t s);
// Uploads the n = 4 tables of the specialised kernel (they depend on n only).
cudaError_t init_cell6d_tables(const Tab1D<float>& t, int tab);
// A block whose bounded mbarrier wait runs out by construction (dg_cell6d.cu).
cudaError_t launch_wait_probe(int* err, cudaStream_t s);

// Records the thread's last-error message and returns s (dg_api.cu).
dg_status report(dg_status s, const char* msg);
// LSRK(5,4) coefficients a_1..a_4 and b_1..b_5 (dg_api.cu).
void lsrk_coefficients(double* a4, double* b5);

// Small kernels (dg_misc.cu).
cudaError_t launch_convert(const double* u, void* w, int w_is_float, long long n, cudaStream_t s);
cudaError_t launch_integrals(const KParams& p, int n, const double* u, double* partial,
                             int blocks, double detJ, const double* jx, int nqx, cudaStream_t s);
// Zero-mean periodic antiderivative of rho - mean(rho) on a 1D mesh (the
// Poisson solve of Sec. 6 for dim_x = 1), and contravariant v speeds from a
// device field (dg_misc.cu).
struct PoissonTab {
  double Iq[kMaxN * kMaxN];   // [q][i]
  double w[kMaxN];
};
cudaError_t launch_poisson_1d(const double* rho, double* e, long long ncx, int n,
                              const PoissonTab& t, double hphys, cudaStream_t s);
// pieces of the transposed Vlasov-Poisson stage (dg_vp_adjoint.cu)
cudaError_t launch_field_adjoint(const double* w, const double* lam, const double* cv64, long long ncx,
                                 long long ncv, int npc, int nqx, int nqv, int n, int dv, long long ncv1,
                                 const Tab1D<double>& t, double two_over_h, double* g, cudaStream_t s);
cudaError_t launch_poisson_1d_adjoint(const double* y, double* out, long long ncx, int n,
                                      const PoissonTab& t, double hphys, cudaStream_t s);
cudaError_t launch_charge_adjoint_add(double* out, const double* m, long long ncx, long long ncells,
                                      int npc, int nqx, int n, int dv, const Tab1D<double>& t,
                                      double detJv, cudaStream_t s);
cudaError_t launch_lincomb(double* y, double a, const double* x, double b, const double* z, long long n,
                           cudaStream_t s);
cudaError_t launch_field_speeds(const double* e, int comps, double scale, long long ncx, int nq,
                                int dv, const double* two_over_hv, double* cv64, float* cv32,
                                int* flags, int* err, cudaStream_t s);
// An n x n matrix (row-major, leading dimension kMaxN) passed by value.
struct BasisMat {
  double m[kMaxN * kMaxN];
};
// Tensor-product change of basis on every cell (dg_misc.cu).  tmp: an FP64
// vector of n_dofs for cells too large for shared memory (FP64 in and out
// only there; cudaErrorNotSupported otherwise).
cudaError_t launch_basis_change(const void* x, int x_is_float, void* y, int y_is_float, double* tmp,
                                long long ncells, int d, int n, const BasisMat& M, cudaStream_t s);
// y = f32(a - b) (delta-f input), and z = k + f64(y) (delta-f output), and
// x += s * r in FP64 (dg_misc.cu).
cudaError_t launch_sub_to_f32(const double* a, const double* b, float* y, long long n, cudaStream_t s);
cudaError_t launch_add_f32(const double* k, const float* y, double* z, long long n, cudaStream_t s);
cudaError_t launch_axpy(double* x, double sc, const double* r, long long n, cudaStream_t s);
// u[cell * npc + q] *= f[q] for every cell (dg_misc.cu).
cudaError_t launch_scale_nodes(double* u, long long ncells, int npc, const double* f, cudaStream_t s);
cudaError_t launch_charge_density(const void* f, int f_is_float, long long ncx, long long ncv,
                                  int npc, int nqx, int nqv, int dv, int n,
                                  const Tab1D<double>& t, double detJv, double* rho,
                                  cudaStream_t s);

}  // namespace dg

// The handle.
struct dg_ctx {
  int dx = 0, dv = 0, d = 0, k = 0, n = 0;
  int ncell[dg::kMaxDim] = {0};
  long long cstride[dg::kMaxDim] = {0};
  long long ncells = 0, ncx = 0, ncv = 0, n_dofs = 0;
  int npc = 0;            // n^d
  int nqx = 0, nqv = 0;   // n^dx, n^dv
  double h[dg::kMaxDim] = {0};
  double lo[dg::kMaxDim] = {0};
  double S[9] = {0}, Sinv[9] = {0};
  double detJ = 0.0;
  int field_kind = 0;
  int basis = 0;            // dg_basis
  bool curved = false;      // deformed x-mesh (dg_geometry.deform)
  double deform[3] = {0, 0, 0};
  std::vector<double> geo_c_host, geo_f_host, ax_host;
  double* geo_c64 = nullptr; float* geo_c32 = nullptr;
  double* geo_f64 = nullptr; float* geo_f32 = nullptr;
  double* ax64 = nullptr; float* ax32 = nullptr;
  double* jx_d = nullptr;   // |J_x| per x point (FP64) for the integrals
  double* wnode_d = nullptr;  // node weights W_q = prod_i w_{q_i} and their inverses (2 npc)
  double* bc_tmp[4] = {nullptr, nullptr, nullptr, nullptr};   // DG_BASIS_GLL_GAUSS temporaries
  double a_const[dg::kMaxDim] = {0};
  double speed_sum = 0.0;
  // every cell has a single upwind side per direction (no speed component
  // changes sign inside a cell): required by the specialised kernels
  bool uniform_sides = true;
  bool cx_uniform = true;       // the x-direction part of uniform_sides (fixed by the v mesh)
  int device = 0;
  dg::HostTables tables;
  std::vector<double> cx_host, cv_host;   // contravariant speeds (FP64)
  std::vector<float> cx32_host, cv32_host; // FP32 copies with side-consistent zeros
  double* cx_d64 = nullptr; float* cx_d32 = nullptr;
  double* cv_d64 = nullptr; float* cv_d32 = nullptr;
  int* err_d = nullptr;
  unsigned* work_d = nullptr;   // work-queue counter
  int* field_flags_d = nullptr; // device-fed field: bit 0 mixed upwind side in a cell, bit 1 non-finite
  // delta-f form: reference state, its operator in FP64 and FP32, and the
  // K_ref the next enqueued stages add (set only inside dg_rk_step_df)
  double* df_u = nullptr;
  double* df_k64 = nullptr;
  float* df_k32 = nullptr;
  const float* kref_active = nullptr;
  double* df_tmp = nullptr;     // two FP32 vectors for dg_apply_df
  bool df_ready = false;
  double* vp_rho = nullptr;     // Vlasov-Poisson scratch: rho and E at the x nodes
  double* vp_e = nullptr;
  double* vpa = nullptr;        // adjoint Vlasov-Poisson step: 9 FP64 vectors and 2 x-node arrays
  // device staging of the host-buffer stage call: u (FP64) and two stage vectors
  void* host_stage = nullptr; size_t host_stage_bytes = 0;
  float* in32 = nullptr;        // FP32 copy of an FP64 kernel input (n_dofs)
  // pipelined host-buffer stage: copy streams and events (created on first use)
  static constexpr int kMaxChunks = 8;
  cudaStream_t xfer_in = nullptr, xfer_out = nullptr;
  cudaEvent_t xev[2 * kMaxChunks + 2] = {};
  void* scratch = nullptr; size_t scratch_bytes = 0;
  double* partial = nullptr; int partial_blocks = 0;
  cudaStream_t capture_stream = nullptr;
  dg::LaunchCfg cfg[3];
  // cached RK graphs
  struct GraphKey {
    const void* u = nullptr; const void* w0 = nullptr; const void* w1 = nullptr;
    double dt = 0.0; int prec = -1; int adjoint = -1; int parity = -1;
    const void* kref = nullptr;
    bool operator==(const GraphKey& o) const {
      return u == o.u && w0 == o.w0 && w1 == o.w1 && dt == o.dt && prec == o.prec &&
             adjoint == o.adjoint && parity == o.parity && kref == o.kref;
    }
  };
  // a small least-recently-used cache: the checkpointed backward of the
  // autograd wrapper alternates between the recomputation and the adjoint
  // steps, which are different graphs
  static constexpr int kGraphSlots = 8;
  GraphKey gkey[kGraphSlots];
  cudaGraphExec_t gexec[kGraphSlots] = {};
  unsigned long long gused[kGraphSlots] = {};
  unsigned long long gclock = 0;
};
