/*
 * dg.h -- C ABI of the GB300 (sm_103a) high-dimensional DG advection library.
 *
 * The library applies the matrix-free, sum-factorised, upwind discontinuous
 * Galerkin advection operator of Munch, Kormann & Kronbichler, "hyper.deal:
 * An efficient, matrix-free finite-element library for high-dimensional
 * partial differential equations" (arXiv 2002.08110), on the tensor product
 * of a configuration-space mesh (x, dim_x <= 3) and a velocity-space mesh
 * (v, dim_v <= 3), and integrates it in time with the five-stage, fourth-order
 * low-storage Runge-Kutta scheme the paper uses (Sec. 5.4).
 *
 * Discretisation (fixed by this library):
 *  - PDE df/dt + div(a f) = 0 on a periodic box (Sec. 1.2, Eq. intro:advection);
 *  - tensor-product polynomials of degree k, d = dim_x + dim_v (Sec. 2.3),
 *    by default nodal at the k+1 Gauss-Legendre points of each direction,
 *    with the same points as quadrature (collocation: diagonal mass matrix,
 *    Sec. 1.3 and Algorithm 2 step 4); dg_geometry.basis selects the
 *    Gauss-Lobatto collocation or the paper's Gauss-Lobatto nodes with
 *    Gauss quadrature (Sec. 1.3, 2.5) instead;
 *  - weak form in reference coordinates with the phase-space Jacobian
 *    J = diag(J_x, J_v) (Sec. 1.3 Eq. into:adv:ref, Sec. 3) and the upwind flux;
 *  - element-centric evaluation over all cell pairs (Algorithms 1 and 2).
 *
 * Supported: 1 <= dim_x <= 3, 1 <= dim_v <= 3, 2 <= d <= 6, 1 <= k <= 5.
 *
 * Conventions shared by every call:
 *  - Vectors are device memory owned by the caller, contiguous, at least
 *    16-byte aligned, n_dofs elements, laid out as
 *        index = cell * (k+1)^d + q,
 *    cell = sum_j c_j * prod_{m<j} N_m over the d cell coordinates (the x
 *    dimensions first, x_1 fastest; i.e. cell = c_x + N_x * c_v as in the
 *    paper's lexicographic enumeration, Sec. 3.2), and q = sum_j q_j (k+1)^j
 *    over the node indices (x_1 fastest).
 *  - Precision codes (argument ``prec``):
 *      DG_PREC_FP64  (0): FP64 vectors, FP64 arithmetic;
 *      DG_PREC_FP32  (1): FP32 vectors / stage vectors, FP32 sweeps
 *                         (in dg_rk_step the state u stays FP64);
 *      DG_PREC_MIXED (2): FP64 vectors, FP32 sweeps and fluxes.
 *  - Calls that take ``stream`` (a cudaStream_t, NULL = legacy default
 *    stream) only enqueue work: they are asynchronous with respect to the
 *    host.  Errors found on the host are returned at once; errors found on
 *    the device (non-finite results) are latched in the handle and reported
 *    by dg_check().
 *  - No function throws; every function returns a dg_status.  After an
 *    error, dg_last_error() gives a message (thread-local).
 *  - A handle may be used from one host thread at a time.  Its internal
 *    buffers (the FP32 input copy of DG_PREC_MIXED applies and stages, the
 *    delta-f, basis-change and host-staging buffers, the copy streams of the
 *    host-buffer stage) are shared by its calls, so calls on one handle that
 *    run on different streams must not overlap on the GPU; use one handle
 *    per stream for concurrent work.
 */
#ifndef DG_H
#define DG_H

#ifdef __cplusplus
extern "C" {
#endif

#define DG_ABI_VERSION 4

typedef struct dg_ctx* dg_handle;
typedef struct dg_batch_ctx* dg_batch;

typedef enum {
    DG_OK = 0,
    DG_ERR_INVALID_ARG = 1,   /* bad pointer, size, precision or geometry   */
    DG_ERR_UNSUPPORTED = 2,   /* dimension or degree outside the ranges     */
    DG_ERR_CUDA = 3,          /* a CUDA runtime call failed                 */
    DG_ERR_OOM = 4,           /* device or host allocation failed           */
    DG_ERR_NONFINITE = 5,     /* a kernel produced NaN or Inf               */
    DG_ERR_TIMEOUT = 6,       /* a bounded wait inside a kernel gave up     */
    DG_ERR_BOUNDS = 7         /* bounds-check build only (libdg_bounds.so,
                                 compiled with -DDG_BOUNDS_CHECK): a kernel
                                 computed a cell, neighbour, tile or slab
                                 index out of its range (the access was
                                 redirected to index 0; results invalid)   */
} dg_status;

typedef enum {
    DG_PREC_FP64 = 0,
    DG_PREC_FP32 = 1,
    DG_PREC_MIXED = 2
} dg_precision;

/* Velocity field kinds. */
typedef enum {
    /* a = a_const, constant and uniform (the setting of Sec. 5.1). */
    DG_FIELD_CONSTANT = 0,
    /* Phase space (Sec. 6): a_x = (v_1, ..., v_{dim_x}) (needs dim_v >= dim_x)
     * and a_v = E(x), E given at the x quadrature nodes (e_nodes). */
    DG_FIELD_PHASE_SPACE = 1
} dg_field_kind;

/* Nodal bases of the element (Sec. 1.3, 2.3, 2.5, 5.3). */
typedef enum {
    /* Nodes and quadrature at the k+1 Gauss-Legendre points (collocation,
     * diagonal mass matrix).  The default (a zero-initialised geometry). */
    DG_BASIS_GL = 0,
    /* Nodes and quadrature at the k+1 Gauss-Lobatto points (the collocation
     * variant the paper mentions; diagonal mass, quadrature exact to degree
     * 2k-1). */
    DG_BASIS_GLL = 1,
    /* Nodes at the Gauss-Lobatto points, quadrature at the Gauss-Legendre
     * points (the paper's default element).  Its operator equals
     * V^{-1} L_GL V with V_qi = phi_i(Gauss point q) in every direction, which
     * is how the library evaluates it: vectors are changed to values at the
     * Gauss points, the Gauss-Legendre operator runs, and the result is
     * changed back (around each dg_apply, dg_rk_stage and dg_rk_step call). */
    DG_BASIS_GLL_GAUSS = 2
} dg_basis;

/*
 * Geometry and velocity field (Sec. 3: tensor product of two meshes; the
 * mapping is block diagonal).  Configuration space is the lattice box
 * [x_lo, x_hi] (first dim_x entries) with N_x cells per direction, mapped
 * affinely by x = S y (S = shear_x, row-major dim_x x dim_x; an all-zero
 * matrix means identity).  Velocity space is the box [v_lo, v_hi] with N_v
 * cells per direction.  All boundaries are periodic.
 *
 * e_nodes (DG_FIELD_PHASE_SPACE only; NULL means E = 0): host array of
 *   n_xcells * (k+1)^dim_x * dim_v doubles, E_i at the x quadrature point
 *   (cell c_x, point q_x), index (c_x * (k+1)^dim_x + q_x) * dim_v + i, with
 *   c_x and q_x lexicographic, x_1 fastest; point coordinates as given by
 *   dg_node_coordinates(space 2).  For the collocated bases the quadrature
 *   points are the nodes.  The library copies it; the caller keeps ownership.
 *
 * basis: a dg_basis value (0, the Gauss-Legendre collocation, if the struct
 *   is zero-initialised).
 *
 * deform: amplitudes delta_i of a curved (non-affine) configuration mesh; all
 *   zero (the default) keeps the affine map.  The map is
 *     x_i = y_i + delta_i L_m / (2 pi) sin(2 pi (y_m - x_lo_m) / L_m),
 *   m = (i + 1) mod dim_x, L = x_hi - x_lo: periodic, with a Jacobian of its
 *   own at every quadrature point (Sec. 5.1 deforms the Cartesian mesh for
 *   this reason).  |delta_i| < 0.5; not combined with shear_x; collocated
 *   bases (DG_BASIS_GL, DG_BASIS_GLL) only.  Fields and initial data stay
 *   functions of the lattice coordinates y.  The curved mesh runs in the
 *   generic kernel; its transposed operator (dg_apply_adjoint, adjoint
 *   steps) and the 1D Poisson solve are UNSUPPORTED.
 */
typedef struct {
    double x_lo[3], x_hi[3];
    double v_lo[3], v_hi[3];
    double shear_x[9];
    int field_kind;
    double a_const[6];
    const double* e_nodes;
    int basis;
    double deform[3];
} dg_geometry;

typedef struct {
    long long n_dofs;         /* |C| (k+1)^d  (Sec. 2.3, Eq. dealii:totalunkonwns) */
    long long n_cells;        /* |C_x| |C_v|                                */
    long long n_xcells, n_vcells;
    int dofs_per_cell;        /* (k+1)^d                                    */
    int dim_x, dim_v, degree;
    double speed_sum;         /* sum_j max over nodes of |a_j| / h_j        */
    double det_jacobian;      /* |J| of every cell                          */
    double h[6];              /* cell sizes (lattice sizes in x)            */
    int uniform_sides;        /* 1 if no speed component changes sign inside
                                 a cell (each cell has one upwind neighbour
                                 per direction); the specialised 6D kernel
                                 runs only then                             */
    int basis;                /* dg_basis of the handle                     */
} dg_info_t;

/* Launch configuration of the cell kernels (chosen by dg_autotune). */
typedef struct {
    int threads;              /* threads per block                          */
    int cells_per_block;      /* cells handled by one block (small cells)   */
    int order[6];             /* order in which the d directions are swept  */
    int variant;              /* 0 = generic; 6D, k = 3, FP32 sweeps: 1 = specialised,
                                 64 threads per cell; 2 = specialised, 128 threads per
                                 cell (default).  4D with dim_x = dim_v = 2, FP32
                                 sweeps: 2 = specialised, n^2 threads per cell, cell
                                 in registers (default; the delta-f stage and
                                 curved meshes use the generic kernel).  5D with
                                 dim_x = 2, dim_v = 3, k = 3, FP32 sweeps: 2 =
                                 specialised, 64 threads per cell in three
                                 register phases (default; the transpose, the
                                 delta-f stage and curved meshes use the generic
                                 kernel)                                     */
} dg_launch;

/* Library version (DG_ABI_VERSION). */
int dg_version(void);

/* Message of the last error on this thread ("" if none).  The pointer stays
 * valid until the next call on this thread. */
const char* dg_last_error(void);

/*
 * n = degree+1 Gauss-Legendre nodes and weights on [-1, 1] (Sec. 2.5), in
 * ascending order, written to host arrays of n doubles (weights may be NULL).
 * INVALID_ARG if degree < 0 or degree > 5 or nodes == NULL.
 */
dg_status dg_reference_nodes(int degree, double* nodes, double* weights);

/*
 * The 1D points of a dg_basis of degree ``degree`` on [-1, 1], ascending,
 * into host arrays of degree+1 doubles (each may be NULL): the DoF nodes, and
 * the quadrature points and weights of the cell integrals (where fields are
 * sampled).  DG_BASIS_GLL and DG_BASIS_GLL_GAUSS need degree >= 1.
 * INVALID_ARG for an unknown basis or degree outside [0, 5].
 */
dg_status dg_basis_nodes(int basis, int degree, double* nodes, double* qpoints, double* qweights);

/*
 * Create a handle for the mesh T_x (x) T_v (Sec. 3, Eq. concept:tria:tensor)
 * of degree ``degree`` on the current CUDA device.  cells_x[dim_x] and
 * cells_v[dim_v] give cells per direction (>= 1).  Computes the 1D tables in
 * FP64 on the host and the contravariant speeds c = J^{-1} a at every x and
 * v node (never the d-dimensional field, Sec. 6), and uploads them.  No
 * vector is allocated.  Errors: INVALID_ARG (NULL pointers, bad sizes,
 * empty boxes, singular shear, field kind), UNSUPPORTED (dimensions or degree
 * out of range, phase-space field with dim_v < dim_x), OOM, CUDA.
 */
dg_status dg_create(int dim_x, int dim_v, int degree, const int* cells_x, const int* cells_v,
                    const dg_geometry* geometry, dg_handle* out);

/* Release the handle and all device memory it owns.  NULL is a no-op. */
dg_status dg_destroy(dg_handle h);

/* Sizes and geometry of a handle (host struct filled by the library). */
dg_status dg_info(dg_handle h, dg_info_t* info);

/*
 * Node coordinates (host output).  space 0: x nodes, n_xcells*(k+1)^dim_x
 * rows of dim_x lattice coordinates y (physical x = S y); space 1: v nodes,
 * n_vcells*(k+1)^dim_v rows of dim_v velocity coordinates.  Row order is
 * (cell, node), both lexicographic with the first direction fastest.
 * space 2 and 3: the same for the x and v quadrature points (equal to the
 * nodes except for DG_BASIS_GLL_GAUSS).  space 4: physical coordinates x of
 * the x nodes (x = S y, or the curved map of dg_geometry.deform).
 */
dg_status dg_node_coordinates(dg_handle h, int space, double* out);

/*
 * Replace E(x) of a DG_FIELD_PHASE_SPACE handle (host array, layout as
 * dg_geometry.e_nodes).  Stream-ordered against work on ``stream``.
 */
dg_status dg_set_field(dg_handle h, const double* e_nodes, void* stream);

/*
 * dst = M^{-1} A(src): one application of the DG advection operator
 * (Algorithm 2: gather, cell integrals, 2d face integrals with the upwind
 * flux and the neighbour's trace across periodic faces, inverse mass,
 * scatter).  src and dst are device vectors of n_dofs elements of the type
 * given by prec (FP64 for DG_PREC_FP64 and DG_PREC_MIXED, FP32 for
 * DG_PREC_FP32); they must not overlap (neighbours of src are read while dst
 * is written).  Errors: INVALID_ARG (NULL, aliasing, misalignment, prec),
 * CUDA.
 */
dg_status dg_apply(dg_handle h, const void* src, void* dst, int prec, void* stream);

/*
 * dst = L^T src with L = M^{-1} A, i.e. the transposed operator:
 * L^T = M L(-a) M^{-1} -- the weak operator with the negated velocity (the
 * downwind flux with respect to a) applied to the mass-scaled input.  Same
 * arguments and errors as dg_apply.  (The paper has no adjoint; this is the
 * exact transpose of dg_apply's operator.)
 */
dg_status dg_apply_adjoint(dg_handle h, const void* src, void* dst, int prec, void* stream);

/*
 * One fused stage s (0..4) of LSRK(5,4) in 2R form (Sec. 5.4; coefficients of
 * Kennedy, Carpenter & Lewis 2000):
 *     K = L(w_in)        (L^T if adjoint != 0)
 *     w_out = u + a_s dt K    (s < 4)   or   w_out = u + b_4 dt K (s = 4)
 *     u     = u + b_s dt K
 * u is the FP64 state (updated in place); w_in/w_out are stage vectors of
 * the type given by prec and must be distinct from each other and from u.
 * Writing u + b_4 dt K at the last stage makes w_out the next step's first
 * stage vector.
 */
dg_status dg_rk_stage(dg_handle h, const void* w_in, void* w_out, double* u, int stage,
                      double dt, int prec, int adjoint, void* stream);

/*
 * dg_rk_stage with HOST buffers: w_in, w_out (type by prec) and u (FP64) live
 * in host memory (pinned for asynchronous copies; pageable works but the
 * copies then synchronise).  The call copies w_in and u to device staging
 * buffers owned by the handle (n_dofs * (8 + 2 * element size) bytes,
 * allocated on first use, kept until dg_destroy), runs the fused stage and
 * copies u and w_out back, all ordered on ``stream``.  The host buffers must
 * stay valid until the stream reaches the end of the call.  This is the
 * end-to-end form of one stage for callers whose state lives on the host.
 * Where the 128-thread 6D kernel runs (dg_launch variant 2, FP32 sweeps, at
 * least 2 cells along v3), the stage is pipelined over up to 8 slabs of v3
 * cells: copies in, kernels and copies out of different slabs overlap on two
 * handle-owned copy streams joined to ``stream`` by events; the results are
 * bit-identical to dg_rk_stage.  Otherwise the copies and the stage run one
 * after the other on ``stream``.
 */
dg_status dg_rk_stage_host(dg_handle h, const void* w_in, void* w_out, double* u, int stage,
                           double dt, int prec, void* stream);

/*
 * nsteps full LSRK(5,4) steps of size dt on the FP64 state u (in place),
 * using the caller's stage vectors w0 and w1 (type by prec; contents on entry
 * ignored, on exit unspecified).  Copies u into w0, then runs 5 fused stages
 * per step, replayed from a CUDA graph that the handle captures on first use
 * and re-captures when pointers, dt, prec or adjoint change.  If ``stream``
 * is being captured by the caller, the kernels are enqueued directly.
 * adjoint != 0 integrates with L^T (the adjoint step of a linear,
 * autonomous problem: R(dt L)^T = R(dt L^T)).
 */
dg_status dg_rk_step(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps,
                     int prec, int adjoint, void* stream);

/*
 * delta-f form (FP32 sweeps with an FP64 reference).  With smooth data the
 * result of the operator is much smaller than its terms, so FP32 sweeps lose
 * relative accuracy; splitting u = u_ref + du and using linearity,
 * L(u) = L(u_ref) + L(du), with L(u_ref) evaluated once in FP64, leaves FP32
 * rounding only on the small part du.
 *
 * dg_set_reference: copies the FP64 device vector u_ref into the handle and
 * evaluates K_ref = L(u_ref) in FP64 (kept in FP64 and FP32); the handle then
 * holds 20 bytes per DoF until dg_destroy.  UNSUPPORTED for
 * DG_BASIS_GLL_GAUSS.  Stream-ordered.
 *
 * dg_apply_df: dst = K_ref + L(f32(src - u_ref)) with FP32 sweeps; src and
 * dst are FP64 device vectors.
 *
 * dg_rk_step_df: nsteps LSRK(5,4) steps on the FP64 state u (in place) in
 * the form du = u - u_ref, K = K_ref + L(dw): FP32 stage vectors w0, w1 hold
 * dw; u is turned into du before the steps and back after them (two FP64
 * passes; the round trip rounds u at the level of its own ulp).  Graph-
 * replayed like dg_rk_step.
 */
dg_status dg_set_reference(dg_handle h, const double* u_ref, void* stream);
dg_status dg_apply_df(dg_handle h, const double* src, double* dst, void* stream);
dg_status dg_rk_step_df(dg_handle h, double* u, float* w0, float* w1, double dt, int nsteps,
                        void* stream);

/*
 * Integrals of the FP64 vector u with the cell quadrature: out[0] = int u,
 * out[1] = int u^2, out[2] = max |u_i| over the nodes.  Synchronises
 * ``stream``; out is a host array of 3 doubles.
 */
dg_status dg_integrals(dg_handle h, const double* u, double* out, void* stream);

/*
 * Charge density of the Vlasov-Poisson coupling (Sec. 6, Eq. vp:close):
 * rho(x) = 1 - int f(x, v) dv at every x node, the velocity integral taken
 * with the cell quadrature of the v mesh (|J_v| times the product of the GL
 * weights).  f: device vector (FP64 for DG_PREC_FP64, FP32 for
 * DG_PREC_FP32); rho: device array of n_xcells * (k+1)^dim_x doubles in the
 * layout of dg_geometry.e_nodes without the component index (x cell, x node;
 * both lexicographic, x_1 fastest).  Accumulates in FP64.  Stream-ordered.
 * (Computing E from rho -- the Poisson solve -- is outside this library;
 * dg_set_field takes the result.)
 */
dg_status dg_charge_density(dg_handle h, const void* f, int prec, double* rho, void* stream);

/*
 * Periodic Poisson problem of Sec. 6 (Eq. vp:close) for dim_x = 1:
 * -phi'' = rho, E = -phi', i.e. E' = rho in the physical coordinate
 * x = S y.  Periodicity needs a neutral rho: its mean is removed first.  E is
 * the exact antiderivative of the nodal degree-k polynomial of rho - mean in
 * each cell (a continuous piecewise polynomial of degree k+1) with zero mean
 * over the period, written at the x nodes.  rho, e: device arrays of
 * n_xcells * (k+1) doubles (x cell, x node), not overlapping.  One block;
 * deterministic.  Stream-ordered.  Errors: UNSUPPORTED if dim_x != 1.
 * (The paper solves this with geometric multigrid in dim_x = 2, 3; that
 * solver is not part of this library.)
 */
dg_status dg_poisson_periodic_1d(dg_handle h, const double* rho, double* e, void* stream);

/*
 * Replace the v part of the velocity field of a DG_FIELD_PHASE_SPACE handle
 * from DEVICE memory: a_v = scale * e at every x node, e laid out (x cell,
 * x node, component) with ``components`` (1..dim_v) values per node; the
 * remaining components are zero.  For the Vlasov field (v, -E) pass the
 * electric field and scale = -1 (Sec. 6).  Stream-ordered.  For d = 6, k = 3
 * the sign pattern of the field selects the kernel, so the call reads one
 * flag back and synchronises ``stream``; otherwise it does not synchronise.
 * Non-finite values are latched and reported by dg_check (DG_ERR_NONFINITE).
 * dg_info's uniform_sides reflects the field for d = 6, k = 3 and reads 0
 * otherwise.
 */
dg_status dg_set_field_device(dg_handle h, const double* e, int components, double scale,
                              void* stream);

/*
 * nsteps LSRK(5,4) steps of the Vlasov-Poisson system (Sec. 6) for dim_x = 1
 * on the FP64 state f = u (in place).  Every stage evaluates, on its input
 * stage vector: the charge density (dg_charge_density), the electric field
 * (dg_poisson_periodic_1d), the field a_v = (-E, 0, ...) (dg_set_field_device)
 * and the fused advection stage (dg_rk_stage).  Arguments as dg_rk_step; the
 * handle owns the two x-node scratch arrays (allocated on first use).  Not
 * replayed from a graph.  Errors: UNSUPPORTED if dim_x != 1, INVALID_ARG for
 * a constant-field handle.
 */
dg_status dg_vp_rk_step(dg_handle h, double* u, void* w0, void* w1, double dt, int nsteps, int prec,
                        void* stream);

/*
 * Adjoint of one FP64 Vlasov-Poisson step of dg_vp_rk_step (the gradient of
 * a final-time functional through the coupled steps, Sec. 6 with the
 * differentiation of the north-star's pattern 3).  u: the state at the start
 * of the step (FP64, read only); ubar: on entry dJ/du after the step, on
 * return dJ/du before it (FP64, in place).  The step is not linear in u: its
 * stage right-hand side is F(w) = L(a(w)) w with a_v = -E(w), E = P rho(w),
 * so the call recomputes the step's five stage inputs from u and takes, in
 * reverse stage order, J(w)^T = L(a)^T + R^T P^T B(w)^T with L^T the
 * transposed operator (dg_apply_adjoint), B(w) the operator's derivative with
 * respect to the field at the x nodes (upwind sides fixed by the current
 * field), P^T the transposed Poisson map and R^T the transposed v
 * quadrature.  All in FP64 kernels.  The handle owns 9 FP64 vectors of scratch
 * for it (allocated on first use); on return its field is that of the
 * step's first stage.  Errors: as dg_vp_rk_step.
 */
dg_status dg_vp_step_adjoint(dg_handle h, const double* u, double* ubar, double dt, void* stream);

/*
 * The integrals of dg_integrals() for callers that cannot allocate device
 * memory: for example code inside a framework whose allocator owns all
 * device memory, or a long run that must not call cudaMalloc after start-up
 * (cudaMalloc synchronises the device and can fail on a fragmented heap).  It
 * needs no handle and calls no cudaMalloc, cudaFree or other allocating
 * routine: its scratch is a fixed array of 98,328 bytes compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The paper has no counterpart to this entry point.
 *
 * Elements covered: the collocated bases on affine meshes, i.e. basis
 * DG_BASIS_GL (Gauss-Legendre weights) or DG_BASIS_GLL (Gauss-Lobatto
 * weights) with one |J| for every cell.  DG_BASIS_GLL_GAUSS (whose states
 * need a change of basis first) is rejected with DG_ERR_UNSUPPORTED.  A
 * curved mesh (dg_geometry.deform) has a |J| per point and is not covered:
 * use dg_integrals for it.
 *
 * u: device vector of n_cells * (degree+1)^dim FP64 values in the layout of
 * this header (16-byte aligned); det_jacobian: |J| of every cell
 * (dg_info.det_jacobian); out: host array of 3 doubles, receives
 * (int u, int u^2, max |u_i|).  At most 2^32 DoFs per call: larger vectors
 * are rejected with DG_ERR_INVALID_ARG (use dg_integrals).  The call
 * synchronises ``stream`` (it reads the three results back into ``out``).
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; the address is not valid across cudaDeviceReset, so do not
 * use this call after resetting the device.  All calls on a device share the
 * one array and a call leaves its partial sums there; calls that overlap on
 * the GPU (for instance on two streams at once) race on it, so serialise
 * them.  Every slot a call reads is written by that call first, so nothing
 * needs clearing.
 */
dg_status dg_integrals_noalloc(const double* u, long long n_cells, int dim, int degree, int basis,
                               double det_jacobian, double* out, void* stream);

/*
 * Synchronise ``stream`` and report device-side errors latched since the
 * last check: DG_ERR_BOUNDS (bounds-check build only) if a kernel computed an
 * index out of its range, else DG_ERR_TIMEOUT if a kernel's bounded wait for
 * an asynchronous copy gave up (its results are invalid in both cases), else
 * DG_ERR_NONFINITE if any kernel produced NaN or Inf.  Clears the latch.
 */
dg_status dg_check(dg_handle h, void* stream);

/*
 * Self-test of the failure path of the bounded waits: launches one block
 * that waits on an mbarrier whose expected bytes never arrive (no copy is
 * issued), gives up after about 1 ms of SM clock and latches the timeout,
 * so the next dg_check returns DG_ERR_TIMEOUT and clears it.  Nothing is
 * left in flight; the context stays usable.  (The cell kernels wait up to
 * about 2 s before giving up the same way.)
 */
dg_status dg_selftest_wait(dg_handle h, void* stream);

/* Current launch configuration for ``prec`` (host struct). */
dg_status dg_get_launch(dg_handle h, int prec, dg_launch* cfg);

/* Override the launch configuration for ``prec`` (validated). */
dg_status dg_set_launch(dg_handle h, int prec, const dg_launch* cfg);

/*
 * Autotuner: times the candidate launch configurations of dg_apply on the
 * caller's buffers src/dst (prec as in dg_apply) and keeps the fastest for
 * ``prec`` (and for the RK stages of the same prec).  dst is overwritten.
 * Synchronises ``stream``.  best_ms (host, may be NULL) receives the time of
 * the chosen configuration.
 */
dg_status dg_autotune(dg_handle h, const void* src, void* dst, int prec, void* stream,
                      double* best_ms);

/*
 * Batched execution of independent problems (constant velocity only; d = 3
 * or 4).  The paper runs one problem at a time; advancing many independent
 * problems together is this library's addition.
 * dg_batch_create groups ``count`` handles (each stays owned by the caller
 * and must outlive the batch).  dg_batch_rk_step advances every member i by
 * nsteps LSRK(5,4) steps of size dt[i] on its FP64 state u[i] with stage
 * vectors w0[i], w1[i] (host arrays of device pointers).  Members are grouped
 * by (dimension, degree); each stage of a group is one persistent launch of
 * a kernel specialised for that pair, which takes work tiles (a run of one
 * member's cells) from a device queue, and each step (5 stages of every
 * group) is replayed from a CUDA graph.  prec: DG_PREC_FP64 or DG_PREC_FP32
 * (FP32 stage vectors and sweeps, FP64 state); with DG_PREC_FP32 the d = 4
 * groups run the register-resident 4D cell algorithm.
 */
dg_status dg_batch_create(int count, const dg_handle* handles, dg_batch* out);
dg_status dg_batch_destroy(dg_batch b);
dg_status dg_batch_rk_step(dg_batch b, double* const* u, void* const* w0, void* const* w1,
                           const double* dt, int nsteps, int prec, void* stream);
/* Number of work tiles and total DoFs of a batch (host outputs, may be NULL). */
dg_status dg_batch_info(dg_batch b, long long* tiles, long long* n_dofs);
/* dg_check for a batch: synchronise and report non-finite results. */
dg_status dg_batch_check(dg_batch b, void* stream);
/* Launch configuration of the batched kernels. */
typedef struct {
    int tile_dofs;   /* shared-memory kernel: DoFs per work tile (whole cells,
                        >= one cell), 64..65536; default 4096                 */
    int threads;     /* shared-memory kernel: threads per block; default 256 */
    int threads4;    /* 4D register kernel: threads per block, 128, 256 or 512
                        (n^2 per cell, so threads4 / n^2 cells per block and
                        per tile; 512 only for n <= 4); default 128.  n = 6
                        runs a pair-split kernel of its own (two threads per
                        column and row, 3 cells per 224-thread block)        */
    int order;       /* direction order, bits: 1 = the second x direction
                        first, 2 = the second v direction first (4D register
                        kernel); 4 = all directions in reverse order (shared-
                        memory kernel).  Results differ only by rounding.     */
    int r4_max_n;    /* FP32 d = 4 groups with n = degree + 1 <= r4_max_n run
                        the 4D register kernel, the others the shared-memory
                        kernel (1: none); default 6                           */
} dg_batch_launch;
/* One configuration timed by dg_batch_autotune and its time per step (ms). */
typedef struct {
    int tile_dofs, threads, threads4, order, r4_max_n;
    double ms;
} dg_batch_trial;
/* Tile size and threads per block of the shared-memory kernel (the rest of
 * the configuration unchanged). */
dg_status dg_batch_set_launch(dg_batch b, int tile_dofs, int threads);
/* Set / read the whole configuration (validated; captured graphs are
 * dropped). */
dg_status dg_batch_set_launch_ex(dg_batch b, const dg_batch_launch* cfg);
dg_status dg_batch_get_launch(dg_batch b, dg_batch_launch* cfg);
/* Autotuner of the batched launch: times two LSRK steps (after one untimed
 * step) for each candidate on the caller's vectors (which are advanced by
 * those steps); best_ms (may be NULL) receives the kept configuration's time
 * per step.  The groups are separate launches whose times add, so it tunes
 * by coordinate descent: which 4D groups run the register kernel, then its
 * block size and direction order, then the shared-memory kernel's tile size
 * and block size, then its direction order; parameters that no group of the
 * batch uses are not varied.  The three fastest candidates and the starting
 * configuration are then timed again over four steps and the fastest of
 * those is kept. */
dg_status dg_batch_autotune(dg_batch b, double* const* u, void* const* w0, void* const* w1,
                            const double* dt, int prec, void* stream, double* best_ms);
/* The configurations the last dg_batch_autotune timed, in the order tried:
 * *count receives their number, and up to max_trials of them are written to
 * trials (host array, may be NULL). */
dg_status dg_batch_autotune_record(dg_batch b, dg_batch_trial* trials, int max_trials, int* count);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
