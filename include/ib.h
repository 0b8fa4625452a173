/*
 * ib.h -- C ABI of the GB300 immersed-boundary acoustic finite-difference library.
 *
 * Method (Caunt, Nelson, Luporini, Gorman, "A Novel Immersed Boundary Approach
 * for Irregular Topography with Acoustic Wave Equations"): grid points near an
 * irregular surface, given as a signed-distance field (SDF) discretised on the
 * FD grid, get modified derivative stencils.  Exterior values needed by an
 * interior stencil are extrapolated by an N-dimensional truncated Taylor
 * polynomial fitted, by the Moore-Penrose pseudoinverse, to interior values
 * and to boundary conditions imposed at boundary points inside a
 * hyperspherical support ("Approximating Boundary Conditions",
 * "Reconciliation with the Interior Numerical Discretization").  The modified
 * operators drive explicit time stepping of the second-order acoustic wave
 * equation (2nd-order application section) or of the first-order staggered
 * pressure-velocity system (1st-order section).
 *
 * Conventions shared by every entry point
 *   - Grid: ndim = 2 or 3, n[0] = nx (fastest), n[1] = nz (2D) or ny (3D),
 *     n[2] = nz (3D); arrays are row-major [nz][nx] or [nz][ny][nx].  Node
 *     (i_x, .., i_z) sits at (i_x h, .., i_z h); z is depth (positive down).
 *   - SDF s > 0 in the physical domain; a node with s <= 0 is exterior and its
 *     fields are held at zero.  Values beyond the array are zero (zero
 *     Dirichlet edges, as in the paper's examples).
 *   - Coordinates (sources, receivers) are metres in logical order
 *     (x, [y,] z), float64, in DEVICE memory.
 *   - Every array argument named *_dev is a device pointer; the caller owns
 *     it.  The library owns tables and its internal scratch (wavefields).
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream).  Entry points return after enqueueing; argument errors are
 *     returned synchronously; device-side faults surface from the next call
 *     or from ib_sync_status().
 *   - No entry point throws.  On failure the status is non-zero and
 *     ib_last_error() returns a thread-local message.
 *   - A table may be used concurrently by several streams for forward and
 *     adjoint runs (read-only); building or freeing it must not overlap them.
 */
#ifndef IB_H
#define IB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IB_OK = 0,
    IB_ERR_ARG = 1,       /* invalid argument (shape, order, pointer, size)        */
    IB_ERR_RANK = 2,      /* a node stayed unconstrained at the largest radius
                             and the lowest basis order (rank paragraph)           */
    IB_ERR_CUDA = 3,      /* a CUDA call failed                                    */
    IB_ERR_OOM = 4,       /* device allocation failed                              */
    IB_ERR_UNSTABLE = 5,  /* NaN/Inf in a run's final fields (ib_sync_status), or
                             a growing mode found by ib_stability                  */
    IB_ERR_TIMEOUT = 6,   /* a bounded device wait gave up.  From a time step the
                             run's results are then not valid, and a copy that never
                             arrived may leave the context unusable; only the
                             self-test (ib_selftest_bounded_wait), which issues no
                             copy, leaves it known to be usable                    */
    IB_ERR_STATE = 7      /* call not valid for this table (e.g. wrong form)       */
} ib_status;

typedef enum { IB_FREE = 0, IB_RIGID = 1 } ib_bc;
/* How exterior values are extrapolated: the paper's N-dimensional Taylor basis
 * over a hyperspherical support ("Approximating Boundary Conditions"), or the
 * per-axis 1D extrapolation it derives as a sub-case ("Reduction to 1D"; the
 * free surface of the second-order form only). */
typedef enum { IB_EXTRAP_ND = 0, IB_EXTRAP_1D = 1 } ib_extrap;
typedef enum { IB_SECOND_ORDER = 0, IB_FIRST_ORDER_STAGGERED = 1 } ib_form;

typedef struct {
    int32_t ndim;          /* 2 or 3                                               */
    int32_t reserved;
    int64_t n[3];          /* nx, (ny,) nz; unused entries 1                       */
    double h;              /* grid step (metres), isotropic                        */
} ib_grid;

typedef struct {
    int32_t space_order;   /* M of the interior stencils: 2, 4, 6 or 8             */
    int32_t basis_order;   /* order of the extrapolation basis; 0 -> min(M, 4)
                              (the reduced basis of the order-reduction paragraph;
                              M gives the consistent-error basis)                  */
    int32_t min_order;     /* lowest basis order of the fallback (>= 2)            */
    int32_t extrapolation; /* ib_extrap: IB_EXTRAP_ND (default) or IB_EXTRAP_1D.
                              1D: on each grid line an axial stencil crosses the
                              surface, the boundary is where the SDF, interpolated
                              linearly between the last interior and the first
                              exterior node, is zero; the 1D Taylor basis of order
                              M (lowered by 2 while the line is too short) is fitted
                              to the M/2 nearest nodes at more than eta_p from it
                              and to p = p'' = .. = p^(M) = 0 there, a square
                              system; basis_order, radius, growth and rank_tol
                              do not apply                                         */
    double radius;         /* initial support radius in grid units; <= 0 ->
                              (basis_order + 1) / 2 (support paragraph)            */
    double growth;         /* radius grows by 0.5 up to radius + growth            */
    double eta_p;          /* pressure cut-off eta; < 0 -> 0.5 for the free surface
                              (the paper's value) and 0.25 for the rigid surface
                              (the paper gives none; 0.5 leaves a growing mode)     */
    double eta_v;          /* velocity cut-off eta (paper: 0)                      */
    double rank_tol;       /* full rank iff sigma_min > rank_tol * sigma_max; <= 0
                              -> 1e-3 for the free surface, 1e-2 for the rigid one  */
} ib_opts;

/* Fill `opts` with the defaults for space order M (basis 0 = min(M, 4), min
 * order 2, radius (basis+1)/2, growth 3, eta_p -1 and rank_tol -1 (by
 * boundary condition), eta_v 0). */
void ib_opts_default(ib_opts* opts, int32_t space_order);

typedef struct ib_table ib_table;   /* opaque, library-owned */

/*
 * ib_build_stencils -- geometry, boundary points and modified stencils.
 * Paper: boundary points and eta cut-off (boundary-point paragraph of
 * "Approximating Boundary Conditions"); support growth and rank test (rank
 * paragraph); fit by pseudoinverse and extrapolation B A^+ ("Reconciliation
 * ..."); free-surface and velocity free-surface hierarchies.
 *   grid     host pointer, read during the call.
 *   sdf_dev  device float64 [N] SDF in metres (N = nx*ny*nz), read during the
 *            call (the call synchronises `stream` before returning).
 *   bc       IB_FREE or IB_RIGID;  form: IB_SECOND_ORDER (modified Laplacian)
 *            or IB_FIRST_ORDER_STAGGERED (modified gradients at velocity
 *            nodes and modified divergence at pressure nodes).
 *   opts     host pointer or NULL (defaults for M = 4).
 *   out      receives a new table; free with ib_table_free.
 * Errors: IB_ERR_ARG (shape/order), IB_ERR_RANK (some node could not be
 * constrained; the table is still returned with those rows marked and left
 * unmodified beyond the standard stencil), IB_ERR_OOM, IB_ERR_CUDA.
 */
ib_status ib_build_stencils(const ib_grid* grid, const double* sdf_dev, ib_bc bc,
                            ib_form form, const ib_opts* opts, ib_table** out,
                            void* stream);

void ib_table_free(ib_table* table);

/* Per-operator statistics of a table. */
typedef struct {
    int32_t n_ops;              /* 1 (Laplacian) or 2*ndim (staggered: the ndim
                                   gradients at velocity nodes, then the divergence
                                   blocks, one per velocity component)              */
    int32_t ndim;
    int64_t rows[8];            /* IB rows per operator                              */
    int64_t nnz[8];             /* correction entries per operator                   */
    int64_t n_boundary_points;  /* accepted boundary points                          */
    int64_t n_rank_failures;    /* rows left without a correction                    */
    int64_t n_grown;            /* rows whose support grew beyond the first radius   */
    int64_t n_reduced;          /* rows whose basis order was lowered                */
    int64_t table_bytes;        /* device bytes of the correction tables             */
    double setup_seconds;       /* wall time of ib_build_stencils                    */
} ib_table_info;

ib_status ib_table_stats(const ib_table* table, ib_table_info* info);

/*
 * ib_table_export -- copy one operator's corrections to HOST buffers (for
 * inspection and tests).  op indexes as in ib_table_info.  Columns are given as
 * integer node offsets (dx, dy, dz) from the row node (x_row, y_row, z_row).
 *   row_node   int64 [rows]   linear index of the row node in [nz][ny][nx]
 *   row_ptr    int64 [rows+1]
 *   col_off    int32 [nnz][3] (dx, dy, dz); dy = 0 in 2D
 *   weight     float64 [nnz]  correction weight in grid units (multiply by
 *                             1/h^2 for the Laplacian, 1/h for first derivatives)
 *   row_info   int32 [rows][4] (radius in half grid units, basis order,
 *                             boundary points used, status 0 ok / 1 rank failure)
 * Any pointer may be NULL to skip it.  Buffers must hold the sizes reported
 * by ib_table_stats.
 */
ib_status ib_table_export(const ib_table* table, int32_t op, int64_t* row_node,
                          int64_t* row_ptr, int32_t* col_off, double* weight,
                          int32_t* row_info);

/*
 * One shot: model, sources, receivers.  Element type of vel/rho/wavelet/
 * traces is float for precision 32 and double for precision 64.
 */
typedef struct {
    const void* vel_dev;        /* [N] wave speed c (m/s)                            */
    const void* rho_dev;        /* [N] density (kg/m^3) or NULL = 1; first-order form */
    const double* src_dev;      /* [nsrc][ndim] metres                               */
    const double* rec_dev;      /* [nrec][ndim] metres                               */
    const void* wavelet_dev;    /* [nt] source time function, sample n is used in
                                   the step that produces p^{n+1}                    */
    void* traces_dev;           /* [nrec][nt] output: trace[r][n] = p^{n+1} at r     */
    int32_t nsrc;               /* 0 .. 32 (more: IB_ERR_ARG)                       */
    int32_t nrec;
    /* Absorbing layer along the side edges and the bottom (the paper's
     * examples use zero Dirichlet edges and note that a damping boundary of
     * choice combines with the method, Examples section).  The second-order
     * form solves p_tt + eta(x) p_t = c^2 lap p + f there, eta = eta_max
     * min(1, d^2 / W^2), d the node's distance (in nodes) into the layer of W
     * = damp_width nodes: from x = 0 and x = nx-1 (and y = 0, y = ny-1 in
     * 3D) and from the last z plane; the top carries the immersed boundary.
     * The step is p^{n+1} = (2 p^n - (1 - a) p^{n-1} + dt^2 c^2 L p^n +
     * dt^2 f) / (1 + a) with a = eta dt / 2.  damp_width = 0 or damp_eta = 0:
     * no layer (zero Dirichlet edges).  Second-order form only (the
     * first-order form and ib_forward_noalloc return IB_ERR_STATE); the
     * adjoint is that of the damped map.  IB_ERR_ARG unless damp_eta >= 0 and
     * 0 <= damp_width < nx / 2. */
    double damp_eta;            /* eta_max (1/s)                                     */
    int32_t damp_width;         /* W (nodes)                                         */
    int32_t reserved;
} ib_shot;

/*
 * ib_forward -- nt explicit time steps (2nd-order application section:
 *   p^{n+1} = 2p^n - p^{n-1} + dt^2 c^2 L_mod p^n + dt^2 f^n;
 * 1st-order section: v += dt/rho G_mod p;  p += dt rho c^2 D_mod v + dt f),
 * p^0 = p^{-1} = 0, fused source injection (multilinear delta, 1/h^d) and
 * receiver interpolation (multilinear, exterior nodes read as zero).
 *   precision  32 or 64.
 *   dt         time step (s); nt >= 1.
 *   ckpt_dev   NULL, or device buffer of ib_checkpoint_bytes(table, precision,
 *              nt, n_ckpt) bytes that receives the wavefield checkpoints the
 *              adjoint needs (second-order form only); n_ckpt >= 1.
 * Errors: IB_ERR_ARG, IB_ERR_STATE, IB_ERR_OOM, IB_ERR_CUDA.
 */
ib_status ib_forward(const ib_table* table, const ib_shot* shot, int32_t precision,
                     double dt, int32_t nt, void* ckpt_dev, int32_t n_ckpt, void* stream);

/* Bytes of the checkpoint buffer for (precision, nt, n_ckpt). */
int64_t ib_checkpoint_bytes(const ib_table* table, int32_t precision, int32_t nt,
                            int32_t n_ckpt);

/*
 * ib_adjoint -- exact transpose of the discrete second-order map (the
 * modified operator transposed, source and receiver maps transposed) with
 * checkpointed recomputation of the forward wavefield.  For
 * J = 1/2 sum_{r,n} (trace[r][n] - d[r][n])^2 and residual = trace - d:
 *   grad_vel_dev[x]     = dJ/dc(x)  (zero at exterior nodes), overwritten;
 *   grad_wavelet_dev[n] = dJ/dw[n]  if not NULL, overwritten.
 * The shot, dt, nt, precision and n_ckpt must be those of the ib_forward call
 * that filled ckpt_dev.  The shot's traces_dev is not read.
 */
ib_status ib_adjoint(const ib_table* table, const ib_shot* shot, int32_t precision,
                     double dt, int32_t nt, const void* ckpt_dev, int32_t n_ckpt,
                     const void* residual_dev, void* grad_vel_dev,
                     void* grad_wavelet_dev, void* stream);

/*
 * ib_forward_batch -- many independent shots, each with its own table (grid
 * and topography), advanced together: every time step is one launch that
 * covers the tiles (or z-marched strips of tiles) of all shots, and all steps
 * are one captured CUDA graph.  The tile shape is timed on the first batch of
 * a size class and remembered; the environment variable IB_BATCH_SHAPE=<0..9>
 * fixes it instead (IB_ERR_ARG outside that range).  Same semantics per shot
 * as ib_forward (precision 32, no checkpoints).  tables[i] and shots[i] are
 * host arrays of length nshot.
 */
ib_status ib_forward_batch(const ib_table* const* tables, const ib_shot* shots,
                           int32_t nshot, int32_t precision, double dt, int32_t nt,
                           void* stream);

/*
 * ib_forward_batch_ckpt -- ib_forward_batch that also fills each shot's
 * checkpoint buffer ckpts[i] (device, ib_checkpoint_bytes(tables[i], 32, nt,
 * n_ckpt) bytes, the layout ib_forward writes), so that either ib_adjoint per
 * shot or ib_adjoint_batch can follow.  ckpts is a host array of nshot device
 * pointers.  Errors: those of ib_forward_batch; IB_ERR_ARG for a null array
 * or buffer or n_ckpt < 1.
 */
ib_status ib_forward_batch_ckpt(const ib_table* const* tables, const ib_shot* shots,
                                int32_t nshot, int32_t precision, double dt, int32_t nt,
                                void* const* ckpts, int32_t n_ckpt, void* stream);

/*
 * ib_adjoint_batch -- ib_adjoint (same transpose, same checkpoint segments)
 * for many shots at once: every recompute step and every adjoint step is one
 * launch over the tiles of all shots, and the whole backward pass is one
 * captured graph.  Per shot i: checkpoints ckpts[i] from ib_forward_batch_ckpt
 * or ib_forward with the same dt, nt and n_ckpt; residuals[i] [nrec][nt];
 * grads[i] [N] receives dJ/dc (overwritten).  Host arrays of nshot device
 * pointers; FP32, 2D second-order tables sharing the space order; no wavelet
 * gradient.  Errors: IB_ERR_ARG (null or mismatched inputs), IB_ERR_STATE
 * (other forms), IB_ERR_OOM, IB_ERR_CUDA.
 */
ib_status ib_adjoint_batch(const ib_table* const* tables, const ib_shot* shots,
                           int32_t nshot, int32_t precision, double dt, int32_t nt,
                           const void* const* ckpts, int32_t n_ckpt,
                           const void* const* residuals, void* const* grads, void* stream);

/*
 * ib_forward_noalloc -- ib_forward for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a deployment variant).  Some
 * callers own every device allocation themselves -- a host framework with its
 * own memory manager or a fixed device-memory budget, or a serving loop that
 * must not allocate once it is running, since cudaMalloc/cudaFree can
 * synchronise the device and stall other streams.  This entry point runs the
 * 2D second-order FP32 forward of ib_forward (same shot semantics, no
 * checkpoints) with all of its scratch (two wavefields, the coefficient
 * field, source and receiver interpolation weights) in one file-scope device
 * array of IB_NOALLOC_SCRATCH_BYTES = 64 MiB.  Every GPU that loads the
 * library holds that array until the process exits.  The call makes no
 * cudaMalloc/cudaFree or other allocating call; the table and the shot
 * buffers are the caller's.
 *   - Needs 3 padded fields (about 12 bytes per grid point) plus 96 bytes per
 *     source and receiver; larger problems return IB_ERR_ARG with the sizes.
 *   - Each call made outside stream capture looks up the array's device
 *     address (cudaGetSymbolAddress) for the current device; a call made
 *     while `stream` is capturing reuses the address from the last
 *     uncaptured call on that device, so make the first call on a device
 *     before any stream capture (a captured first call: IB_ERR_STATE).
 *   - All calls share the array and it keeps the last call's contents: each
 *     call clears what must start at zero, but calls that overlap on the GPU
 *     (other streams, other threads) race on it and must be serialised by the
 *     caller.
 *   - Tables of the first-order form or 3D grids return IB_ERR_STATE.
 */
ib_status ib_forward_noalloc(const ib_table* table, const ib_shot* shot, double dt,
                             int32_t nt, void* stream);

/* ------------------------------------------------------------------------
 * Learned modified stencils.  The paper builds every modified row by its
 * constrained least-squares fit ("Reconciliation with the Interior Numerical
 * Discretization"); it has no learned component.  These entry points add a
 * predictor on top of the method without changing it: a multilayer
 * perceptron maps the signed distance around an IB row's node to the row's
 * correction weights, and a prediction is kept only if it passes the
 * exactness test the fit itself guarantees; every other row is fitted as in
 * ib_build_stencils.  Second-order (Laplacian) rows only.
 * ------------------------------------------------------------------------ */
typedef struct ib_mlp ib_mlp;        /* opaque, library-owned */

typedef struct {
    int32_t ndim;          /* 2 or 3                                           */
    int32_t space_order;   /* M of the rows it predicts (even, 2..8)           */
    int32_t n_hidden;      /* width of every hidden layer, 8..1024, multiple of 8 */
    int32_t n_layers;      /* hidden layers, 1..8                              */
    double in_radius;      /* inputs: SDF / h at lattice offsets |o| <= in_radius
                              around the row node (nearest in-array node past
                              the array edge), then [free, rigid, M / 8]       */
    double out_radius;     /* outputs: corrections at offsets |o| <= out_radius,
                              which must equal the first support radius of the
                              fit, (basis order + 1) / 2                       */
} ib_mlp_config;

/*
 * ib_mlp_create -- network on the current device with zeroed parameters.
 * Offsets are ordered by distance, then by array order (z, y, x), as the
 * fit orders its support.  Layers: Linear -> ReLU for each hidden layer, then
 * Linear.  Weights W_l are [n_out_l][n_in_l] row-major, FP32 masters in one
 * flat vector (W_0, b_0, W_1, b_1, ...); the products use bfloat16 copies of
 * the weights and activations with FP32 accumulation.
 * Errors: IB_ERR_ARG (config out of range), IB_ERR_OOM, IB_ERR_CUDA.
 */
ib_status ib_mlp_create(const ib_mlp_config* cfg, ib_mlp** out);
void ib_mlp_free(ib_mlp* mlp);

/* Sizes: inputs per row, outputs per row, parameters. */
ib_status ib_mlp_info(const ib_mlp* mlp, int64_t* n_in, int64_t* n_out, int64_t* n_params);

/*
 * ib_mlp_buffers -- library-owned device vectors of n_params FP32 values:
 * parameters, last gradient, Adam first and second moments.  Any may be NULL.
 * After writing parameters directly call ib_mlp_sync_weights.
 */
ib_status ib_mlp_buffers(ib_mlp* mlp, float** params, float** grads, float** adam_m, float** adam_v);
ib_status ib_mlp_sync_weights(ib_mlp* mlp, void* stream);

/*
 * ib_mlp_features -- inputs of n rows: X[i][*] (bfloat16, n_in per row) for
 * the node with linear index nodes_dev[i] (x fastest) of the grid whose FP64
 * SDF is sdf_dev.  Errors: IB_ERR_ARG (ndim differs from the config).
 */
ib_status ib_mlp_features(const ib_mlp* mlp, const ib_grid* grid, const double* sdf_dev,
                          const int64_t* nodes_dev, int64_t n, ib_bc bc, void* X_dev, void* stream);

/* ib_mlp_forward -- Y[n][n_out] (FP32) = network(X[n][n_in] bfloat16). */
ib_status ib_mlp_forward(ib_mlp* mlp, const void* X_dev, int64_t n, float* Y_dev, void* stream);

/*
 * ib_mlp_train_step -- one Adam step (Kingma & Ba) on the mean over rows and
 * outputs of (Y - T)^2 for the minibatch rows idx_dev[0..n) of X (bfloat16
 * [*][n_in]) and T (FP32 [*][n_out]).  The gradient is left in the grads
 * buffer; *loss_dev (device FP32) receives the minibatch loss before the
 * step.  Scratch grows with n and is kept.  Errors: IB_ERR_ARG, IB_ERR_OOM.
 */
ib_status ib_mlp_train_step(ib_mlp* mlp, const void* X_dev, const float* T_dev,
                            const int64_t* idx_dev, int64_t n, float lr, float beta1,
                            float beta2, float eps, float* loss_dev, void* stream);

/*
 * ib_mlp_targets -- training rows from a table built by ib_build_stencils
 * (second-order form): the Laplacian rows fitted at the first support radius
 * and full basis order whose entries all lie on the output footprint.
 * Writes their node indices (nodes_dev, int64) and correction weights in grid
 * units on the footprint (T_dev, FP32 [*][n_out]), at most cap rows, and
 * their count to *n_rows (host).  Synchronises the stream.
 */
ib_status ib_mlp_targets(const ib_table* table, const ib_mlp* mlp, int64_t* nodes_dev,
                         float* T_dev, int64_t cap, int64_t* n_rows, void* stream);

/*
 * ib_build_stencils_learned -- ib_build_stencils (second-order form) in
 * which each IB row first takes the network's prediction and keeps it if its
 * exactness residual is at most accept_tol; the residual is
 * |N^T (A_I^T c - u)| / |u| with A_I the fit's interior rows at the first
 * support radius, u = sum_e w_e a(x_e - x0) and N an orthonormal basis of the
 * null space of the fit's boundary-condition rows (rank threshold 1e-10 of
 * the largest row norm after QR): zero iff the row is exact on every basis
 * polynomial that satisfies the boundary conditions.  Rows whose BC rows
 * have full column rank (no such polynomial: the test would pass vacuously)
 * are not checked.  Rejected and unchecked rows (and rows whose support
 * leaves the footprint) are fitted as in
 * ib_build_stencils, so accept_tol < 0 reproduces its table.
 * Errors: those of ib_build_stencils; IB_ERR_ARG if the form is not
 * second order or the config does not match the grid and options.
 */
ib_status ib_build_stencils_learned(const ib_grid* grid, const double* sdf_dev, ib_bc bc,
                                    const ib_opts* opts, ib_mlp* mlp, double accept_tol,
                                    ib_table** out, void* stream);

/*
 * ib_table_learned -- rows checked against and accepted from the network in
 * ib_build_stencils_learned; resid_host (nullable, [rows of op 0]) receives
 * each row's residual (+inf where the prediction was not applicable, NaN
 * where the table was built without a network).
 */
ib_status ib_table_learned(const ib_table* table, int64_t* n_checked, int64_t* n_accepted,
                           double* resid_host);

/*
 * Measurement hooks (no counterpart in the paper).  ib_profile_enable(stride)
 * resets the per-kernel counters; with stride > 0 every stride-th launch of
 * each time-step kernel is bracketed by CUDA events recorded on its stream.
 * ib_profile_get(i, ...) returns, for the i-th kernel name seen since the
 * reset (0 <= i < ib_profile_count()), its launch count, the number of
 * sampled launches and their summed device time in ms (synchronising on the
 * sampled events).  Setup kernels are counted, not sampled.
 */
ib_status ib_profile_enable(int32_t stride);
int32_t ib_profile_count(void);
ib_status ib_profile_get(int32_t i, char* name, int32_t name_len, int64_t* launches,
                         int64_t* sampled, double* sampled_ms);

/*
 * ib_selftest_bounded_wait -- diagnostics hook (no counterpart in the paper).
 * Runs one kernel that waits on a shared-memory barrier nothing will complete,
 * with the iteration bound the TMA step kernels use.  The wait gives up, the
 * kernel reports it, and the call returns IB_ERR_TIMEOUT with the context still
 * usable -- the path a stalled copy takes in ib_forward.  IB_OK would mean the
 * bound did not work.  Synchronises the stream.
 */
ib_status ib_selftest_bounded_wait(void* stream);

/*
 * ib_sync_status -- synchronise `stream`; IB_ERR_CUDA on a pending device
 * error.  Every forward and adjoint run ends with a pass over its final
 * wavefields (gradients for the adjoint) that sets a per-device status word on
 * a NaN or Inf; this call then returns IB_ERR_UNSTABLE (the scheme blew up
 * for that model and time step) and clears the word.  The word is shared by
 * all streams of the device, so the report names no particular run.
 */
ib_status ib_sync_status(void* stream);

/*
 * ib_stability -- estimate the per-step growth factor of the time stepping
 * with this table's modified operators (the paper gives no stability analysis;
 * its explicit schemes are those of the 2nd-order application section and the
 * 1st-order section).  The modified operators are not symmetric, so their
 * spectrum can leave the interval on which the leapfrog (or staggered) update
 * is neutrally stable.  The call runs the time-step kernels source-free from a
 * random state (SplitMix64 of `seed` and the node index, on interior nodes),
 * renormalising every 50 steps: a power iteration on the one-step map.  It
 * runs n_steps rounded up to an even number of 50-step blocks and returns in
 * *growth the geometric-mean growth per step over the second half, an
 * estimate of the spectral radius of the one-step map (1 for a neutrally
 * stable scheme, > 1 when some mode grows).
 *   shot              its vel_dev, rho_dev (first-order form) and absorbing
 *                     layer are used; sources and receivers are ignored.
 *   precision         32 or 64;  dt the time step of the intended run.
 *   max_gain          IB_ERR_UNSTABLE (with *growth set) when
 *                     growth^n_steps > max_gain, i.e. an unstable mode would
 *                     grow by more than max_gain over a run of n_steps.
 * Synchronises the stream.  Errors: IB_ERR_ARG, IB_ERR_STATE (first-order form
 * in 3D), IB_ERR_OOM, IB_ERR_CUDA, IB_ERR_UNSTABLE.
 */
ib_status ib_stability(const ib_table* table, const ib_shot* shot, int32_t precision,
                       double dt, int32_t n_steps, uint64_t seed, double max_gain,
                       double* growth, void* stream);

/* Thread-local message of the last failure ("" if none). */
const char* ib_last_error(void);

/* Library version string. */
const char* ib_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IB_H */
