/*
 * lattice.h -- C ABI of the GB300 reduced-order Newton / FETI-DP lattice library (liblattice.so).
 *
 * The library implements, on one GPU, the per-Newton-iteration hot path of the reduced-basis
 * solver for neo-Hookean lattice structures of Guillet, Hirschler, Jolivet, Antolin & Bouclier,
 * "Efficient fine-scale simulation of nonlinear hyperelastic lattice structures" (arXiv 2603.10741):
 * per-cell residual and tangent evaluation at quadrature points, the greedy selection of
 * principal cells with their coefficients (Algorithm 1), the reduced tangent action
 * (Eq. romstiffnessmatrix) inside a FETI-DP-preconditioned flexible Krylov solve (Section 3.3),
 * Newton-Raphson with Armijo backtracking (Section 2.2.5) and an adjoint gradient.
 *
 * Conventions (all entry points):
 *  - Every call returns lat_status; no exception crosses the ABI and no kernel traps.  On error,
 *    lattice_last_error() returns a message.  A handle is not thread safe.
 *  - Pointers marked (dev) are device pointers owned by the caller; (host) are host pointers
 *    owned by the caller.  The handle owns every internal workspace.
 *  - Calls are ordered on the handle's CUDA stream; calls that return host values synchronise it.
 *  - Global vectors are FP64, node-major: dof = node * dim + component.
 *  - Cell-stacked local vectors are [n_loc][n_cells]: entry (k, s) at k * n_cells + s, with the
 *    local dof k = local_node * dim + component of the reference cell.
 *  - Local tangent values are stored on the reference cell's sparsity pattern: all local node
 *    pairs (a, b) that share an element, sorted by a then b, each pair a dim x dim block in
 *    row-major (i, j) order: nnz = n_blocks * dim * dim values per cell.  Arrays of such values
 *    are cell-major: [n_cells][nnz].
 */
#ifndef LATTICE_H
#define LATTICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lat_ctx* lat_handle;

typedef enum {
  LAT_OK = 0,
  LAT_EINVAL = 1,          /* bad argument or size */
  LAT_ENOMEM = 2,          /* device allocation failed */
  LAT_ECUDA = 3,           /* CUDA runtime error */
  LAT_ENEG_JACOBIAN = 4,   /* some quadrature point has det F <= 0 */
  LAT_ENOT_CONVERGED = 5,  /* Newton, Armijo or Krylov iteration cap reached */
  LAT_EINDEFINITE = 6,     /* a local remaining-DOF matrix or the coarse matrix is singular (a zero
                              or non-finite pivot; negative pivots are tolerated and trigger the
                              primal enrichment) */
  LAT_ETIMEOUT = 7         /* a bounded device-side wait (tensor-core pipeline) gave up */
} lat_status;

typedef enum {
  LAT_FP64 = 0,        /* everything FP64 */
  LAT_MIXED_FP32 = 1,  /* residual, Newton update, Krylov vectors and operator (the reduced tangent
                          action inside FGMRES), coarse factorisation FP64; preconditioner
                          (local inverses, dual Schur complements, coarse application) FP32;
                          apply_reduced_tangent also accepts FP32 vectors */
  LAT_MIXED_BF16 = 2   /* as FP32, with the local inverse products on the tensor cores: operands as
                          BF16 high/low pairs, FP32 accumulation */
} lat_precision;

/* Lattice description: one reference cell of Q1 elements, repeated by unit translations
 * (Section 2.1, identity macro-map), neo-Hookean material (Eq. sig_eq).  All arrays are host
 * arrays read during lattice_setup only. */
typedef struct {
  int32_t dim;                 /* 2 (plane strain) or 3 */
  int32_t n_cells;             /* N_s */
  int32_t n_nodes_cell;        /* nodes of the reference cell */
  int32_t n_el_cell;           /* Q1 elements of the reference cell */
  int64_t n_glob_nodes;        /* nodes of the lattice */
  const double* X_ref;         /* [n_nodes_cell][dim] reference-cell coordinates, cell in [0,1]^dim */
  const int32_t* elems;        /* [n_el_cell][2^dim] element nodes, Q1 order, positive Jacobian */
  const int32_t* cell_nodes;   /* [n_cells][n_nodes_cell] global node of each local node (A^s) */
  const uint8_t* dof_fixed;    /* [n_glob_nodes*dim] 1 = Dirichlet DOF */
  const double* dirichlet_unit;/* [n_glob_nodes*dim] prescribed value per unit load parameter */
  const double* affine_unit;   /* [n_glob_nodes*dim] first-step predictor per unit load parameter */
  const double* mu_scale;      /* [n_cells] shear-modulus factor theta_s, or NULL for all ones */
  double mu, lam;              /* Lame parameters */
  const int32_t* cell_layer;   /* [n_cells] index of the cell's layer along the load axis, or NULL;
                                  with it the coarse problem is solved through its
                                  block-tridiagonal structure instead of a dense inverse */
} lat_mesh_desc;

typedef struct {
  int64_t n_dof;        /* global DOFs */
  int32_t n_cells;
  int32_t n_loc;        /* local DOFs per cell */
  int32_t n_blocks;     /* node blocks of the local pattern */
  int64_t nnz;          /* values per local tangent */
  int32_t n_r_local;    /* remaining (non-corner) local DOFs */
  int32_t n_p_local;    /* corner (primal) local DOFs */
  int64_t n_primal;     /* free global primal DOFs */
  int64_t n_lambda;     /* Lagrange multipliers */
  int64_t n_krylov;     /* length of a saddle-point vector: n_loc*n_cells + n_primal + n_lambda */
  int32_t n_q_full;     /* quadrature points per cell, full rule */
  int32_t n_q_reduced;  /* quadrature points per cell, reduced (snapshot) rule */
  int32_t n_i_local;    /* remaining DOFs per cell off the cell boundary; the other n_r_local -
                           n_i_local remaining DOFs are the dual (interface) DOFs */
  int32_t n_coarse_blocks; /* diagonal blocks of the block-tridiagonal coarse matrix (cell layers
                              along the load axis), 0 when it is not block tridiagonal */
  int32_t coarse_block;    /* their common padded size */
  int32_t coarse_block_lu; /* 1 when the FP64 coarse solves run as block LU (two sequential
                              sweeps over the blocks, no explicit inverse), 0 when they apply the
                              explicit inverse; set by lattice_prepare_solver */
} lat_sizes;

/* Setup: uploads the reference cell, the maps and the boundary data, builds the local pattern,
 * element colouring, FETI-DP index sets (corners primal, non-redundant multipliers on the other
 * interface DOFs).  stream may be NULL (legacy default stream). */
lat_status lattice_setup(const lat_mesh_desc* desc, lat_precision precision, void* cuda_stream,
                         lat_handle* out);
lat_status lattice_destroy(lat_handle h);
/* The FETI-DP sizes (n_r_local, n_p_local, n_primal, n_lambda, n_krylov) change when
 * newton_step, lattice_prepare_solver or adjoint_gradient enrich the primal set
 * (Section 3.3.2): query them again before sizing saddle-point buffers. */
lat_status lattice_sizes(lat_handle h, lat_sizes* out);
const char* lattice_last_error(lat_handle h);
/* Replace the per-cell shear-modulus factors theta_s (host [n_cells]). */
lat_status lattice_set_mu_scale(lat_handle h, const double* mu_scale);

/* Initial guess of a load step with load parameter `load`: the affine field load*affine_unit
 * when u_prev is NULL, else 2 u_prev - u_prev2 (u_prev2 NULL means 0); then the Dirichlet
 * values load*dirichlet_unit are written.  All (dev) [n_dof]; u_out may alias u_prev. */
lat_status lattice_predictor(lat_handle h, double load, const double* u_prev,
                             const double* u_prev2, double* u_out);

/* Local displacements u^s = A^{sT} u (Eq. residualvector): u_glob (dev) [n_dof] ->
 * x_cells (dev) [n_loc][n_cells]. */
lat_status lattice_gather(lat_handle h, const double* u_glob, double* x_cells);

/* Residual and tangent at quadrature points (Eq. internalloadvec, Section 3.1.4).
 * quad: 0 = full 2^dim Gauss rule per element, 1 = reduced one-point rule (Eq. snapshots).
 * cells (dev) [n_sel] or NULL for all cells (then n_sel must equal n_cells).
 * r_glob (dev) [n_dof] nullable: r = sum_s A^s f^{int,s} over ALL cells (cells must be NULL).
 * f_cells (dev) [n_loc][n_cells] nullable: local internal forces, cell-stacked (cells NULL).
 * K_vals (dev) [n_sel][nnz] nullable: local tangents of the selected cells.
 * min_detF (host) nullable: smallest det F met (evaluated points only).
 * Returns LAT_ENEG_JACOBIAN if some evaluated point has det F <= 0 (outputs then undefined). */
lat_status assemble_residual_tangent(lat_handle h, const double* u_glob, int32_t quad,
                                     const int32_t* cells, int32_t n_sel, double* r_glob,
                                     double* f_cells, double* K_vals, double* min_detF);

/* Algorithm 1 on a caller-provided snapshot matrix T (dev) [n_cols][n_rows] (column s
 * contiguous), FP64.  Stops when max_s ||Delta^s||_inf <= eps or when N_r = min(max_nr, n_cols,
 * n_rows).  Ties of the argmax go to the lowest column.  Outputs: S (dev int32 [max_nr]),
 * n_r (host), alpha (dev [max_nr][n_cols], nullable) from R alpha^s = ||t^s|| beta^s,
 * beta (dev [max_nr][n_cols], nullable), Z (dev [max_nr][n_rows], nullable), and the max
 * residual before each selection plus the final one (host [max_nr+1], nullable). */
lat_status greedy_select(lat_handle h, const double* T, int64_t n_rows, int32_t n_cols, double eps,
                         int32_t max_nr, int32_t* S, int32_t* n_r, double* alpha, double* beta,
                         double* Z, double* max_res);

/* Allocation-free variant of greedy_select, for callers that cannot allocate device memory (a
 * memory arena that owns the device budget, a host application that forbids cudaMalloc/cudaFree,
 * code that cannot create a handle since lattice_setup allocates).  The paper has no counterpart
 * of this entry point.  Same arguments and results as greedy_select for
 * T, n_rows, n_cols, eps, max_nr, S, n_r, alpha, with no handle: the work runs on cuda_stream
 * (NULL = legacy default stream).  All workspace lives in one file-scope device array of
 * 16 MiB (2 Mi doubles) that every device loading the library holds until process exit; it
 * must fit Delta (n_cols * n_rows), Z (min(max_nr, n_cols, n_rows) * n_rows), beta and a few
 * per-column vectors, else LAT_EINVAL is returned before any work.  No cudaMalloc, cudaFree or
 * allocating library call is made.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress with that device current), so make that first call before any
 * stream capture.  Every call reuses the same array (its state is reset at the start of each
 * call); calls that overlap on the GPU, from any stream or thread, race and must be avoided. */
lat_status greedy_select_static(const double* T, int64_t n_rows, int32_t n_cols, double eps, int32_t max_nr,
                                int32_t* S, int32_t* n_r, double* alpha, void* cuda_stream);

/* Principal cells for state u_glob (dev): snapshots with the reduced rule for all cells,
 * Algorithm 1 with tolerance eps, coefficients alpha (Section 3.2.2), then the principal
 * tangents K^r = K^{s_r}(u^{s_r}) with the full rule (Eq. reducedbasis).  force_all != 0 skips
 * the greedy: every cell is principal with alpha = I.  The selection is kept in the handle for
 * apply_reduced_tangent and the solver.  Outputs (nullable): S (dev int32 [n_cells]), n_r (host),
 * alpha (dev [n_r][n_cells]; ignored when force_all), K_p (dev [n_r][nnz]). */
lat_status select_principal_cells(lat_handle h, const double* u_glob, double eps, int32_t max_nr,
                                  int32_t force_all, int32_t* S, int32_t* n_r, double* alpha,
                                  double* K_p);

/* Snapshot kind of select_principal_cells (newton_step and adjoint_gradient take it from their
 * options): 0 the reduced-rule local tangents' data (Eq. snapshots), 1 the pulled-back tangent
 * tensor D^ref_ijmn = |det J| sum_kl D_ijkl (J^-1)_mk (J^-1)_nl, J = dx/dxi = F J0, at the
 * one-point rule of every element (Eq. tensorfunctionPulledback, the Remark after Eq.
 * snapshots), entries ordered (element, i, j, m, n).  LAT_EINVAL for another kind. */
lat_status lattice_set_snapshots(lat_handle h, int32_t kind);

/* Caller-given principal set for the reduced tangent action (Eq. romstiffnessmatrix with S and
 * alpha chosen by the caller instead of by Algorithm 1; the paper has no such entry point, its
 * principal set always comes from the greedy).  u_glob (dev, FP64 [n_dof]): state at which the
 * principal tangents K^r are evaluated (full rule).  S (dev, int32 [n_r]): principal cell
 * indices in [0, n_cells).  alpha (dev, FP64 [n_r][n_cells]): coefficients.  All three are
 * caller-owned and read during the call.  Afterwards apply_reduced_tangent uses this set
 * (newton_step, lattice_prepare_solver and adjoint_gradient run their own selection).
 * Errors: LAT_EINVAL (null pointer, n_r outside [1, n_cells], an index out of range),
 * LAT_ENEG_JACOBIAN (det F <= 0 in a principal cell). */
lat_status set_principal_cells(lat_handle h, const double* u_glob, const int32_t* S, int32_t n_r,
                               const double* alpha);

/* Reduced tangent action Y[:, s] = sum_r alpha_r^s K^r X[:, s] (Eq. romstiffnessmatrix) on
 * cell-stacked vectors (dev) [n_loc][n_cells] of type dtype (0 = FP64, 1 = FP32) with the
 * selection held by the handle (FP32 uses FP32 copies of K^r and alpha). */
lat_status apply_reduced_tangent(lat_handle h, const void* x_cells, void* y_cells, int32_t dtype);

typedef struct {
  double eps;              /* greedy tolerance (Algorithm 1) */
  int32_t max_nr;          /* cap on principal cells per iteration */
  int32_t force_all;       /* 1: every cell principal (the plain full-tangent path) */
  double newton_rtol;      /* stop when ||r_F|| / ||r_F(u^0)|| <= newton_rtol */
  int32_t newton_max_it;
  double krylov_rtol;      /* FGMRES relative residual target */
  int32_t krylov_max_it;   /* total FGMRES iterations per solve */
  int32_t krylov_restart;
  int32_t pcg_iters;       /* cap on PCG iterations of the interface sub-preconditioner */
  int32_t armijo_max_m;    /* backtracking cap */
  double pcg_rtol;         /* interface PCG stops when sqrt(r^T M r / r0^T M r0) <= pcg_rtol
                              (0: always pcg_iters iterations) */
  int32_t interface_precond; /* M of the interface PCG: 0 Dirichlet B_D S_DD B_D^T with the local
                                dual Schur complements of the principals, 1 lumped B_D K_DD B_D^T */
  int32_t max_enrich;      /* cap on the primal enrichment level (Section 3.3.2): when a
                              principal's remaining block is not positive definite, primal
                              nodes are added on every cell edge (level L: the nodes nearest to
                              the points j/2^L of each edge) for all cells, and kept */
  int32_t coarse_block_lu; /* coarse solves of a block-tridiagonal coarse matrix: 1 block LU in
                              FP64 (two sequential sweeps over the cell layers, factors N m^3,
                              no explicit inverse; a sweep step is one thread-block cluster for
                              blocks up to 512 rows, for larger ones the whole solve as one
                              cooperative launch over the whole GPU with a grid-wide barrier
                              between steps), 2 block LU with one whole-GPU launch per step at
                              any block size, 4 block LU as the single cooperative launch at any
                              block size, 3
                              block LU with the cluster sweeps in the forms taken when larger
                              blocks do not fit (8-CTA clusters, block rows read from global
                              memory instead of prefetched), 0 the
                              explicit inverse (N^2 m^3 to build, one dense product per solve;
                              FP32 copy in the mixed modes), -1 (default) block LU when the
                              explicit inverse would hold more than 8192^2 entries (N blocks of
                              size m, N m > 8192) */
  int32_t precond_tangent; /* principal tangents the preconditioner's local blocks are built from:
                              0 the full tangent K^r (Section 3.1.4), 1 its material part (the
                              geometric stress term delta_ij sigma_kl of D dropped: positive
                              definite local blocks whatever the prestress), -1 (default) 1 in 3D,
                              0 in 2D.  The Krylov operator always uses the full reduced tangent,
                              so the choice changes iteration counts, not the solution */
  int32_t min_enrich;      /* primal enrichment level to start from (0 = corners only); the
                              level only grows (Section 3.3.2) */
  int32_t inner_its;       /* mixed modes: > 0 makes FGMRES's preconditioner an inner flexible
                              GMRES of at most inner_its iterations on the same saddle-point
                              system with the FP32 reduced tangent action as its operator and the
                              block preconditioner of Eq. (ifetidp_precond) as its preconditioner;
                              the outer FGMRES keeps the FP64 operator, so the solution is that of
                              the FP64 reduced tangent.  0: the block preconditioner directly.
                              Ignored in LAT_FP64 */
  double inner_rtol;       /* inner GMRES stops early at this relative residual */
  int32_t snapshot;        /* snapshots fed to Algorithm 1: 0 (default) the data of the
                              reduced-rule local tangents (Eq. snapshots), 1 the pulled-back
                              tangent tensor D^ref (Eq. tensorfunctionPulledback) at the
                              one-point rule of every element (the Remark after Eq. snapshots:
                              n_el d^4 values per cell instead of nnz) */
  int32_t eps_refine;      /* greedy tolerance tightenings per call (newton_step and
                              adjoint_gradient), each dividing eps by 10 and kept for the rest of
                              the call: when the line search finds no acceptable step along the
                              reduced-tangent direction (the iteration is then repeated from the
                              same iterate), when two accepted Newton steps in a row each reduce
                              ||r_F|| by less than the factor eps_refine_rate, and when an
                              adjoint defect correction does (the reduced tangent then limits
                              the linear convergence).  0: eps is fixed and a rejected direction
                              ends the call with an error */
  double eps_refine_rate;  /* contraction factor of that test (default 0.5) */
} lat_newton_opts;

typedef struct {
  int32_t iterations;      /* Newton iterations taken by this call */
  int32_t converged;
  double r0_norm;          /* ||r_F|| at entry (the reference of the relative test) */
  double r_norm;           /* ||r_F|| at exit */
  int32_t n_r_last;        /* principal cells in the last iteration */
  int32_t krylov_its_total;
  int32_t armijo_m_max;
  double t_residual_ms, t_select_ms, t_setup_ms, t_krylov_ms, t_linesearch_ms; /* phase times */
  int32_t pcg_its_total;   /* interface PCG iterations inside the preconditioner */
  int32_t enrich_level;    /* primal enrichment level in use at exit */
  int32_t inner_its_total; /* inner FP32-operator GMRES iterations (mixed modes, inner_its > 0) */
  int32_t eps_refinements; /* greedy tolerance tightenings of this call (eps_refine) */
  double eps_last;         /* greedy tolerance in use at exit */
} lat_newton_report;

/* Default options (eps 3e-4 in 2D and 5e-3 in 3D, max_nr 256, newton_rtol 1e-8, krylov_rtol
 * 1e-10 for FP64 and 1e-6 for the mixed modes, restart 60, interface PCG to 3e-2 with at most 100
 * iterations, Armijo cap 30, Dirichlet interface preconditioner, enrichment up to level 3,
 * preconditioner from the full tangent in 2D and from its material part in 3D, starting
 * enrichment level 0; in the mixed modes an inner FP32-operator GMRES of at most 20 iterations
 * to 1e-2 as FGMRES's preconditioner; up to 2 tenfold tolerance tightenings per call, on
 * rejected directions or a contraction above 0.5). */
lat_status lattice_default_opts(lat_handle h, lat_newton_opts* opts);

/* Newton-Raphson for one load step (Section 2.2.5) from the initial guess in u_glob (dev,
 * in/out, Dirichlet values already set): residual, principal selection, FETI-DP setup,
 * FGMRES on the saddle-point system with the reduced tangent, Armijo line search (beta = 1/2,
 * c = 1e-4), update; until ||r_F||/||r_F(u^0)|| <= newton_rtol.  A rejected direction (no
 * acceptable step within armijo_max_m halvings) repeats the iteration with a tighter greedy
 * tolerance while opts->eps_refine allows, else the call returns LAT_ENOT_CONVERGED with u_glob
 * unchanged from its last accepted iterate.  max_iterations > 0 limits the iterations of this
 * call (a call with max_iterations = 1 runs exactly one iteration). */
lat_status newton_step(lat_handle h, double* u_glob, int32_t max_iterations,
                       const lat_newton_opts* opts, lat_newton_report* report);

/* Adjoint gradient of the end compliance J = sum_D u_D f_D(u) with respect to the per-cell
 * shear-modulus factors theta_s at a converged state u_glob (dev):
 *   K_FF lambda = K_FD u_D,  dJ/dtheta_s = w^T A^s f_mu^s(u^s),  w = [-lambda; u_D].
 * The adjoint system is solved by defect correction: the exact tangent action (matrix free) for
 * the defect, the reduced FETI-DP FGMRES solve as the correction.  grad (dev) [n_cells],
 * J (host) nullable, report (host) nullable. */
lat_status adjoint_gradient(lat_handle h, const double* u_glob, const lat_newton_opts* opts,
                            double* grad, double* J, lat_newton_report* report);

/* FETI-DP pieces on saddle-point vectors (dev) [n_krylov] = [local part n_loc*n_cells |
 * primal n_primal | multipliers n_lambda] (Section 3.3.1), with the current selection:
 *  mode 0: w = A v, the saddle-point operator [K~ B^T; B 0]
 *  mode 1: w = K~^{-rom} v on the displacement part (multiplier part copied)
 *  mode 2: w = the block preconditioner of Eq. (ifetidp_precond) applied to v
 * Requires a prior select_principal_cells and newton setup via lattice_prepare_solver. */
lat_status feti_apply(lat_handle h, int32_t mode, const double* v, double* w);
/* Solve the tangent system K~ x = rhs (the partially assembled reduced tangent of the current
 * selection, Eq. linsys with the operator of Eq. romstiffnessmatrix) by FGMRES on the FETI-DP
 * saddle point of Section 3.3.1 with the preconditioner of Eq. (ifetidp_precond).  rhs and x are
 * global (dev) [n_dof]; Dirichlet entries of rhs are ignored and x is 0 there.  Requires
 * select_principal_cells and lattice_prepare_solver.  iters, rel (host, nullable): FGMRES
 * iterations and final relative residual of the saddle-point system. */
lat_status tangent_solve(lat_handle h, const double* rhs, double* x, const lat_newton_opts* opts,
                         int32_t* iters, double* rel);
/* Build the FETI-DP preconditioner for the current selection at state u_glob. */
lat_status lattice_prepare_solver(lat_handle h, const double* u_glob, const lat_newton_opts* opts);
/* Map a saddle-point vector's displacement part to a global vector (mean over copies). */
lat_status feti_to_global(lat_handle h, const double* v, double* u_glob);
/* Map a global vector to the saddle-point layout (copies on every cell, multipliers 0). */
lat_status feti_from_global(lat_handle h, const double* u_glob, double* v);

/* Kernel timing: while enabled, CUDA events are recorded on the handle's stream around every
 * launch of the named kernels ("residual", "tangent_full", "tangent_material",
 * "tangent_reduced", "greedy_update", "apply_reduced" / "apply_reduced_fp32", "apply_percell" /
 * "apply_percell_fp32", "local_segmm", "local_gemv", "local_tc" and their "_dual" / "_dual_in"
 * variants inside the interface solve, "dual_schur" / "dual_schur_tc", "gj_update", "gj_pivot", "densify",
 * "phi_schur", "coarse_blocked", "coarse_gemv", "coarse_solve", "krylov_orth").  enable = 1
 * times every named kernel; the interface PCG iteration then runs launch by launch instead of
 * as a CUDA-graph replay, so that every launch is timed.  enable = 2 times only the tangent
 * action kernels ("apply_*") and keeps the graph replays.  lattice_set_timing clears the
 * records; lattice_kernel_time returns the summed duration (host ms) and the launch count of
 * one name since then. */
lat_status lattice_set_timing(lat_handle h, int32_t enable);
lat_status lattice_kernel_time(lat_handle h, const char* name, double* total_ms, int32_t* launches);

/* Number of kernels launched through this handle since it was created. */
lat_status lattice_launch_count(lat_handle h, int64_t* launches);

/* Load-step checkpoint: the step index, the load parameter and the last two converged states
 * (dev [n_dof]; u_prev may be NULL) to/from a binary file. */
lat_status lattice_checkpoint_save(lat_handle h, const char* path, int32_t step, double load,
                                   const double* u, const double* u_prev);
lat_status lattice_checkpoint_load(lat_handle h, const char* path, int32_t* step, double* load,
                                   double* u, double* u_prev);

#ifdef __cplusplus
}
#endif
#endif /* LATTICE_H */
