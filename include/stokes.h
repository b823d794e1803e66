/*
 * stokes.h - C ABI of a GB300 (sm_103a) solver for the generalized Stokes
 * saddle-point system from P2-P1 Taylor-Hood elements on Kuhn tetrahedral
 * meshes of the unit cube (Creff & Guermond, arXiv 2407.01783).
 *
 * The discrete problem (Sec. 2.2, Eq. Saddle_point_A_BT_B, with a pressure
 * load g added):
 *     A U - B^T P = F,   B U = g,   int p_h = 0,
 *     A = M_V/dt + mu E_V  (Eq. for A_ij; E_V from 2 eps(u):eps(v)),
 *     B_kj = int psi_k div phi_j  (Eq. def_of_Aij_Bij),
 * optionally in augmented-Lagrangian form A_gamma = A + gamma mu B^T M_Q^{-1} B
 * (Eqs. LA_problem, def_of_Alambda; the paper's lambda is gamma here).
 *
 * Solvers (Sec. 2.3 and 2.4): Method 1 = conjugate gradients on the pressure
 * Schur complement S = B A^{-1} B^T preconditioned by the Cahouet-Chabard
 * operator C^Lambda = mu(1+gamma) M_Q^{-1} + dt^{-1} (B Lambda_V^{-1} B^T)^{-1}
 * (or C^Delta with L_Q in place of B Lambda_V^{-1} B^T; Eqs.
 * Schur_complement_preconditioners); Method 2 = FGMRES on the coupled system
 * with the block-LU preconditioner of Eq. inexact_factorization_of_Alambda
 * (or its block-triangular variant, Remark "Alternative preconditioner").
 * Velocity solves are preconditioned by V-cycles on A~_3 = M_V/dt + mu L_V
 * (Eq. precond_A_plus_lambda_D_3).
 *
 * Conventions for every entry point:
 *  - Mesh: n^3 cubes, each split into 6 tetrahedra (one per axis permutation).
 *    Vertices are (n+1)^3 rows of 3 doubles, lexicographic, x fastest.
 *  - P2 nodes: the (2n+1)^3 half-grid, lexicographic, x fastest; velocity
 *    fields are node-interleaved [(2n+1)^3][3]. P1 (pressure) fields are
 *    [(n+1)^3].
 *  - Device pointers live in the CUDA context current when stokes_setup was
 *    called and are used on the stream given there. Functions ending in
 *    _host take host pointers instead and copy inside the call.
 *  - The caller owns every array it passes; the context owns all matrices
 *    and work space and frees them in stokes_destroy.
 *  - Every call returns a stokes_status; none aborts, traps or prints. On
 *    error, stokes_last_error() describes the cause (per thread).
 *  - A context is used by one host thread at a time; separate contexts may
 *    run concurrently (own streams, own host threads).
 *  - With options.graphs = 1 a context records its V-cycles (and C, when its
 *    inner solve has a fixed iteration count) into CUDA graphs the second
 *    time it meets the same buffers, on a private stream, and replays them
 *    on its stream afterwards; results are bitwise those of plain launches.
 */
#ifndef STOKES_H
#define STOKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stokes_ctx stokes_ctx;

typedef enum {
  STOKES_OK = 0,
  STOKES_ERR_ARG = -1,             /* bad argument (size, pointer, option) */
  STOKES_ERR_OOM = -2,             /* device allocation failed */
  STOKES_ERR_CUDA = -3,            /* a CUDA runtime call failed */
  STOKES_ERR_NOT_CONVERGED = -4,   /* iteration cap hit; best iterate written */
  STOKES_ERR_BREAKDOWN = -5,       /* Krylov breakdown (p^T A p <= 0 etc.) */
  STOKES_ERR_NAN = -6,             /* non-finite value in a residual */
  STOKES_ERR_TIMEOUT = -7,         /* a bounded device wait expired */
  STOKES_ERR_INCOMPATIBLE_RHS = -8,/* sum(g) != 0: B U = g has no solution */
  STOKES_ERR_MESH = -9             /* inverted or degenerate tetrahedron */
} stokes_status;

enum { STOKES_METHOD_SCHUR = 0, STOKES_METHOD_COUPLED = 1 };
/* Schur-complement preconditioner (Eq. Schur_complement_preconditioners):
 * C^Lambda (lumped velocity mass, the paper's recommendation), C^Delta
 * (pressure Laplacian) or C_lambda (B M_V^{-1} B^T, with M_V^{-1} by
 * mass_steps_v Chebyshev-Jacobi steps on the P2 mass). */
enum { STOKES_SCHUR_PREC_LUMPED = 0, STOKES_SCHUR_PREC_LAPLACE = 1, STOKES_SCHUR_PREC_MASS = 2 };
/* FP64 everywhere, or FP32 matrices/multigrid/inner Krylov with FP64 outer
 * refinement, dot products, pressure-mean projection and coarse factors. */
enum { STOKES_PRECISION_FP64 = 0, STOKES_PRECISION_MIXED = 1 };

typedef struct {
  int method;            /* STOKES_METHOD_* */
  int schur_prec;        /* STOKES_SCHUR_PREC_* */
  int precision;         /* STOKES_PRECISION_* */
  int vcycles;           /* V-cycles per A~_3^{-1} application ("2Vc": 2) */
  int cheb_degree;       /* Chebyshev-Jacobi steps per pre/post smoothing */
  int mass_steps;        /* Chebyshev steps for (M_Q)^{-1} inside C */
  int mass_steps_al;     /* Chebyshev steps for M_Q^{-1} inside A_gamma */
  int restart;           /* FGMRES restart length (Method 2) */
  int block_lu;          /* Method 2: 1 full block-LU, 0 block-triangular */
  int m2_inner_cg;       /* Method 2: 1 = A~^{-1} by PCG to inner_tol, 0 = V-cycles */
  double inner_tol;      /* relative tolerance of inner velocity solves */
  double schur_inner_tol;/* relative tolerance of the pressure-operator solve in C */
  double eps_pressure;   /* eps of eps M_Q + L_Q (the paper uses 1) */
  int max_outer;         /* outer Krylov iterations per refinement pass */
  int max_inner;         /* inner Krylov iterations per solve */
  int max_refine;        /* refinement passes on the full FP64 residual */
  int profile;           /* 1: count launches and time every kernel class with CUDA
                            events; 2 + k: count all, time only class k
                            (STOKES_KERNEL_*); 0: off */
  int spmv_group;        /* threads per sparse row: 0 autotune, else 1..32 */
  int schur_inner_iters; /* > 0 (default 2): the solve inside C runs exactly this
                            many PCG iterations with no convergence test (no
                            host synchronisation; the outer CG is flexible);
                            0: stop at schur_inner_tol */
  double pass_tol;       /* mixed precision: relative reduction asked of each FP32
                            correction pass (outer Krylov tolerance per pass);
                            its inner velocity solves get max(inner_tol,
                            pass_tol/30). Default 3e-2. */
  int format;            /* 0: stencil-structured storage for A~_3, eps M_Q + L_Q,
                            M_Q, L_Q on levels with >= 2^18 rows, CSR below; the
                            strain-form A in symmetric stencil storage (diagonal
                            and upper 3x3 blocks only: half the matrix bytes)
                            for its products and the double-float refinement
                            residual;
                            1: CSR everywhere (A as BSR3, CSR of 3x3 blocks);
                            2: stencil storage on every level, A as in 0;
                            3: as 0 but the products of A from BSR3 (the
                            refinement residual still symmetric) */
  int graphs;            /* 1 (default): V-cycles, and C when schur_inner_iters
                            > 0, are recorded into CUDA graphs on a private
                            stream the second time the same buffers come by and
                            replayed on the context's stream afterwards (while
                            finest-level launches are timed per class, only
                            levels >= 1 are); 0: plain launches */
  int vel_prec;          /* velocity preconditioner inside A^{-1} solves and the
                            block preconditioners (Sec. 5.1, Eqs.
                            precond_A_plus_lambda_D_1..3): 3 (default) A~_3 =
                            M_V/dt + mu L_V, one scalar V-cycle per component;
                            2: A~_2 = A; 1: A~_1 = A + gamma mu D (D the
                            grad-div matrix); 1 and 2 run a V-cycle on the 3x3
                            block operator (re-assembled on every level,
                            point-Jacobi Chebyshev smoothing) */
  int mass_steps_v;      /* Chebyshev-Jacobi steps for (M_V)^{-1} inside C_lambda
                            (schur_prec = STOKES_SCHUR_PREC_MASS) on the exact
                            P2 interval [1/4, 4.3475]: 8 (default, the paper's
                            economical "2Vc" reading) ... 48 (~1e-10, "th") */
  int coarse_kernel;     /* 1: the levels below the finest of each V-cycle of
                            A~_3 and eps M_Q + L_Q run in one cooperative
                            kernel (grid-wide barriers between the steps,
                            bounded waits: STOKES_ERR_TIMEOUT if one expires);
                            0 (default): one launch per step, replayed from a
                            CUDA graph (faster on GB300 at 48^3: the barriers
                            cost more than the launches they replace) */
  int pass_schedule;     /* defect-correction schedule: 0 (default) = 1 for mixed
                            precision, 2 for FP64; 1 = passes that each ask for a
                            reduction of pass_tol with inner velocity solves at
                            max(inner_tol, pass_tol/30); 2 = one pass aimed
                            straight at tol with inner solves at inner_tol (the
                            paper's setting) */
  double cheb_low;       /* Chebyshev-Jacobi smoothing interval [cheb_low, */
  double cheb_high;      /* cheb_high] x the Lanczos estimate of
                            lambda_max(D^{-1} M) on every level (the paper
                            names the smoother only): 0.1 and 1.1 by default.
                            An interval far below the spectrum makes the
                            V-cycle indefinite; the Krylov solvers then report
                            STOKES_ERR_BREAKDOWN. */
  int sym_batch;         /* symmetric A products: block entries whose loads one
                            thread issues before using them (2, 4 or 8; 0:
                            default 8) */
  int stencil_min_rows;  /* formats 0 and 3: levels with at least this many rows
                            use stencil storage (0: 2^18) */
  int host_wait;         /* how the host thread waits for the device scalars
                            it reads: 0 spins (lowest latency; the default),
                            1 sleeps until the GPU signals (blocking-sync
                            events: the better choice when more solver threads
                            than host cores wait at once, as in a batch) */
  int vcycle_split;      /* parity-split node numbering (each x-line's even and
                            odd nodes stored apart, so stencil gathers are
                            contiguous; the cycle's result is bitwise the
                            same) on the stencil-stored finest level of the
                            velocity V-cycles: 1 (default) in the lockstep
                            (several right-hand-side, node-interleaved)
                            cycles, 2 in every cycle, 0 never. With one
                            right-hand side the renumbering passes cost more
                            than the faster gathers save (measured at 48^3) */
} stokes_options;

typedef struct {
  int outer_iters;       /* outer Krylov iterations, summed over passes */
  int inner_iters;       /* inner Krylov iterations, summed */
  int refinements;       /* passes on the full residual */
  int status;            /* stokes_status of the solve */
  double rel_residual;   /* ||[F - A U + B^T P; g - B U]|| / ||[F; g]|| (FP64) */
  double solve_ms;       /* wall time of the call (host clock) */
} stokes_info;

/* Fill *opt with the defaults: Method 1, C^Lambda, FP64, 2 V-cycles, degree 2
 * Chebyshev, 8 mass steps, inner tolerance 1e-10 (the paper's Sec. 3.1). */
void stokes_default_options(stokes_options* opt);

/* Build every operator for one mesh and (mu, dt, gamma): element-coloured
 * assembly on the device, multigrid hierarchy n -> n/2 -> ... , smoother
 * spectra, coarse factors. `vertices` is a HOST array [(n+1)^3][3]; n >= 2.
 * `stream` is a cudaStream_t (NULL = legacy default stream). mu, dt > 0,
 * gamma >= 0. Returns STOKES_ERR_MESH if a jittered tetrahedron is inverted.
 * On success *out owns all device memory of the solver. */
stokes_status stokes_setup(int n, const double* vertices, double mu, double dt,
                           double gamma, const stokes_options* opt,
                           void* stream, stokes_ctx** out);

/* Solve for (u, p). f: device [(2n+1)^3][3] nodal body force (the load is
 * F = M_V f_h on interior rows). g: device [(n+1)^3] pressure load or NULL
 * (zero); sum(g) must vanish (else STOKES_ERR_INCOMPATIBLE_RHS). tol: target
 * for the true relative residual of the full system. u: device
 * [(2n+1)^3][3] (boundary rows written as 0). p: device [(n+1)^3] with
 * int p_h = 0. info may be NULL. */
stokes_status stokes_solve(stokes_ctx* ctx, const double* f, const double* g,
                           double tol, double* u, double* p, stokes_info* info);

/* k systems with the same operator (Eq. Saddle_point_A_BT_B, k right-hand
 * sides): f device [k][(2n+1)^3][3], g device [k][(n+1)^3] or NULL, u device
 * [k][(2n+1)^3][3], p device [k][(n+1)^3], info NULL or an array of k. The
 * systems are solved four at a time in lockstep, each with its own Krylov
 * coefficients and convergence test (Method 1: flexible Schur CG of Sec. 2.3
 * with lockstep inner PCG; Method 2: FGMRES of Sec. 2.4 with its own basis
 * and Hessenberg matrix per system): every V-cycle, Chebyshev mass inverse,
 * product with A, B or B^T and vector kernel sweeps its matrix and launches
 * once for the four systems. A last group of two or three systems is padded
 * with zero systems; a single one takes the stokes_solve path. Each system
 * meets tol on its own full residual (info[i].rel_residual);
 * info[i].outer_iters counts the outer iterations system i took part in,
 * info[i].inner_iters the lockstep inner iterations of its group.
 * Returns STOKES_OK if every system converged, else the first failing status.
 * A following stokes_adjoint uses the last system's solution.
 * 1 <= k <= 4096. */
stokes_status stokes_solve_multi(stokes_ctx* ctx, int k, const double* f, const double* g,
                                 double tol, double* u, double* p, stokes_info* info);

/* Same as stokes_solve with HOST arrays; the host<->device copies are part
 * of the call. */
stokes_status stokes_solve_host(stokes_ctx* ctx, const double* f, const double* g,
                                double tol, double* u, double* p, stokes_info* info);

/* Adjoint of stokes_solve for J(u, p): given dJ/du (device [(2n+1)^3][3],
 * boundary rows ignored) and dJ/dp (device [(n+1)^3] or NULL), solve the
 * transposed saddle system K^T [lu; lp] = [dJ/dU; dJ/dP] and return
 * dJ/df (device [(2n+1)^3][3], = M_V^T lu spread to all nodes), dJ/dg
 * (device [(n+1)^3] or NULL) and dJ/dmu (host scalar, = -lu^T E_V U for the
 * (U, P) of the last stokes_solve). Requires a prior stokes_solve. */
stokes_status stokes_adjoint(stokes_ctx* ctx, const double* dJdu, const double* dJdp,
                             double tol, double* dJdf, double* dJdg, double* dJdmu,
                             stokes_info* info);

/* Release everything owned by ctx (NULL is accepted). */
stokes_status stokes_destroy(stokes_ctx* ctx);

/* Static description of a status code. */
const char* stokes_status_string(int status);
/* Message of the last failing call on this host thread ("" if none). */
const char* stokes_last_error(void);

/* ---- operator access: building blocks of the solve, for tests and tools ----
 * Operators act on REDUCED vectors: velocity = interior P2 nodes stored
 * component-major [3][(2n-1)^3] (the solver's internal layout: component c of
 * interior node i at c*(2n-1)^3 + i), pressure = [(n+1)^3]. x and y are device
 * arrays of the operator's column / row length. `level` selects a multigrid
 * level (0 = the mesh given to setup) where it applies, else must be 0. */
typedef enum {
  STOKES_OP_A = 0,            /* y = A x (strain form, 3x3 blocks)            */
  STOKES_OP_A3 = 1,           /* y = A~_3 x per component (any level)         */
  STOKES_OP_B = 2,            /* y = B x    (velocity -> pressure)            */
  STOKES_OP_BT = 3,           /* y = B^T x  (pressure -> velocity)            */
  STOKES_OP_MQ = 4,           /* y = M_Q x                                    */
  STOKES_OP_LQ = 5,           /* y = L_Q x                                    */
  STOKES_OP_KQ = 6,           /* y = (eps M_Q + L_Q) x  (any level)           */
  STOKES_OP_LUMPED_INV = 7,   /* y = Lambda_V^{-1} x                          */
  STOKES_OP_VCYCLE_A3 = 8,    /* y = vcycles V-cycles for A~_3 from 0 (level) */
  STOKES_OP_VCYCLE_KQ = 9,    /* y = one V-cycle for eps M_Q + L_Q from 0     */
  STOKES_OP_SCHUR_PREC = 10,  /* y = C x (C^Lambda or C^Delta per options)    */
  STOKES_OP_SCHUR = 11,       /* y = B A^{-1} B^T x with the inner PCG        */
  STOKES_OP_AGAMMA = 12,      /* y = A x + gamma mu B^T M_Q^{-1} B x           */
  STOKES_OP_PROLONG_P2 = 13,  /* y(level) = P x(level+1), 3 components         */
  STOKES_OP_RESTRICT_P2 = 14, /* y(level+1) = P^T x(level)                     */
  STOKES_OP_PROLONG_P1 = 15,  /* y(level) = P x(level+1)                       */
  STOKES_OP_LOAD = 16,        /* y = M_V f on interior rows, x = nodal f on all
                                 nodes [(2n+1)^3][3] (node-interleaved)       */
  STOKES_OP_A_DF = 17,        /* y = A x as the mixed-precision refinement
                                 residual computes it: FP32 hi/lo pairs of A
                                 and x, exact FP32 products, double-float sums
                                 (mixed-precision contexts only)              */
  STOKES_OP_VCYCLE_VEL = 18   /* y = the configured velocity preconditioner
                                 (vcycles V-cycles of A~_{vel_prec}) applied
                                 to x, from level 0                          */
} stokes_op;

stokes_status stokes_apply(stokes_ctx* ctx, int op, int level, const double* x, double* y);

/* y = A x + gamma mu B^T M_Q^{-1} B x without allocating any device memory.
 * The paper has no counterpart: this exists for callers that must not call
 * cudaMalloc once they are running (a host loop that owns a fixed device
 * memory budget, or code running while another framework owns the device
 * allocator). Same arithmetic and result as stokes_apply(ctx,
 * STOKES_OP_AGAMMA, 0, x, y); x and y are device arrays [3][(2n-1)^3] on the
 * stream given to stokes_setup, and the call returns after that stream has
 * finished the work.
 * Work space: one fixed array of 4 x 2^20 doubles (32 MiB) that every GPU
 * loading this library holds until the process exits. Meshes with more than
 * 2^20 pressure nodes (n > 100) are rejected with STOKES_ERR_ARG. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture. All calls
 * share the array and leave their data in it; the call overwrites every entry
 * it reads, so nothing needs clearing, but calls whose kernels overlap on the
 * GPU (other streams or threads at the same time) race on it. */
stokes_status stokes_apply_agamma_noalloc(stokes_ctx* ctx, const double* x, double* y);

/* Assembled matrices, for checks against an independent assembly. */
typedef enum {
  STOKES_MAT_A = 0,    /* BSR 3x3, interior P2 x interior P2                 */
  STOKES_MAT_A3 = 1,   /* scalar, interior P2 (any level)                     */
  STOKES_MAT_B = 2,    /* 1x3 blocks, P1 x interior P2                        */
  STOKES_MAT_BT = 3,   /* 3x1 blocks, interior P2 x P1                        */
  STOKES_MAT_MQ = 4, STOKES_MAT_LQ = 5,
  STOKES_MAT_KQ = 6,   /* any level */
  STOKES_MAT_LUMPED = 7,/* diagonal Lambda_V per interior P2 node (rows=cols) */
  STOKES_MAT_AV = 8    /* BSR 3x3 velocity preconditioner A~_1 / A~_2 (any
                          level; vel_prec 1 or 2 only)                       */
} stokes_matrix;

/* dims = {rows, cols, nnz (blocks), block_rows, block_cols}. */
stokes_status stokes_matrix_shape(stokes_ctx* ctx, int which, int level, int64_t dims[5]);
/* Copy CSR arrays to HOST buffers sized from stokes_matrix_shape: rowptr
 * [rows+1], colidx [nnz], vals [nnz*block_rows*block_cols] (row-major blocks).
 * For STOKES_MAT_LUMPED only vals [rows] is written. */
stokes_status stokes_matrix_export(stokes_ctx* ctx, int which, int level,
                                   int32_t* rowptr, int32_t* colidx, double* vals);

/* Problem sizes: {n, levels, interior P2 nodes, P1 nodes, all P2 nodes, dofs}. */
stokes_status stokes_sizes(stokes_ctx* ctx, int64_t sizes[6]);

/* Per-kernel statistics (options.profile != 0): kernel ids are STOKES_KERNEL_*.
 * Returns all launches (graph replays included), the summed CUDA-event
 * milliseconds of the timed ones and the algorithmic bytes of all launches
 * (matrix read once, each vector read/written once) since the last reset. */
typedef enum {
  STOKES_KERNEL_SPMM_A3 = 0,      /* A~_3 x 3 RHS on the finest level (smoother/residual) */
  STOKES_KERNEL_SPMV_A = 1,       /* BSR3 strain-form A                     */
  STOKES_KERNEL_B = 2,            /* divergence B                           */
  STOKES_KERNEL_BT = 3,           /* gradient B^T                           */
  STOKES_KERNEL_SPMV_P1 = 4,      /* P1 CSR (M_Q, L_Q, eps M_Q + L_Q)       */
  STOKES_KERNEL_TRANSFER = 5,     /* prolongation / restriction             */
  STOKES_KERNEL_BLAS1 = 6,        /* dots, axpys, projections               */
  STOKES_KERNEL_OTHER = 7,        /* load vectors, coarse solves, layouts   */
  STOKES_KERNEL_SPMM_A3_COARSE = 8, /* A~_3 x 3 RHS on the coarser levels   */
  STOKES_KERNEL_RESIDUAL = 9,     /* A U in the FP64 full-system residual    */
  STOKES_KERNEL_COARSE_CYCLE = 10,/* every level below the finest of a V-cycle
                                     in one cooperative kernel               */
  STOKES_KERNEL_COUNT = 11
} stokes_kernel;
stokes_status stokes_kernel_stats(stokes_ctx* ctx, int kernel, int64_t* launches,
                                  double* total_ms, double* bytes);
/* The launches of a class that were bracketed by CUDA events since the last
 * reset (all of them with profile = 1, which runs without graphs; with
 * profile = 2 + k the graphs stay on and only class k's launches outside graph
 * replays are timed), their summed milliseconds and algorithmic bytes, so that
 * timed_bytes / timed_ms is the class's achieved bandwidth. */
stokes_status stokes_kernel_timing(stokes_ctx* ctx, int kernel, int64_t* timed_launches,
                                   double* timed_ms, double* timed_bytes);
stokes_status stokes_kernel_stats_reset(stokes_ctx* ctx);
/* Change the profiling mode of a context (same values as options.profile). */
stokes_status stokes_profile_mode(stokes_ctx* ctx, int mode);

/* Exercises the bounded device waits (the grid-wide barriers of the
 * cooperative coarse-level kernel, options.coarse_kernel = 1): launches a
 * barrier that nothing completes, on the context's stream. Every wait gives up
 * after a bounded number of polls (about a second), records the expiry and
 * returns, so the call returns STOKES_ERR_TIMEOUT and the context stays
 * usable (the status flag is cleared again). No counterpart in the paper. */
stokes_status stokes_check_bounded_wait(stokes_ctx* ctx);

/* Wall-clock milliseconds that stokes_setup spent per phase (host clock, the
 * stream synchronised at the end of each phase): mesh hierarchy, patterns and
 * element-coloured assembly of every level (the paper's Sec. 2.2 operators);
 * transfers and stencil / symmetric storages; dense coarsest-level inverses;
 * smoother spectra (Lanczos); FP32 copies and auxiliaries; threads-per-row
 * tuning. ms must hold STOKES_SETUP_PHASES doubles. */
enum { STOKES_SETUP_ASSEMBLY = 0, STOKES_SETUP_STORAGE = 1, STOKES_SETUP_COARSE = 2, STOKES_SETUP_SPECTRA = 3,
       STOKES_SETUP_COPIES = 4, STOKES_SETUP_TUNING = 5, STOKES_SETUP_PHASES = 6 };
stokes_status stokes_setup_phases(stokes_ctx* ctx, double ms[STOKES_SETUP_PHASES]);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_H */
