/*
 * bddc.h -- C ABI of the GB300 multilevel BDDC library (libbddc_gb300.so).
 *
 * The library implements the data-parallel hot path of multilevel BDDC as described in
 * Sistek, Mandel, Sousedik, Burda, "Parallel implementation of Multilevel BDDC":
 * the reduced interface problem S u = g solved by a Krylov method (Sec. 2), with the
 * BDDC preconditioner of two and more levels set up by Algorithm 1 and applied by
 * Algorithm 2 (Sec. 3).  All numerical work runs in CUDA kernels on one GPU; the host
 * side of the library performs the index analysis (interface classification, corner
 * selection, coarse numbering) and orchestrates the launches.
 *
 * Conventions shared by every entry point
 *   - Return value: BDDC_OK (0) or a negative BDDC_ERR_* code.  Nothing aborts and no
 *     kernel traps; bddc_last_error() returns a message for the calling thread.
 *   - "host" pointers are read during the call only and stay owned by the caller.
 *     "device" pointers are CUDA device memory owned by the caller.
 *   - A handle owns all device memory it allocates (factors, maps, work vectors) until
 *     bddc_free().  All work is enqueued on the CUDA stream given to bddc_setup(); calls
 *     returning a status synchronise that stream before returning.
 *   - Free-DOF numbering: the DOF of (node p, component c) is p*dofs_per_node + c; DOFs
 *     marked in `dirichlet` are removed and the remaining ones are numbered ascending.
 *     Vectors of several right-hand sides are stored column after column
 *     ([nrhs][n_free], column k at offset k*n_free).
 *   - A handle is not thread-safe; distinct handles may be used from distinct threads.
 */
#ifndef BDDC_GB300_H
#define BDDC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BDDC_MAX_LEVELS 6

/* status codes */
#define BDDC_OK 0
#define BDDC_ERR_INVALID (-1)       /* bad argument, mesh or partition (empty subdomain, id out of range, ...) */
#define BDDC_ERR_BREAKDOWN (-2)     /* non-positive pivot in a subdomain factorisation (stats: level, subdomain) */
#define BDDC_ERR_NOT_CONVERGED (-3) /* Krylov iteration cap reached; x holds the last iterate */
#define BDDC_ERR_NAN (-4)           /* NaN/Inf met in a reduction */
#define BDDC_ERR_CUDA (-5)          /* CUDA runtime error */
#define BDDC_ERR_OOM (-6)           /* device allocation failed */
#define BDDC_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up */

/* physics */
#define BDDC_POISSON 0      /* -div(coef grad u) = f, 1 DOF per node */
#define BDDC_ELASTICITY 1   /* isotropic linear elasticity, coef = Young's modulus, nu = Poisson ratio */
#define BDDC_STOKES 2       /* Stokes flow, Taylor-Hood Q2-Q1 hexes (27 nodes, 4 DOF slots u,v,w,p per
                               node; the pressure slot exists on the 8 vertex nodes only, the others
                               must be marked prescribed), coef = viscosity */

/* constraint classes (Sec. 2: corners, averages over edges and faces) */
#define BDDC_CORNERS 1u
#define BDDC_EDGES 2u
#define BDDC_FACES 4u

/* precision of the subdomain factorisations and the preconditioner */
#define BDDC_PREC_FP64 0    /* plain: every factor and solve in FP64 */
#define BDDC_PREC_MIXED 1   /* FP32 factors and preconditioner; FP64 Krylov, FP64 Schur operator, FP64 coarsest level */

/* interface weights D_i of E_i^T = D_i R_i (Sec. 2) */
#define BDDC_WEIGHTS_STIFFNESS 0     /* D_i(j) = K_i(jj) / sum_k K_k(jj) */
#define BDDC_WEIGHTS_MULTIPLICITY 1  /* D_i(j) = 1 / (number of subdomains sharing the node) */

typedef struct bddc_handle_s* bddc_handle;

/* Mesh of the first level (host pointers).  Element types (Sec. 4: hexahedra for the Stokes
 * cavity, linear tetrahedra for the geocomposite elasticity problem):
 * Q1: local node a at reference position xi_d = 2*((a >> d) & 1) - 1 (2**dim nodes);
 * linear simplex (triangle, tetrahedron; dim + 1 nodes, Poisson and elasticity): any vertex
 *   order, either orientation (the element uses |det J|); degenerate simplices are invalid input;
 * Q2 (Stokes): a = ix + 3 iy + 9 iz at xi = (ix-1, iy-1, iz-1). */
typedef struct {
  int dim;                  /* 2 or 3 */
  int nodes_per_elem;       /* 4 (2D Q1), 8 (3D Q1), 3 (triangle), 4 in 3D (tetrahedron) or 27 (Q2-Q1 Stokes) */
  int dofs_per_node;        /* 1 (Poisson), dim (elasticity) or 4 (Stokes) */
  int physics;              /* BDDC_POISSON | BDDC_ELASTICITY | BDDC_STOKES */
  int64_t n_nodes;
  int64_t n_elems;
  const double* coords;     /* [n_nodes * dim] */
  const int32_t* conn;      /* [n_elems * nodes_per_elem] node ids */
  const double* coef;       /* [n_elems] coefficient (Young's modulus / conductivity), > 0 */
  double nu;                /* Poisson ratio (elasticity) */
  const uint8_t* dirichlet; /* [n_nodes * dofs_per_node], 1 = prescribed */
  const double* dir_values; /* [n_nodes * dofs_per_node] prescribed values, or NULL (all zero);
                               bddc_solve then solves K_ff u = f - K_fd u_d */
} bddc_mesh;

/* Division into subdomains per level (Algorithm 1 takes it as an input: ParMETIS/METIS in
 * the paper).  part[0][e] = level-1 subdomain of element e; part[l][s] = level-(l+1)
 * subdomain of level-l subdomain s.  n_levels counts the coarsest direct solve as a level
 * (two-level BDDC: n_levels = 2, one partition array). */
typedef struct {
  int n_levels;                              /* 2 .. BDDC_MAX_LEVELS */
  const int32_t* part[BDDC_MAX_LEVELS - 1];  /* host arrays */
  int64_t n_parts[BDDC_MAX_LEVELS - 1];      /* number of subdomains of level l+1 (at most 65,535:
                                                batched launches index subdomains by gridDim.y) */
} bddc_partition;

typedef struct {
  int precision;            /* BDDC_PREC_FP64 | BDDC_PREC_MIXED */
  int weights;              /* BDDC_WEIGHTS_* */
  unsigned all_corners;     /* bit (l-1) set: every interface node of level l is a corner */
  int maxit;                /* Krylov iteration cap */
  int refine_steps;         /* mixed: FP64 refinement steps of each interior solve in S; 0 = automatic */
  int flexible;             /* 1: Polak-Ribiere beta; 0: Fletcher-Reeves; -1: automatic (mixed -> 1) */
  int use_graph;            /* 1: capture one Krylov iteration in a CUDA graph */
  int verbose;              /* >= 2: phase times of the host index analysis on stderr */
  int profile;              /* 1: time kernel classes with CUDA events (bddc_stats.prof_*) */
  int tensor_cores;         /* mixed: 1 = FP32 trailing updates and panel solves of the factorisation on
                               the tcgen05 tensor cores (two row-scaled FP16 parts, three products;
                               Stokes levels read a copy with the pivot signs on the columns as the
                               second operand): per 256-wide sub-panel the 256 x 256 diagonal block
                               is factored and inverted on CUDA cores and the rows below it are
                               solved as A(i, D) X^T S_D with X = L_D^{-1}; 2 = trailing updates only
                               (panel solves tile by tile on CUDA cores); 0 = FP32 CUDA cores */
  int inner_steps;          /* mixed PCG: FP64 outer refinement x += S~^{-1}(g - S x) (residual with the
                               FP64 operator S) around an inner PCG with a cheaper operator S~:
                               0 = S~ from the stored interface factor (L_GG S L_GG^T - C^T R C, no
                               interior solve), k >= 1 = S with k interior-solve steps,
                               -1 = no outer loop (every PCG iteration applies the FP64 operator) */
  double inner_tol;         /* first inner residual reduction of the outer refinement (later ones adapt to
                               the observed outer reduction); 0 = automatic (1e-2) */
  int krylov;               /* BDDC_KRYLOV_*; 0 = automatic: PCG for the SPD problems; for Stokes
                               BiCGstab (FP64) or flexible GMRES (mixed: FP32 factors of the
                               saddle points make the preconditioner inexact beyond what
                               BiCGstab's short recurrences tolerate) */
  int autotune;             /* 1: time the sweep launch variants (CTAs per SM, tile-ring depth, task order)
                               on every level at set-up and keep the fastest; results are cached per level
                               shape for the life of the process.  0: fixed defaults */
  int wait_probe;           /* test only, default 0.  1: every wait of the streaming sweeps for a
                               published solution block polls a device word that nothing sets, with
                               a short limit, so that each sweep runs
                               its bounded-wait error path and the call reports BDDC_ERR_TIMEOUT (the
                               results of such a call are meaningless; the CUDA context stays usable).
                               Tile-copy waits are not affected. */
  int inner_operator;       /* mixed PCG, inner operator S~ of the outer refinement: 0 = automatic
                               (the explicit form when the interior padding it needs adds at most 8 %
                               to the interior factor, else the factor products), 1 = products with
                               the stored interface factor, S~ x = L_GG S L_GG^T x - C^T R C x,
                               2 = the explicit augmented Schur complement S_i + C_i^T R C_i, copied
                               from the tiles when the interior is eliminated (the interior block
                               count is padded to a multiple of 4 tiles), one pass over its lower
                               triangle per product.  Elasticity and Poisson with tensor cores only;
                               otherwise 1 */
  int retain_host_memory;   /* 1 (default): at the first set-up of the process, ask the C library's
                               allocator (glibc) to keep freed heap memory (M_TOP_PAD 256 MB,
                               M_TRIM_THRESHOLD 1 GB), so that repeated set-ups do not page-fault
                               their host index arrays in again; 0: leave the allocator alone */
} bddc_opts;

#define BDDC_KRYLOV_AUTO 0
#define BDDC_KRYLOV_PCG 1        /* preconditioned CG (Sec. 4), SPD problems */
#define BDDC_KRYLOV_BICGSTAB 2   /* right-preconditioned BiCGstab (Sec. 4, Stokes) */
#define BDDC_KRYLOV_FGMRES 3     /* right-preconditioned flexible GMRES(50) */

/* kernel classes timed when bddc_opts.profile = 1 */
#define BDDC_PROF_TRSV 0    /* streaming triangular sweeps over interior block rows (Schur operator) */
#define BDDC_PROF_FACTOR 1  /* batched blocked Cholesky steps on CUDA cores (diagonal, panel, in-panel update) */
#define BDDC_PROF_SPMV 2    /* FP64 sparse products with K_i */
#define BDDC_PROF_TRMV 3    /* inner Schur operator: products with the stored interface factor */
#define BDDC_PROF_TRSV_IFACE 4   /* sweeps over interface block rows (subdomain corrections) */
#define BDDC_PROF_COARSE 5  /* sweeps of the coarsest level's FP64 factor */
#define BDDC_PROF_TC_UPDATE 6   /* tensor-core trailing updates of the factorisation (FP32-equivalent flops) */
#define BDDC_PROF_TC_PANEL 7    /* tensor-core panel solves below the diagonal blocks (flops of the
                                   triangular solves they replace) */
#define BDDC_PROF_CLASSES 8

typedef struct {
  int iterations;           /* Krylov iterations of the last solve (max over right-hand sides) */
  int converged;            /* 1 when every right-hand side met the tolerance */
  double rel_residual;      /* max over right-hand sides of ||g - S u|| / ||g|| at exit */
  double rhs_norm;          /* ||g|| (condensed right-hand side) of the first right-hand side */
  double lambda_min, lambda_max;  /* Lanczos estimate from PCG (first right-hand side) */
  int n_levels;
  int64_t n_sub[BDDC_MAX_LEVELS];     /* subdomains of BDDC level l (index l-1) */
  int64_t n_dof[BDDC_MAX_LEVELS];     /* free DOFs of the level's problem */
  int64_t n_iface[BDDC_MAX_LEVELS];   /* interface DOFs of the level */
  int64_t n_coarse[BDDC_MAX_LEVELS];  /* coarse DOFs of the level */
  int64_t n_promoted[BDDC_MAX_LEVELS];/* corners added by the rigid-body test */
  int breakdown_level, breakdown_sub; /* set with BDDC_ERR_BREAKDOWN */
  int refine_steps;                   /* refinement steps in use (mixed) */
  int inner_steps;                    /* inner operator in use: -1 none, 0 factor products, k steps */
  int outer_iterations;               /* FP64 outer refinement steps of the last solve (max over rhs) */
  double analysis_ms, factor_ms, solve_ms;
  int64_t factor_bytes;               /* device bytes held by factors */
  double prof_ms[BDDC_PROF_CLASSES];          /* summed CUDA-event durations per class */
  int64_t prof_launches[BDDC_PROF_CLASSES];   /* launches per class */
  double prof_bytes[BDDC_PROF_CLASSES];       /* algorithmic bytes moved (TRSV, SPMV) */
  double prof_flops[BDDC_PROF_CLASSES];       /* algorithmic flops (FACTOR) */
  /* sweep launch configuration per level l (index 2 (l-1) + part; part 0 interior, 1 interface) */
  int sweep_ctas[2 * BDDC_MAX_LEVELS];        /* CTAs per SM of the persistent grid (1 or 2) */
  int sweep_deep[2 * BDDC_MAX_LEVELS];        /* 1: deep tile ring (FP32 6 / FP64 3 stages), 0: shallow (4 / 2) */
  int sweep_order[2 * BDDC_MAX_LEVELS];       /* 0: subdomain order, 1: longest chains first within each depth */
  double tune_ms;                              /* time spent autotuning in the last set-up (0 when cached) */
  double prepare_ms;                           /* device set-up of the last bddc_setup: level layouts, maps,
                                                  allocations and uploads (between analysis and factor) */
  int inner_operator;                          /* inner operator of the mixed PCG: 0 none, 1 factor
                                                  products, 2 explicit augmented Schur complement */
} bddc_stats;

/* Index maps of one level, library-owned, valid until bddc_free (for bit-exact checks).
 * Subdomain-local DOF order: interior DOFs ascending by level DOF id, then interface DOFs
 * ascending.  C_i is stored row by row: the rows of subdomain s are
 * sub_coarse_ptr[s] .. sub_coarse_ptr[s+1]-1, row r has entries c_ptr[r] .. c_ptr[r+1]-1
 * with local column c_col[] (position in the local order) and value c_val[]. */
typedef struct {
  int64_t n_dof, n_sub, n_iface, n_coarse, n_globs, n_promoted;
  const int64_t* iface_dofs;       /* [n_iface] level DOF ids, ascending */
  const int64_t* sub_dof_ptr;      /* [n_sub+1] */
  const int64_t* sub_dofs;         /* [sub_dof_ptr[n_sub]] level DOF ids in local order */
  const int64_t* sub_nI;           /* [n_sub] interior count */
  const int64_t* sub_iface;        /* [sub_dof_ptr[n_sub]] position in iface_dofs of each local DOF, -1 interior */
  const double* sub_wmult;         /* [sub_dof_ptr[n_sub]] multiplicity weight, 0 interior */
  const int64_t* sub_coarse_ptr;   /* [n_sub+1] */
  const int64_t* sub_coarse;       /* R_Ci: global coarse ids, ascending */
  const int64_t* c_ptr;            /* [sub_coarse_ptr[n_sub]+1] */
  const int64_t* c_col;
  const double* c_val;
  const int64_t* glob_ptr;         /* [n_globs+1] */
  const int64_t* glob_nodes;       /* nodes of every glob, ascending */
  const int32_t* glob_kind;        /* 0 vertex, 1 edge, 2 face */
  const int32_t* glob_promoted;    /* 1 = corner added by the rigid-body test */
  const int64_t* coarse_glob;      /* [n_coarse] */
  const int32_t* coarse_comp;      /* [n_coarse] */
} bddc_level_maps;

/* Fill *opts with the defaults (mixed precision, stiffness weights, maxit 500, automatic
 * refinement, automatic beta, graph on). */
void bddc_default_opts(bddc_opts* opts);

/* Index analysis only (Algorithm 1 without the numerical steps): interface classification
 * into faces/edges/vertices, corner selection, constraint rows and coarse numbering on every
 * level, pseudo-meshes of the levels above the first.  Makes no CUDA call, so it runs on a
 * machine without a GPU; the handle then serves bddc_get_maps and bddc_free only.
 * mesh, part: host.  constraints: BDDC_CORNERS|BDDC_EDGES|BDDC_FACES.  opts may be NULL.
 * Errors: BDDC_ERR_INVALID for an inconsistent mesh/partition. */
int bddc_analyze(const bddc_mesh* mesh, const bddc_partition* part, unsigned constraints,
                 const bddc_opts* opts, bddc_handle* out);

/* Full set-up, Algorithm 1: index analysis, then on the GPU per level: element matrices,
 * sub-assembly of K_i (Sec. 2), factorisation of the augmented constrained Neumann matrix
 * K_i + rho C_i^T C_i with the constraint rows (yields the interior factor, Eq. psi_def's
 * coarse basis Psi_i and K_Ci = -Lambda_i), assembly of the next level, and the FP64
 * factorisation of the coarsest matrix K_C.  stream: a cudaStream_t (NULL = default).
 * Errors: INVALID, BREAKDOWN (stats via bddc_get_stats), CUDA, OOM. */
int bddc_setup(const bddc_mesh* mesh, const bddc_partition* part, unsigned constraints,
               const bddc_opts* opts, void* stream, bddc_handle* out);

/* Replace the element coefficients (host [n_elems]) and redo the numerical set-up, keeping
 * the index analysis.  Errors as bddc_setup. */
int bddc_update_coef(bddc_handle h, const double* coef);

/* Solve K u = f for nrhs right-hand sides (Sec. 2): condensed right-hand side
 * g = f_G - sum R_i^T K_GI K_II^{-1} f_I,i (minus K_fd u_d when prescribed values are non-zero),
 * a Krylov method on S u_G = g preconditioned by Algorithm 2 (opts.krylov: PCG, BiCGstab for
 * Stokes as in Sec. 4, flexible GMRES; in the mixed form PCG runs inside the FP64 outer
 * refinement of opts.inner_steps), stop when ||g - S u_G|| / ||g|| <= tol on the true residual
 * with the FP64 operator, then interior recovery u_I = K_II^{-1} (f_I - K_IG u_G).  rhs: device [nrhs][n_free] FP64.  x: device
 * [nrhs][n_free] FP64, output (the initial guess is zero).  stats: host, may be NULL.
 * Errors: NOT_CONVERGED (x holds the last iterate), NAN, CUDA, TIMEOUT. */
int bddc_solve(bddc_handle h, const double* rhs, double* x, int nrhs, double tol, bddc_stats* stats);

/* Same as bddc_solve with host buffers: copies rhs to the device and x back (end to end). */
int bddc_solve_host(bddc_handle h, const double* rhs_host, double* x_host, int nrhs, double tol,
                    bddc_stats* stats);

/* One application of the multilevel BDDC preconditioner, Algorithm 2, to interface
 * residuals.  r, z: device [nrhs][n_iface] FP64 in the order of bddc_level_maps.iface_dofs
 * of level 1.  Errors: INVALID, CUDA. */
int bddc_apply_precond(bddc_handle h, const double* r, double* z, int nrhs);

/* The reduced interface operator of Sec. 2, y = S x = sum_i R_i^T (K_GG - K_GI K_II^{-1} K_IG) R_i x,
 * computed with discrete Dirichlet problems.  x, y: device [nrhs][n_iface] FP64. */
int bddc_apply_schur(bddc_handle h, const double* x, double* y, int nrhs);

/* The inner operator of the mixed form's outer refinement (mixed-precision PCG handles only):
 * y = sum_i R_i^T S~_i R_i x with S~_i = S_i + C_i^T R C_i - C_i^T R C_i evaluated from FP32 data
 * (the factor products or the explicit augmented Schur complement, see bddc_opts.inner_operator),
 * FP32 products, FP64 in and out; it equals the FP64 operator of bddc_apply_schur up to the FP32
 * factorisation's error.  Same layout and streams as bddc_apply_schur.  Errors: INVALID (no
 * set-up, not a mixed-precision PCG handle), CUDA. */
int bddc_apply_inner_schur(bddc_handle h, const double* x, double* y, int nrhs);

/* Adjoint gradient of a scalar J(u) with u = K(coef)^{-1} f: solves K lambda_k = dJdu_k with
 * the same factors (K is symmetric), then grad_rhs = lambda and
 * grad_coef[e] = - sum_k lambda_k,e^T (dK_e/dcoef_e) u_k,e with dK_e/dcoef_e = K_e / coef_e
 * (Poisson and elasticity, whose element matrices are linear in the coefficient; for Stokes the
 * viscosity scales only the viscous block, so grad_coef must be NULL there).
 * dJdu, u: device [nrhs][n_free].  grad_coef: device [n_elems] or NULL.  grad_rhs: device
 * [nrhs][n_free] or NULL.  tol: Krylov tolerance of the adjoint solve.
 * Errors as bddc_solve; INVALID for grad_coef on a Stokes handle. */
int bddc_grad(bddc_handle h, const double* dJdu, const double* u, int nrhs, double tol,
              double* grad_coef, double* grad_rhs);

/* bddc_grad without device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot let a library allocate device memory -- applications that hand
 * (almost) all of it to their own pool, where a cudaMalloc from the library would fail or
 * fragment that pool, and latency-critical loops, where cudaMalloc/cudaFree would stall the
 * device.  Same results as bddc_grad (the element contraction sums right-hand sides in another
 * order).  grad_rhs is required (it receives lambda); grad_coef may be NULL.  The full-DOF
 * scratch of the contraction lives in one fixed 16 MiB device array inside the library, held
 * by every GPU that loads the library until the process exits: meshes with
 * n_nodes * dofs_per_node > 1,048,576 are rejected with BDDC_ERR_INVALID.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress).  The adjoint solve is the
 * handle's own: the first solve on a handle, and the first after the Krylov method changes,
 * builds the handle's cached CUDA graph of one iteration with its capture stream and events, so
 * warm a handle with one bddc_solve (or one call of this entry point) before relying on
 * allocation-free calls in a loop.  The call synchronises the handle's stream (it reads the
 * Krylov scalars back every iteration), so it must not be made while that stream or the calling
 * thread is capturing a CUDA graph.  Every call on a device shares the array and overwrites the
 * part it reads, so calls whose work overlaps on the GPU (several streams, several host threads)
 * race and must be serialised by the caller.  Errors as bddc_grad. */
int bddc_grad_noalloc(bddc_handle h, const double* dJdu, const double* u, int nrhs, double tol,
                      double* grad_coef, double* grad_rhs);

/* Index maps of BDDC level `level` (1-based).  Errors: INVALID. */
int bddc_get_maps(bddc_handle h, int level, bddc_level_maps* out);

/* Local coarse matrices K_Ci = Psi_i^T K_i Psi_i = -Lambda_i of BDDC level `level` (1-based) after
 * set-up (Sec. 2, Eq. psi_def; on levels below the coarsest they are the element matrices of the
 * next level).  kc: host FP64 buffer of n entries; receives, subdomain after subdomain, the
 * nc_i x nc_i matrix of subdomain i row-major, rows and columns in the order of
 * bddc_level_maps.sub_coarse (R_Ci), where nc_i = sub_coarse_ptr[i+1] - sub_coarse_ptr[i].  The
 * entries needed are sum_i nc_i^2; a smaller n is rejected.  In both precisions the matrices are
 * FP64, formed as G_i^{-1} - R with G_i = C_i A_i^{-1} C_i^T from the factor of A_i (FP32 factor in
 * the mixed form).  Errors: INVALID (no numeric set-up, bad level, buffer too small), CUDA. */
int bddc_get_coarse(bddc_handle h, int level, double* kc, int64_t n);

/* Copy the statistics of the last set-up / solve into *out. */
int bddc_get_stats(bddc_handle h, bddc_stats* out);

/* Sizes of the problem: number of free DOFs of level 1 and of its interface. */
int bddc_sizes(bddc_handle h, int64_t* n_free, int64_t* n_iface);

/* Release every resource of the handle (safe on NULL). */
void bddc_free(bddc_handle h);

/* Number of kernels the library has launched in this process (all handles). */
int64_t bddc_kernel_launches(void);

/* Reset the per-class timers of bddc_stats.prof_* on a handle. */
int bddc_reset_profile(bddc_handle h);

/* Batching ablation (measurement only; no counterpart in the paper): on level 1 of a set-up
 * handle, times with CUDA events on the handle's stream
 *   ms[0]  one forward + backward interior sweep pair, all subdomains in one launch each,
 *   ms[1]  the same sweeps launched once per subdomain,
 *   ms[2]  the CUDA-core tiled factorisation (no tensor cores) batched over all subdomains,
 *   ms[3]  the same factorisation launched once per subdomain per step.
 * The factorisation runs are repeated work: afterwards the handle's level-1 factors are
 * recomputed by the normal path, so the handle stays valid and bit-identical.  Mixed-precision
 * SPD handles only.  Errors: INVALID, CUDA. */
int bddc_batching_ablation(bddc_handle h, double* ms);

/* Test and measurement entry point for the tensor-core trailing update of the mixed factorisation
 * (Algorithm 1, "factorize the matrices of local saddle point problems"; the FP32 block Cholesky's
 * rank-256 or rank-512 update on tcgen05 from two row-scaled FP16 parts, three products).
 * rank: 256 or 512.  a: host FP32 n x n row-major, n = 64 nb with n >= rank + 64.  The first rank
 * columns play the factored panel P and the rest the trailing matrix: on return
 * a(i, j) -= sum_{q < rank} a(i, q) a(j, q) for every i, j >= rank whose 64 x 64 tiles satisfy
 * tile(j) <= tile(i) (diagonal tiles are updated in full); the other entries are returned
 * unchanged.  The data pass through the factor's tile layout and the same two
 * kernels (panel split, persistent tcgen05 update) that bddc_setup launches.  ms: host, receives
 * the update kernel's duration from CUDA events, or NULL.  Device buffers are allocated and freed
 * by the call, on the default stream.  Errors: INVALID (n, rank), CUDA, OOM, TIMEOUT (a bounded
 * wait of the update kernel gave up). */
int bddc_tc_update_check(int64_t n, int rank, float* a, double* ms);

/* Message of the last failure on the calling thread ("" if none). */
const char* bddc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_GB300_H */
