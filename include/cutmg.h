/*
 * cutmg: GB300 (sm_103a) CutFEM multigrid — C ABI.
 *
 * Solves the Nitsche-Dirichlet Poisson problem on a level-set domain cut out
 * of a Cartesian background mesh, with face-based ghost penalties, by CG
 * preconditioned with a V-cycle whose smoother is the multiplicative
 * vertex-patch smoother (Cui & Kanschat, arXiv 2508.11608):
 *   operator       eqs. "cutfem_nitsche" and "cutfem-ghost" (Sec. 2.1)
 *   transfer       embedding prolongation, restriction = transpose (Sec. 2.2)
 *   smoother       eqs. "local-solver", "smoother", "smoother-split" (Sec. 2.3, Sec. 3)
 *
 * Conventions shared by every call:
 *  - Vectors are caller-owned DEVICE arrays of doubles of length
 *    cf_level_n_dofs(problem, level) (cf_n_dofs for the finest level).  DoFs
 *    are the lattice nodes of active cells, numbered by increasing lattice
 *    flat index i_0 + n i_1 + n^2 i_2 (n = p N + 1 nodes per direction), i.e.
 *    first coordinate fastest; cf_dof_lattice returns that index per DoF.
 *  - Every call that takes a stream is stream-ordered and does not
 *    synchronise unless stated.  `stream` is a cudaStream_t (0 = legacy
 *    default stream).
 *  - Every call returns a cf_status; on failure cf_last_error() holds a
 *    message (thread-local).  A problem handle stays valid after CF_ENOCONV.
 *  - The problem handle owns every hierarchy buffer on the device it was
 *    created on (the current device at cf_setup).
 *  - Supported: dim 2 with degree 1..4 (degree 4 goes beyond the paper,
 *    whose experiments stop at Q3), dim 3 with degree 1..2.
 */
#ifndef CUTMG_H
#define CUTMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CF_OK = 0,
  CF_EINVAL = 1,
  CF_ENOMEM = 2,
  CF_ECUDA = 3,
  CF_ENOCONV = 4,
  CF_ETIMEOUT = 5,
  CF_EUNSUPPORTED = 6
} cf_status;

/* Level-set kinds (Omega = {phi < 0}; Sec. 4 uses an analytic level set).
 * y = rot (x - center) are body coordinates (rot row-major, rows = axes). */
typedef enum {
  CF_LS_SPHERE = 0,    /* phi = |x - center| - radius (disk in 2D)                        */
  CF_LS_PLANE = 1,     /* phi = normal . x - offset (half space; used in tests)            */
  CF_LS_ELLIPSOID = 2, /* phi = sqrt(sum (y_i / axes_i)^2) - 1 (3D)                         */
  CF_LS_TORUS = 3,     /* phi = sqrt((sqrt(y_0^2 + y_1^2) - major)^2 + y_2^2) - radius (3D) */
  CF_LS_FLOWER = 4,    /* phi = |x - c| - (radius + amplitude cos(lobes (theta - phase))) (2D) */
  CF_LS_CALLBACK = 5   /* phi and its gradient from the user's callbacks (see cf_levelset)  */
} cf_levelset_kind;

typedef enum { CF_FP64 = 0, CF_MIXED = 1 } cf_precision;

/* Background mesh [lo, hi]^dim with n_cells cells per direction on the finest
 * level and n_levels levels; level l has n_cells / 2^(n_levels-1-l) cells per
 * direction (Sec. 2.1 nested hierarchy).  n_cells must be divisible by
 * 2^(n_levels-1). */
typedef struct {
  int dim;
  int n_cells;
  double lo, hi;
  int n_levels;
} cf_mesh;

typedef struct {
  int kind;          /* cf_levelset_kind */
  double center[3];  /* centre (sphere, ellipsoid, torus, flower) */
  double radius;     /* sphere radius; torus minor radius; flower base radius */
  double normal[3];  /* plane normal */
  double offset;     /* plane offset */
  double axes[3];    /* ellipsoid semi-axes */
  double rot[9];     /* ellipsoid / torus rotation, row-major, rows = body axes */
  double major;      /* torus major radius */
  int lobes;         /* flower: number of lobes */
  double amplitude;  /* flower: radius amplitude */
  double phase;      /* flower: rotation angle theta_0 */
  /* CF_LS_CALLBACK: phi(x, user) and grad(x, g, user) = d phi / dx; x and g
   * have 3 components (unused ones 0).  Known only at points, the level set
   * is bounded on a cell or face from a 5-point-per-direction lattice of
   * samples widened by the largest sampled |grad phi| times the distance to
   * the nearest sample (an exact enclosure when that bounds |grad phi|, e.g.
   * for signed distances); the quadrature's monotonicity test samples the
   * gradient the same way.  Both must be pure functions of x, callable
   * concurrently from several host threads (see cf_params.setup_threads).
   * They are called during cf_setup / cf_setup_host, during cf_rhs_user /
   * cf_host_rhs_user (which integrate the cut cells again), and during
   * cf_server_run for a served request; they and `user` must stay valid
   * until the handle is destroyed (the server: until cf_server_run returns).
   * Ignored for the other kinds. */
  double (*phi)(const double* x, void* user);
  void (*grad)(const double* x, double* g, void* user);
  void* user;
} cf_levelset;

/* Method parameters.  Zero / negative entries select the defaults given. */
typedef struct {
  double gamma_D;        /* Nitsche penalty, used as gamma_D / h (eq. "cutfem_nitsche"); default 20 p^2 */
  double gamma_ghost[4]; /* ghost penalty gamma_k, k = 1..p (eq. "cutfem-ghost"); default 0.1 each */
  int n_c;               /* repetitions of the cut-patch sweep (eq. "smoother-split"); default 2 */
  int quad_q;            /* Gauss points per sub-interval of the cut-cell rules; default p + 2 */
  int precision;         /* cf_precision of cf_vcycle / cf_solve; default CF_FP64 */
  int smoother;          /* cf_smoother: CF_SMOOTHER_MVS (default) or CF_SMOOTHER_CHEBYSHEV */
  int smoother_degree;   /* degree of the Chebyshev smoother (Sec. 4 compares degree 5); default 5 */
  int setup_threads;     /* host threads of the setup (OpenMP); default: the OpenMP default.  One
                            suits level-set callbacks that serialise (an interpreter's lock) */
} cf_params;

/* Smoother of the V-cycle.  MVS: the multiplicative vertex-patch smoother
 * (Sec. 2.3, the method).  CHEBYSHEV: the baseline the paper compares it with
 * (Sec. 4): point-Jacobi-scaled Chebyshev smoothing of the given degree on
 * [lambda / 20, lambda], lambda = 1.2 x lambda_max(D^{-1} A_l) estimated by 30
 * power iterations from the all-ones vector; the same polynomial pre and post
 * (a symmetric V-cycle).  The batched form supports MVS only. */
typedef enum { CF_SMOOTHER_MVS = 0, CF_SMOOTHER_CHEBYSHEV = 1 } cf_smoother;

typedef struct {
  int iterations;          /* CG iterations taken */
  double rel_residual;     /* final recursive ||r|| / ||b|| */
  double true_rel_residual;/* ||b - A x|| / ||b|| recomputed at exit */
  double solve_ms;         /* wall time of the solve on the stream (device events) */
} cf_info;

typedef struct cf_problem cf_problem;

/* Build the hierarchy (Sec. 2.1 operators on every level, Sec. 2.2 transfer,
 * Sec. 2.3 / Sec. 3 patches): classification, cut-cell quadrature, cell and
 * patch matrices (host, FP64), then the upload to the current device, ordered
 * on `stream` (a cudaStream_t, 0 = legacy default stream).  Blocking: the
 * call synchronises `stream` before it returns, so the handle is ready for
 * any stream.  *out receives the handle (NULL on failure); the caller owns
 * it and releases it with cf_destroy.
 * Errors: CF_EINVAL (null argument, bad sizes, degree, kind; a domain that
 * misses the mesh or whose boundary crosses no cell, which leaves no
 * Dirichlet condition; a coarsest level above 12,000 DoFs), CF_EUNSUPPORTED
 * (dim 3 with degree 3 or 4), CF_ENOMEM, CF_ECUDA. */
cf_status cf_setup(const cf_mesh* mesh, const cf_levelset* ls, int degree,
                   const cf_params* params, void* stream, cf_problem** out);
void cf_destroy(cf_problem* pb);
const char* cf_last_error(void);

int cf_n_levels(const cf_problem* pb);
int64_t cf_n_dofs(const cf_problem* pb);
int64_t cf_level_n_dofs(const cf_problem* pb, int level);
/* Host array of cf_level_n_dofs int64 lattice flat indices. */
cf_status cf_dof_lattice(const cf_problem* pb, int level, int64_t* h_idx);
/* Host array of dim * n doubles, node coordinates (x_0, x_1, ..) per DoF. */
cf_status cf_dof_coords(const cf_problem* pb, int level, double* h_xyz);
/* Host counters of the finest level: [active cells, cut cells, ghost faces,
 * patches, cut patches, cut-patch matrix entries]. */
cf_status cf_stats(const cf_problem* pb, int level, int64_t* h_out6);
/* Algorithmic work of one colour step on a level, from the host setup
 * (Sec. 3's two patch kinds): kind 0 = interior patches (fast
 * diagonalisation, Sec. 2.3), 1 = cut patches (residual rows, the ghost-face
 * moments of the patch rows where the cut kernel forms them itself (3D
 * degree 2), and the dense local inverse), 2 = the ghost-face moments a
 * separate launch computes for the cut-patch rows of the colour (face
 * penalty of Sec. 2.1; zero where the cut kernel forms them).  h_out3 = [flops, scalars moved, index
 * bytes moved]; bytes = scalars x sizeof(precision) + index bytes.
 * CF_EINVAL for a bad level, kind or colour (0 <= colour < 2^dim); level 0
 * (the coarsest, solved exactly) has no colour steps and reports zeros. */
cf_status cf_work_model(const cf_problem* pb, int level, int kind, int colour, double* h_out3);

/* Finest-level right-hand side for user data (Sec. 2.1 with Nitsche data,
 * reading 7): b_i = (f, phi_i)_Omega + (g, gamma_D/h phi_i - d_n phi_i)_Gamma,
 * integrated with the same cut-cell rules as the operator.  f(x, user) is the
 * source, g(x, user) the Dirichlet data on Gamma; x has 3 components (unused
 * ones 0); a NULL function counts as zero.  The callbacks run sequentially on
 * the calling thread during the call (host assembly), then b is copied to d_b
 * (cf_n_dofs doubles, DoF order) on `stream` and the call waits for it.
 * CF_EINVAL on null problem or output. */
cf_status cf_rhs_user(cf_problem* pb, double (*f)(const double* x, void* user),
                      double (*g)(const double* x, void* user), void* user, double* d_b, void* stream);

/* Select the precision of cf_vcycle and cf_solve (CF_FP64 or CF_MIXED). */
cf_status cf_set_precision(cf_problem* pb, int precision);

/* Launch variant of a kernel family, for tests and tuning; every variant
 * computes the same colour step (Sec. 2.3), and the variants that share an
 * arithmetic give the same bits.  family CF_VAR_INTERIOR (interior-patch
 * step): FP32 (mixed form) 1 = dense map, one patch per thread; 2 = dense
 * map, two patches per thread; 3 = dense map, several threads per patch;
 * 4 = dense map on the tensor cores (TF32 products, FP32 accumulation; the
 * automatic choice where it exists, else the same as 0); FP64 1 = two
 * patches per warp (one per half-warp), 2 = one block per patch.  family CF_VAR_CUT (cut-patch step,
 * 3D degree 2; one warp per patch, records read from global memory):
 * 1 = each patch's record (inverse and cut-cell rows) prefetched into L2 by
 * a bulk prefetch when its loads are issued, 2 = no prefetch, 3 = the next
 * patch's record prefetched while the current patch is worked on, 4 = eight
 * warps per block, one patch each, at every colour size, 5 = one warp per
 * block for colours of fewer than 8 patches per SM (the automatic choice
 * runs such colours one patch per block with four warps working on it),
 * 6 = one patch per block with four warps at every colour size.
 * family
 * CF_VAR_OPERATOR (operator
 * rows of nodes whose cells are all uncut): 1 = element-matrix form, 2 =
 * sum factorisation (the automatic choice in FP64).  variant 0 restores the
 * automatic choice.  The next
 * launches use it; captured CUDA graphs of the handle are dropped.
 * CF_EINVAL for an unknown family or variant, or a host-only handle. */
typedef enum { CF_VAR_INTERIOR = 1, CF_VAR_CUT = 2, CF_VAR_OPERATOR = 3 } cf_variant_family;
cf_status cf_set_kernel_variant(cf_problem* pb, int family, int variant);

/* Polls the tensor-core interior-patch kernel (mixed form, 2D and 3D) makes on the
 * mbarrier of its tensor-core product before it gives up (default 2^22).  A
 * block that gives up records the failure and waits (bounded, 2^22 polls)
 * for its own product to complete before it reads it; the next cf_solve /
 * cf_solve_vcycle / cf_solve_gmres then returns CF_ETIMEOUT and the handle
 * stays usable.  A limit of 0 makes every wait give up at once (a test of
 * that path).  CF_EINVAL outside [0, 2^30] or on a host-only handle. */
cf_status cf_set_wait_limit(cf_problem* pb, int64_t polls);

/* b = right-hand side of the manufactured solution u = prod_k sin(pi x_k),
 * f = d pi^2 u, Dirichlet data g = u (Nitsche data terms), finest level. */
cf_status cf_rhs(cf_problem* pb, double* d_b, void* stream);

/* y = A_L x on the finest level, FP64 (matrix-free). */
cf_status cf_apply(cf_problem* pb, const double* d_x, double* d_y, void* stream);

/* z = B r: one V-cycle with zero initial guess (precision as selected). */
cf_status cf_vcycle(cf_problem* pb, const double* d_r, double* d_z, void* stream);

/* CG preconditioned by one V-cycle per iteration, x_0 = 0, until
 * ||r||_2 <= rtol ||b||_2 (recursive residual) or maxit.  Synchronises the
 * stream once per iteration to read ||r||.  Returns CF_ENOCONV if maxit was
 * reached (x holds the last iterate). */
cf_status cf_solve(cf_problem* pb, const double* d_b, double* d_x, double rtol,
                   int maxit, cf_info* info, void* stream);
/* The V-cycle as the solver (Sec. 2.2, the direct V-cycle iteration):
 * x_{k+1} = x_k + B (b - A x_k) from x_0 = 0, B one V-cycle in the precision
 * set by cf_set_precision, until ||b - A x_k||_2 <= rtol ||b||_2 (the residual
 * in FP64).  Vectors and info as for cf_solve; CF_ENOCONV when maxit is
 * reached first (x then holds the last iterate). */
cf_status cf_solve_vcycle(cf_problem* pb, const double* d_b, double* d_x, double rtol, int maxit,
                          cf_info* info, void* stream);
/* GMRES(restart) with one V-cycle as right preconditioner (Sec. 2.2; the
 * paper's outer solver): minimises ||b - A x||_2 over x_0 + B K_k(A B, r_0),
 * x_0 = 0, modified Gram-Schmidt Arnoldi in FP64, restarted from the true
 * residual after `restart` steps; stops when the residual estimate falls to
 * rtol ||b||_2.  info->iterations counts Arnoldi steps over all cycles.  The
 * first call with a given restart allocates (2 restart + 2) finest-level
 * vectors on the device.  CF_EINVAL for restart < 1; CF_ENOCONV when maxit
 * is reached first (x holds the iterate after the last step). */
cf_status cf_solve_gmres(cf_problem* pb, const double* d_b, double* d_x, double rtol, int restart, int maxit,
                         cf_info* info, void* stream);

/* ---- single steps of the hot path on one level (parity testing) ---------
 * All vectors are FP64 device arrays in the level's DoF order; `precision`
 * selects the FP64 kernels or the FP32 kernels of the mixed form (inputs are
 * rounded to FP32, outputs widened back). */

/* y = A_l x (Sec. 2.1 operator, matrix-free). */
cf_status cf_level_apply(cf_problem* pb, int level, int precision,
                         const double* d_x, double* d_y, void* stream);
/* One colour step of the smoother: for every patch of the given colour and
 * kind (cut != 0: cut patches, else interior patches) x[I_j] += A_j^{-1}
 * (b - A x)[I_j], all from one residual (Sec. 2.3 inconsistent treatment). */
cf_status cf_level_colour_step(cf_problem* pb, int level, int precision, int cut,
                               int colour, double* d_x, const double* d_b, void* stream);
/* One full smoothing step (eq. "smoother-split"), post != 0: reversed order. */
cf_status cf_level_smooth(cf_problem* pb, int level, int precision, int post,
                          double* d_x, const double* d_b, void* stream);
/* b_{l-1} = P_l^T r_l (level >= 1). */
cf_status cf_level_restrict(cf_problem* pb, int level, int precision,
                            const double* d_r_fine, double* d_b_coarse, void* stream);
/* x_l += P_l x_{l-1} (level >= 1). */
cf_status cf_level_prolongate(cf_problem* pb, int level, int precision,
                              const double* d_x_coarse, double* d_x_fine, void* stream);
/* x_0 = A_0^{-1} b_0 (exact coarsest solve). */
cf_status cf_coarse_solve(cf_problem* pb, int precision, const double* d_b0,
                          double* d_x0, void* stream);

/* Same result as cf_coarse_solve(pb, CF_FP64, ...), for callers that cannot
 * have the call allocate device memory (work captured into a CUDA graph,
 * services that own all device memory in their own arena, loops that forbid
 * allocation on the hot path).  The paper has no counterpart.  The two
 * coarsest-level staging vectors live in one fixed file-scope device array
 * of 2 x 32768 doubles (512 KiB, held by every GPU that loads the library
 * until the process exits); the call allocates nothing.
 *  - Rejects (CF_EINVAL) a problem whose coarsest level has more than 32768
 *    lattice nodes ((p N_0 + 1)^d), and a current device other than the
 *    problem's.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is kept for the life of the process: do not call this entry
 *    point after a cudaDeviceReset of that device (the kept address would no
 *    longer name the array).
 *  - Every call on a device shares the array: calls that overlap on the GPU
 *    (different streams or threads without ordering) race and give wrong
 *    results.  Calls ordered on one stream are safe.
 *  - d_b0 / d_x0: FP64 device arrays of cf_level_n_dofs(pb, 0) entries. */
cf_status cf_coarse_solve_noalloc(cf_problem* pb, const double* d_b0, double* d_x0, void* stream);

/* ---- batched form -----------------------------------------------------------
 * Many independent problems (any geometries, mesh sizes and degrees) solved
 * together: problems with the same (dim, degree) share every launch of the
 * hot path, one persistent grid-stride launch per (V-cycle depth, colour,
 * step) over a work list of (problem, patch) pairs, with tile shapes chosen
 * by a timing autotuner at cf_batch_create.  Each problem runs its own CG
 * (own scalars, own convergence; converged problems drop out of the work
 * lists) and performs the same floating-point operations as cf_solve on it
 * alone.  The batch references the problems; they must outlive it and must
 * not be used on other streams while a batched solve runs. */
typedef struct cf_batch cf_batch;
/* Errors: CF_EINVAL (empty list, problems on different devices or host-only,
 * different n_c within one (dim, degree) group). */
cf_status cf_batch_create(cf_problem* const* problems, int count, cf_batch** out);
/* d_b[i], d_x[i]: FP64 device vectors of problem i (host arrays of count
 * pointers); infos: host array of count entries (solve_ms = the batch's time).
 * Returns CF_ENOCONV if any problem reached maxit. */
cf_status cf_batch_solve(cf_batch* bt, int precision, const double* const* d_b, double* const* d_x,
                         double rtol, int maxit, cf_info* infos, void* stream);
int64_t cf_batch_launch_count(const cf_batch* bt);
void cf_batch_destroy(cf_batch* bt);

/* ---- served form -------------------------------------------------------------
 * A stream of solve requests with arrival times, solved with continuous
 * batching: a host thread builds each hierarchy after its arrival (up to four
 * at once; a request whose params leave setup_threads at 0 is built on the
 * host cores no other running setup holds, at least a quarter of them, so a
 * request that arrives alone uses them all; the result does not depend on
 * the thread count); a prepared
 * request is admitted (FIFO) when its estimated device footprint fits the HBM
 * budget next to the resident problems and an active slot is free; every tick
 * runs one CG iteration of all active problems with the batched kernels;
 * finished problems retire at once and free their memory.  Each request
 * performs the same floating-point operations as cf_solve on it alone.
 * Precision applies to every request (CF_FP64 or CF_MIXED). */
typedef struct cf_server cf_server;
cf_status cf_server_create(size_t hbm_budget_bytes, int max_active, int precision, int keep_solutions,
                           cf_server** out);
/* Queue a request (arrival_s: seconds after cf_server_run starts; requests in
 * non-decreasing arrival order).  id receives its index. */
cf_status cf_server_submit(cf_server* s, const cf_mesh* mesh, const cf_levelset* ls, int degree,
                           const cf_params* params, double rtol, int maxit, double arrival_s, int64_t* id);
/* Serve every queued request (blocking, on `stream`, on the current device). */
cf_status cf_server_run(cf_server* s, void* stream);
/* Result of request id: info (solve_ms = admission to completion), times3 =
 * {arrival, admission, completion} in seconds, ndof, and the solution (host
 * array of ndof doubles, only with keep_solutions).  CF_EINVAL if the request
 * failed (message in cf_last_error) or has not finished. */
cf_status cf_server_result(const cf_server* s, int64_t id, cf_info* info, double* times3, int64_t* ndof,
                           double* h_x);
/* {peak device bytes of resident problems, peak active problems, ticks, run seconds} */
cf_status cf_server_stats(const cf_server* s, double* out4);
void cf_server_destroy(cf_server* s);

/* ---- instrumentation ----------------------------------------------------- */
/* Number of kernel launches this handle has issued (all calls). */
int64_t cf_launch_count(const cf_problem* pb);
/* Kernel families for cf_profile_start. */
typedef enum {
  CF_K_CUT_SOLVE = 1, /* cut-patch residual + dense local solve */
  CF_K_INTERIOR = 2,  /* interior-patch residual + fast diagonalisation */
  CF_K_APPLY_BULK = 3,/* operator, interior positions */
  CF_K_APPLY_BND = 4, /* operator, positions near the boundary */
  CF_K_FACE_MOMENTS = 5 /* ghost-face moments G_m of the current iterate */
} cf_kernel;
/* From now on record a CUDA event pair (on the launching stream) around every
 * launch of one kernel family; cf_profile_read synchronises those events and
 * returns their summed duration, the launch count and the algorithmic flops
 * and bytes of those launches (a model computed at setup: see the design
 * notes), then stops recording.  Adds two event records per launch. */
cf_status cf_profile_start(cf_problem* pb, int kernel);
/* The same, restricted to the launches on one level (-1: all levels);
 * CF_EINVAL for a level outside [-1, cf_n_levels). */
cf_status cf_profile_start_level(cf_problem* pb, int kernel, int level);
cf_status cf_profile_read(cf_problem* pb, double* ms, int64_t* launches, double* flops, double* bytes);

/* ---- host-only handles (no device work; used to check the setup) ---------
 * cf_setup_host builds the same hierarchy as cf_setup on the host only.  The
 * handle answers the size / map / stats queries above and the calls below;
 * every device call on it returns CF_EINVAL. */
cf_status cf_setup_host(const cf_mesh* mesh, const cf_levelset* ls, int degree,
                        const cf_params* params, cf_problem** out);
/* Device memory cf_setup of this problem would hold (hierarchy in both
 * precisions, CG vectors, graph scratch), estimated BEFORE any setup: the
 * call classifies the cells of every level and builds the index lists
 * (DoFs, ghost faces, patches and their DoF sets), but no cut-cell
 * quadrature, element matrix, inverse or right-hand side.  The served form
 * admits requests by this figure (Sec. 5's resident hierarchies) and refuses
 * one that can never fit before building it.  Equal to cf_problem_footprint
 * of the built problem.  Arguments as for cf_setup; *bytes receives the
 * estimate.  Errors as cf_setup's argument checks (CF_EINVAL,
 * CF_EUNSUPPORTED). */
cf_status cf_footprint(const cf_mesh* mesh, const cf_levelset* ls, int degree, const cf_params* params,
                       size_t* bytes);
/* The same estimate for a built handle (host-only or device). CF_EINVAL on null. */
cf_status cf_problem_footprint(const cf_problem* pb, size_t* bytes);
/* Finest-level right-hand side (host array of cf_n_dofs doubles). */
cf_status cf_host_rhs(const cf_problem* pb, double* h_b);
/* cf_rhs_user into a host array (works on host-only handles). */
cf_status cf_host_rhs_user(const cf_problem* pb, double (*f)(const double* x, void* user),
                           double (*g)(const double* x, void* user), void* user, double* h_b);
/* Element matrix of cell `cell` (flat index c_0 + N c_1 + N^2 c_2) of a level:
 * volume + Nitsche terms for a cut cell, the uncut stiffness for an uncut
 * active cell; (p+1)^d x (p+1)^d row-major, local nodes first coordinate
 * fastest.  CF_EINVAL for an inactive cell. */
cf_status cf_host_cell_matrix(const cf_problem* pb, int level, int64_t cell, double* h_out);
/* Number of interior (fast-diagonalisation) and cut (dense inverse) patches. */
cf_status cf_host_patch_counts(const cf_problem* pb, int level, int64_t* n_interior, int64_t* n_cut);
/* Interior patch j: its vertex (lattice vertex index v_0 + (N+1) v_1 + ..). */
cf_status cf_host_interior_patch(const cf_problem* pb, int level, int64_t j, int64_t* vertex);
/* The exact local solve of an interior patch of a level (Sec. 2.3, every
 * interior patch has the same local matrices) as one dense map:
 * x_I <- A_I^{-1} b_I - A_I^{-1} A_{I,B} x_B.  h_W: (2p-1)^d x (2p+1)^d
 * row-major; rows = interior nodes, columns = closure nodes, both first
 * coordinate fastest; b enters at interior columns, x at boundary columns. */
cf_status cf_host_interior_update(const cf_problem* pb, int level, double* h_W);
/* Diagonal of A_level (host array of cf_level_n_dofs doubles, DoF order):
 * the point-Jacobi scaling of the Chebyshev smoother.  Levels >= 1. */
cf_status cf_host_diagonal(const cf_problem* pb, int level, double* h_d);
/* The coarsest-level solve's explicit inverse A_0^{-1} (Sec. 2.2: exact
 * solve on the coarsest mesh): cf_level_n_dofs(pb, 0)^2 doubles, row-major,
 * rows and columns in the level's DoF order.  Caller-owned host array. */
cf_status cf_host_coarse_inverse(const cf_problem* pb, double* h_inv);
/* Cut patch j: vertex, DoF count m, lattice indices of its m DoFs (h_nodes,
 * room for (2p+1)^d) and, if h_inv is not NULL, the m x m explicit inverse
 * of A[I_j, I_j] (row-major, in the order of h_nodes). */
cf_status cf_host_cut_patch(const cf_problem* pb, int level, int64_t j, int64_t* vertex, int* m,
                            int64_t* h_nodes, double* h_inv);

#ifdef __cplusplus
}
#endif

#endif /* CUTMG_H */
