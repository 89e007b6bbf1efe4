/*
 * rm.h -- C ABI of the GB300 (sm_103a) solvers for the weighted Riesz maps
 *
 *     beta u - div(alpha grad u) = f      (k = 0, H(grad), Q_p)
 *     beta u + curl(alpha curl u) = f     (k = 1, H(curl), NCE_p)
 *     beta u - grad(alpha div u) = f      (k = 2, H(div),  NCF_p)
 *
 * of Brubeck & Farrell, "Multigrid solvers for the de Rham complex with
 * optimal complexity in polynomial degree" (arXiv 2211.14284), Sec. 1 Eqs.
 * hgrad/hcurl/hdiv, weak form Eq. common_weak_formulation with
 * Gamma_D = boundary of the unit cube (or empty: rm_options.boundary).
 *
 * Discretisation: structured n1 x n2 x n3 hexahedral mesh with trilinear
 * cells, the FDM bases of Sec. 2 (interior functions orthonormal in L2 and
 * H(d) on the reference cell), GLL quadrature with ceil(3(p+1)/2) points per
 * direction (Sec. 5).  Preconditioner: the additive two-level Schwarz
 * relaxations of Sec. 4 -- PAFW vertex stars (Eq. asm-afw), their
 * statically-condensed form on the sparse auxiliary operator (Sec. 3.2,
 * Eqs. sc-pafw, sc-asm-afw) and the SC Pavarino-Hiptmair form for H(curl)
 * and H(div) (Eq. sc-asm-hiptmair) -- with exact or incomplete Cholesky patch factors
 * (Sec. 4.5) and a p = 1 coarse correction.
 *
 * VECTOR LAYOUT (every vector argument): FDM-basis coefficients on the
 * per-component lattice.  Component m of form degree k has, per direction
 * d, type 's' (continuous, N_d = n_d p + 1 points) or 'r' (discontinuous,
 * N_d = n_d p points):  k=0: (s,s,s);  k=1: (r,s,s),(s,r,s),(s,s,r);
 * k=2: (s,r,r),(r,s,r),(r,r,s).  Entry (g1,g2,g3) of component m is at
 * offset_m + g1 + N1 (g2 + N2 g3); components are concatenated.  Local
 * index i_d of cell e_d sits at g_d = e_d p + i_d.  Entries with an s-type
 * index g_d in {0, n_d p} are Dirichlet (RM_BC_DIRICHLET): ignored on input,
 * 0 on output; with RM_BC_NONE every entry is a DOF.
 *
 * MESH LAYOUT: vertex (a1,a2,a3) at row a1 + (n1+1)(a2 + (n2+1) a3) of a
 * host array of 3 doubles per vertex; cell (e1,e2,e3) has corners
 * (e1+c1, e2+c2, e3+c3), reference coordinate xi_d = -1 at c_d = 0.
 * Per-cell coefficients: cell (e1,e2,e3) at e1 + n1 (e2 + n2 e3).
 *
 * OWNERSHIP: the caller owns every vector (device memory, 16-byte aligned,
 * valid on the handle's stream).  The handle owns all internal buffers.
 * Host inputs of rm_setup are copied; they may be freed on return.
 *
 * ERRORS: every call returns an rm_status; 0 = RM_OK.  rm_last_error(h)
 * gives a message (h = NULL: the last failure of rm_setup on this thread).
 * There is no CPU fallback: a missing or failing CUDA device is an error.
 */
#ifndef RM_H
#define RM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RM_OK = 0,
  RM_ERR_ARG = 1,           /* invalid argument or unsupported combination */
  RM_ERR_CUDA = 2,          /* a CUDA call failed */
  RM_ERR_OOM = 3,           /* device or host allocation failed */
  RM_ERR_BREAKDOWN = 4,     /* ICC pivot <= 0, or CG p^T A p <= 0 */
  RM_ERR_NOT_CONVERGED = 5, /* max_it reached */
  RM_ERR_NAN = 6,           /* NaN/Inf in a residual */
  RM_ERR_TIMEOUT = 7        /* a bounded device wait gave up (reported by the next rm_solve) */
} rm_status;

typedef enum { RM_HGRAD = 0, RM_HCURL = 1, RM_HDIV = 2 } rm_space;

typedef enum { RM_FP64 = 0, RM_FP32 = 1 } rm_precision;
typedef enum { RM_PAFW = 0, RM_PH = 1 } rm_decomposition;
typedef enum { RM_CHOL = 0, RM_ICC = 1 } rm_factor;
/* RM_COARSE_P1: exact p = 1 coarse solve (dense inverse, <= 16,384 coarse DOFs);
 * RM_COARSE_GMG: the p = 1 problem approximated by one symmetric V(2,2)
 * geometric multigrid cycle (Galerkin levels, damped Jacobi), as the paper's
 * p-coarse GMG; for coarse spaces too large for the dense inverse. */
typedef enum { RM_COARSE_NONE = 0, RM_COARSE_P1 = 1, RM_COARSE_GMG = 2 } rm_coarse;
/* Smoother of the RM_COARSE_GMG cycle for H(curl) and H(div) (H(grad) always
 * uses damped point Jacobi).  RM_SMOOTH_STAR: additive vertex stars (exact
 * star solves, weight 1/8).  RM_SMOOTH_HIPTMAIR: the paper's Hiptmair-Jacobi
 * relaxation on the p-coarse space (Sec. 5.1, solver diagram): a damped
 * Jacobi sweep on A, then one on the potential operator G^T A G through the
 * lowest-order discrete gradient (H(curl)) or curl (H(div)) G, in reverse
 * order after the coarse correction; weights 1 / ||D^-1 M||_inf. */
typedef enum { RM_SMOOTH_STAR = 0, RM_SMOOTH_HIPTMAIR = 1 } rm_smoother;
/* How the fine relaxation S and the coarse correction C combine.
 * RM_ADDITIVE: B = S + C (Eqs. asm-afw, asm-hiptmair).  RM_HYBRID: the
 * hybrid multigrid/Schwarz V(1,1) cycle of the paper's experiments (Sec. 5):
 * z = w S r; z += C (r - A z); z += w S (r - A z), w = hybrid_omega; two
 * operator applies per call. */
typedef enum { RM_ADDITIVE = 0, RM_HYBRID = 1 } rm_composition;
/* Stopping test of rm_solve (Sec. 5.1).  RM_NORM_L2: the recursive residual,
 * ||r_k||_2 <= rtol ||b||_2.  RM_NORM_NATURAL: the paper's test, a reduction of
 * the natural norm of the preconditioned residual by 1/rtol,
 * sqrt(r_k^T B r_k) <= rtol sqrt(r_0^T B r_0), B the preconditioner.  Both
 * histories are recorded in either mode (rm_history). */
typedef enum { RM_NORM_L2 = 0, RM_NORM_NATURAL = 1 } rm_norm;
/* Arithmetic of the operator apply y = A x (the CG operator; FP64 in and out
 * in both).  RM_ARITH_FP64: IEEE double throughout.  RM_ARITH_DF64:
 * double-float -- every value the unevaluated sum of two FP32 numbers (about
 * 48 significant bits, FP32 exponent range), products and sums by error-free
 * transformations on the FP32 pipe, which runs at 64x GB300's FP64 rate;
 * results agree with FP64 to ~1e-14 relative while no input or
 * intermediate leaves the FP32 exponent range (|v| in ~1e-30 .. 1e38). */
typedef enum { RM_ARITH_FP64 = 0, RM_ARITH_DF64 = 1 } rm_arith;
/* Gamma_D of the weak form (Eq. common_weak_formulation).  RM_BC_DIRICHLET:
 * the whole boundary of the cube (entries with an s-type index on the
 * boundary are Dirichlet).  RM_BC_NONE: Gamma_D empty, every lattice entry a
 * DOF (natural boundary conditions; the operator is definite while beta > 0
 * on a set of positive measure, as in the paper's Maxwell test, Sec. 5.2). */
typedef enum { RM_BC_DIRICHLET = 0, RM_BC_NONE = 1 } rm_boundary;

typedef struct {
  int nx, ny, nz;          /* cells per direction, each >= 2 */
  const double *vertices;  /* host, (nx+1)(ny+1)(nz+1) x 3; NULL = uniform unit cube */
} rm_mesh;

typedef struct {
  int precision;           /* rm_precision of the preconditioner data and arithmetic */
  int decomposition;       /* RM_PAFW (vertex stars) or RM_PH (H(curl): edge stars +
                              vertex-star gradient potentials; H(div): face stars
                              (point-Jacobi on S) + edge-star curl potentials with
                              the eps = 1e-2 mass shift; static condensation only) */
  int static_condensation; /* 1: patches on the interface Schur complement */
  int factor;              /* RM_CHOL (exact) or RM_ICC (ICC(0) on the SC pattern).
                              Exact factors of uncondensed patches are dense per
                              block and built on the host at a cost growing with
                              the cube of the patch size (minutes for H(div) at
                              p >= 5): condense or take RM_ICC there */
  int coarse;              /* rm_coarse */
  int flexible;            /* 1: flexible CG (Polak-Ribiere beta) */
  double rtol;             /* relative tolerance of the stopping test (norm) */
  int max_it;
  int check_every;         /* iterations between host reads of the residual */
  int profile;             /* 1: time every operator apply and preconditioner call
                              with CUDA events inside rm_solve (reported in rm_info) */
  int norm;                /* rm_norm of the stopping test (default RM_NORM_L2) */
  int arith;               /* rm_arith of the operator apply (default RM_ARITH_FP64) */
  int boundary;            /* rm_boundary (default RM_BC_DIRICHLET) */
  int coarse_smoother;     /* rm_smoother of RM_COARSE_GMG (default RM_SMOOTH_STAR) */
  int composition;         /* rm_composition (default RM_ADDITIVE) */
  double hybrid_omega;     /* RM_HYBRID relaxation weight, 0 < w <= 1 (default 1/8: at
                              most eight vertex stars overlap a DOF) */
  int relaxation;          /* 1 (default): build the preconditioner; 0: the operator
                              alone (rm_apply only; alpha or beta may then be 0, e.g.
                              a mass matrix alone; rm_precondition and rm_solve
                              return RM_ERR_ARG) */
  int deterministic;       /* 0 (default): the patch solves add into z with atomics and
                              the relaxation's branches run concurrently on their own
                              streams (fastest; z may differ in the last bits from run
                              to run); 1: every patch writes its solution to a scratch
                              array, each lattice entry sums its patches' values in a
                              fixed order, the branches run one after another: z = B r
                              and whole solves are bitwise reproducible.  Single-problem
                              handles only (rm_batch_setup and rm_precondition_noalloc
                              refuse it) */
} rm_options;

typedef struct {
  int iterations;
  int status;              /* rm_status of the solve */
  double rel_res_l2;       /* final recursive ||r|| / ||b|| */
  double rel_res_natural;  /* sqrt(r_k^T B r_k / r_0^T B r_0) at the last iterate whose
                              preconditioned residual was formed (the final one under
                              RM_NORM_NATURAL, the one before it under RM_NORM_L2) */
  int iterations_natural;  /* first k with that ratio <= rtol: the paper's count
                              (Sec. 5.1); -1 if not reached within the solve */
  int history_len;         /* entries recorded per history (rm_history) */
  double setup_s;          /* wall time of rm_setup for this handle */
  double solve_ms;         /* device time of the solve, CUDA events */
  double apply_ms;         /* profile = 1: total time of the operator applies */
  int apply_calls;
  double precond_ms;       /* profile = 1: total time of the preconditioner calls */
  int precond_calls;
  long long kernel_launches; /* kernels this library launched during the solve */
  /* learned coarse corrector (rm_corrector_use mode RM_CORRECTOR_LEARNED) */
  int learned_calls;       /* preconditioner calls whose coarse term came from the network */
  int judge_calls;         /* calls on which the plain coarse correction judged it */
  int fallback_at;         /* call at which the judge rejected it (-1: never) */
  double judge_eta;        /* last judged relative A_0-energy error (see rm_corrector_use) */
} rm_info;

typedef struct rm_handle rm_handle;

/* Defaults: FP64, PAFW, no static condensation, exact Cholesky, P1 coarse,
 * CG, rtol 1e-8, max_it 500, check_every 1, RM_NORM_L2, RM_ARITH_FP64,
 * RM_BC_DIRICHLET, RM_SMOOTH_STAR, RM_ADDITIVE, hybrid_omega 1/8, relaxation 1. */
rm_options rm_default_options(void);

/* Builds the discretisation and the preconditioner (host FP64 setup: 1D
 * eigenproblems, auxiliary operator, Schur complement, patch factors,
 * coarse factor) and uploads it.  alpha, beta: host, length nx*ny*nz, or
 * NULL for 1.  stream: a cudaStream_t (NULL = legacy default stream) used by
 * every later call on this handle.  Supported: p in 1..15 when every cell is
 * an axis-aligned box, p in 1..8 otherwise (the general-cell apply's shared
 * memory; larger p returns RM_ERR_ARG); RM_PH only for RM_HCURL or RM_HDIV
 * with static_condensation = 1. */
int rm_setup(rm_handle **h, int space, const rm_mesh *mesh, int p,
             const double *alpha, const double *beta, const rm_options *opt,
             void *stream);

/* Lattice length (all entries) and number of free (non-Dirichlet) DOFs. */
int rm_ndofs(const rm_handle *h, long long *lattice, long long *free_dofs);

/* Shape of lattice component comp (VECTOR LAYOUT above; Sec. 2.4): dims[d] =
 * N_d (n_d p + 1 for an s-type direction, n_d p for an r-type one) and
 * *offset = the component's first entry in a vector (offset may be NULL).
 * comp in 0 .. ncomp-1, ncomp = 1 for RM_HGRAD, 3 otherwise; other values
 * return RM_ERR_ARG. */
int rm_layout(const rm_handle *h, int comp, int dims[3], long long *offset);

/* y = A x: the matrix-free sum-factorised operator of Eq. sum-factorization
 * on the true (trilinear) geometry, FP64.  x, y: device, lattice length;
 * y is overwritten. */
int rm_apply(rm_handle *h, const double *x, double *y);

/* z = B r, the additive two-level relaxation (FP64 in/out whatever the
 * precision option): the vertex-star PAFW sum of Eq. asm-afw, its
 * statically-condensed form Eq. sc-asm-afw (interior solve, harmonic
 * extension, Eq. schur), or the SC Pavarino-Hiptmair form Eq.
 * sc-asm-hiptmair (edge stars plus the gradient of vertex-star potential
 * solves), each plus the p = 1 coarse correction R_0^T A_0^-1 R_0 of Eq.
 * asm-afw.  r, z: device, lattice length; z is overwritten. */
int rm_precondition(rm_handle *h, const double *r, double *z);

/* Preconditioned (flexible) CG for A x = b (Sec. 5.1: zero initial guess,
 * relative tolerance rtol; the stopping norm is options.norm).  b: device
 * (Dirichlet entries ignored).  x: device, in = initial guess (zeros = the
 * paper's setting), out = solution.  info may be NULL.  The preconditioner of
 * the iterations is captured once per corrector mode as a CUDA graph (on a
 * private stream of the handle) and replayed on the handle's stream; with the
 * learned corrector or while recording training residuals it runs eagerly.
 * The host reads the stopping quantity every check_every iterations. */
int rm_solve(rm_handle *h, const double *b, double *x, rm_info *info);

/* Residual history of the last rm_solve on this handle: which = RM_NORM_L2
 * gives ||r_k|| / ||b|| for k = 0 .. iterations, RM_NORM_NATURAL gives
 * sqrt(r_k^T B r_k / r_0^T B r_0) for the iterates whose preconditioned
 * residual was formed.  out: host, cap doubles; *len = entries written
 * (min(cap, recorded)).  The handle keeps max_it + 1 entries per history. */
int rm_history(const rm_handle *h, int which, double *out, int cap, int *len);

/* Number of patches, patch slots and factor nonzeros of the relaxation
 * (summed over patch families), for reporting. */
int rm_stats(const rm_handle *h, long long *patches, long long *slots,
             long long *factor_nnz);

void rm_destroy(rm_handle *h);
const char *rm_last_error(const rm_handle *h);

/* ---- batched solves --------------------------------------------------------
 * Many independent problems of uneven mesh size and degree (Cartesian meshes:
 * every cell an axis-aligned box) solved together with the same options.
 * The problems are set up one by one on the host (as rm_setup would) and
 * concatenated on the device into one block-diagonal system: one launch per
 * patch template (problems of equal space and p share templates), each
 * problem's operator apply by the Cartesian kernel pair of rm_apply (cell
 * products, then the fixed-order assembly, whose grid per (space, p) is
 * picked by timing at setup), lock-step CG with per-problem scalars and
 * convergence masks (converged problems skip their cells, patches and rows),
 * one iteration captured in a CUDA graph and replayed check_every times
 * between host reads of the convergence flags.
 * Coarse correction: RM_COARSE_P1 (exact) or RM_COARSE_NONE. */
typedef struct rm_batch rm_batch;

/* space, meshes, p: host arrays of nprob entries; alpha, beta: host arrays of
 * nprob host pointers (each per-cell, or NULL for 1), or NULL.  stream is
 * unused (the batch runs on its own stream; see rm_batch_solve). */
int rm_batch_setup(rm_batch **b, int nprob, const int *space, const rm_mesh *meshes, const int *p,
                   const double *const *alpha, const double *const *beta, const rm_options *opt,
                   void *stream);
int rm_batch_ndofs(const rm_batch *b, int i, long long *lattice);
/* bvec, x: host arrays of nprob device pointers (problem i's vectors in the
 * layout of rm_apply); x is the initial guess in and the solution out.
 * stream: the caller's stream holding b and x (synchronised on entry; the
 * call returns after the results are written).  infos: nprob entries or
 * NULL.  Returns RM_ERR_NOT_CONVERGED if any problem misses rtol. */
int rm_batch_solve(rm_batch *b, const double *const *bvec, double *const *x, rm_info *infos,
                   void *stream);
void rm_batch_destroy(rm_batch *b);
const char *rm_batch_last_error(const rm_batch *b);

/* z = B r without allocating: the same relaxation as rm_precondition for a
 * handle built without static condensation (vertex-star patches plus the
 * p = 1 coarse correction), for callers that must not allocate device memory
 * while they run -- code that lives inside a device-memory budget owned by
 * another allocator (a framework's caching allocator hands out every byte),
 * or that cannot afford the device-wide synchronisation cudaMalloc/cudaFree
 * imply.  The paper has no counterpart; it is a library convenience.
 *
 * The call performs no cudaMalloc, cudaFree or other allocating call.  Its
 * scratch (2 x RM_NOALLOC_MAX_COARSE doubles) is a static device array of the
 * library, present on every GPU that loads it until the process exits.  Its
 * device address is looked up by rm_setup on the handle's device (again by
 * every rm_setup, so handles created after a cudaDeviceReset see the new
 * context's address); the call itself only reads it.  Every call shares the
 * array: calls that overlap on the GPU race on it.  Accepted: handles without
 * static condensation whose coarse term is the plain p = 1 correction
 * (RM_COARSE_P1, corrector mode RM_CORRECTOR_PLAIN) or none (RM_COARSE_NONE,
 * or mode RM_CORRECTOR_OFF), in either precision.  Returns RM_ERR_ARG for a
 * statically condensed handle (whose relaxation needs lattice-sized
 * scratch), the coarse multigrid cycle or the learned coarse term (their own
 * buffers), or a coarse space larger than RM_NOALLOC_MAX_COARSE.  r, z:
 * device, lattice length, not aliased; z is overwritten. */
#define RM_NOALLOC_MAX_COARSE 8192
int rm_precondition_noalloc(rm_handle *h, const double *r, double *z);

/* Testing aid for the failure path of the bounded device waits (no
 * counterpart in the paper).  on = 1: every warp-per-patch substitution
 * kernel launched afterwards on the current device waits for 16 bytes that
 * its copies never deliver, so each of its CTAs gives up after ~1 s (twice:
 * its wait, then a last wait for its copies), leaves z untouched and records
 * the timeout; rm_solve then returns RM_ERR_TIMEOUT.  on = 0 restores normal
 * operation.  Affects every handle on the device; not for production use.
 * Returns RM_ERR_CUDA if the flag cannot be written. */
int rm_debug_patch_timeout(int on);

/* ---- mixed Hodge Laplacians (Sec. 5.3) ------------------------------------------
 * Find (sigma, u) in V^{k-1} x V^k (k = 1, 2, 3), Gamma_D empty, with
 *     -(tau, sigma) + (d tau, u) = 0,   (v, d sigma) + (d v, d u) = F(v),
 * i.e. K (sigma, u) = (0, F) with K = [[-M_{k-1}, D^T M_k], [M_k D, K_k]]: M the
 * masses, D the discrete exterior derivative d^{k-1} in FDM coefficients, K_k
 * the (d v, d u) term (0 for k = 3).  MINRES, preconditioned by
 * blockdiag(R_{k-1}^-1, R_k^-1) with the Riesz maps (alpha = beta = 1) each
 * inverted approximately by cheb_its Chebyshev iterations (the paper uses 4)
 * preconditioned by its statically condensed relaxation and the p = 1 coarse
 * correction (SC-PAFW on V^0, SC-PH on V^1 and V^2) or, for the L2 block of
 * k = 3, point-Jacobi on the V^3 mass.  Chebyshev interval: [0.9 theta_min,
 * 1.1 theta_max] from the Ritz values of 20 preconditioned CG steps on a
 * seeded right-hand side at setup.  Stops when the natural norm
 * sqrt(r^T P r) of the preconditioned residual has fallen by 1/rtol, from a
 * zero initial guess.  Vectors are (sigma, u) concatenated, each in the
 * VECTOR LAYOUT of its space (every entry a DOF). */
typedef struct rm_hodge rm_hodge;
/* opt: the Riesz blocks' options (precision, factor, arith, coarse) and the
 * solve's rtol and max_it; boundary, static condensation and composition are
 * fixed as above.  mesh and p as in rm_setup. */
int rm_hodge_setup(rm_hodge **h, int k, const rm_mesh *mesh, int p, const rm_options *opt, int cheb_its,
                   void *stream);
int rm_hodge_ndofs(const rm_hodge *h, long long *n_sigma, long long *n_u);
/* the Chebyshev intervals [a, b] of the two blocks (host, 2 doubles each or NULL) */
int rm_hodge_intervals(const rm_hodge *h, double interval0[2], double interval1[2]);
/* y = K x; x, y device, n_sigma + n_u, not aliased */
int rm_hodge_apply(rm_hodge *h, const double *x, double *y);
/* z = the block preconditioner applied to r (device, not aliased) */
int rm_hodge_precondition(rm_hodge *h, const double *r, double *z);
/* x = MINRES solution of K x = b (b device, x device out; zero initial
 * guess); info: iterations, status, rel_res_natural (the final natural-norm
 * ratio), solve_ms, setup_s; rel_res_l2 = -1. */
int rm_hodge_solve(rm_hodge *h, const double *b, double *x, rm_info *info);
void rm_hodge_destroy(rm_hodge *h);
const char *rm_hodge_last_error(const rm_hodge *h);

/* ---- learned coarse corrector (H(grad) only) ---------------------------------
 * Not in the paper.  A small convolutional network N (a 3D U-Net, BF16
 * weights and activations, FP32 accumulation; its layers are listed at
 * rm_net_create) maps the coarse residual r_0 = R_0 r (R_0 the restriction of
 * the p = 1 coarse correction, Sec. 4.1) and the log-coefficient on the
 * vertex grid of the coarse space to a coarse correction c_L:
 *     x = (sqrt(n_0) r_0 / ||r_0||, log alpha - mean) at the grid vertices
 *     c_L = N(x) at the free vertices,   c = t c_L,   t = (c_L^T r_0) / (c_L^T A_0 c_L)
 * t is the step that minimises the A_0-energy error of c along c_L, so the
 * term added to the Schwarz relaxation is R_0^T c in place of R_0^T A_0^-1 r_0.
 * The plain coarse correction c_P (RM_COARSE_P1 or RM_COARSE_GMG of the
 * handle) is its judge: on judged calls
 *     eta^2 = 1 - (c_L^T r_0)^2 / ((c_L^T A_0 c_L)(r_0^T c_P)),
 * the A_0-energy error of c relative to that of c_P = A_0^-1 r_0, and an eta
 * above judge_max makes the solve fall back to c_P for the rest of the solve.
 * The preconditioner is then nonlinear: rm_solve uses flexible CG. */
typedef struct {
  int pairs;               /* (residual, error) pairs to collect (default 2000) */
  int epochs;              /* passes over the training pairs (default 20) */
  int batch;               /* samples per Adam step (default 16) */
  float lr;                /* Adam step (default 1e-3; halved at 1/2 and 3/4 of the epochs) */
  int levels;              /* network levels below the coarse grid (default 3) */
  int width;               /* channels C_0 of the finest level (default 16) */
  unsigned long long seed; /* initial weights and sample order */
  double val_fraction;     /* pairs held out for validation (default 0.1) */
  int target_cycles;       /* with RM_COARSE_GMG: V-cycles per target (default 12) */
  double off_fraction;     /* pairs recorded from one-level solves (no coarse term,
                              64 iterations each), the rest from plain two-level
                              solves (default 0) */
  int rounds;              /* on-policy rounds after the first training (default 0):
                              each records round_pairs more pairs from solves that
                              use the current network (unjudged), computes their
                              targets and trains round_epochs more epochs on all
                              training pairs */
  int round_pairs;         /* pairs per round (default 500) */
  int round_epochs;        /* epochs per round (default 5) */
} rm_train_options;

typedef struct {
  int pairs, solves;       /* pairs collected (all rounds), solves run to collect them */
  long long params;        /* network parameters */
  double gen_s, train_s;   /* wall time of data generation and of training */
  double train_loss;       /* mean squared error over the last epoch */
  double val_loss;         /* mean squared error on the held-out pairs */
  double val_eta;          /* mean eta (above, with the exact target) on the held-out pairs */
} rm_train_info;

rm_train_options rm_default_train_options(void);

/* Collects training pairs and trains the handle's corrector on the GPU.
 * Pairs: the handle's solver is run on the right-hand sides rhs[i * lattice ..]
 * (device, nrhs vectors in the layout of rm_apply), first without a coarse
 * term (off_fraction of the pairs), then with the plain coarse correction; at
 * every preconditioner call r_0 = R_0 r is recorded, until o->pairs are
 * collected (nrhs too small: RM_ERR_ARG).  Each
 * pair's target is A_0^-1 r_0 (RM_COARSE_P1: the dense inverse; RM_COARSE_GMG:
 * target_cycles iterations of the V-cycle).  Inputs and targets are scaled to
 * sqrt(n_0) / norm.  Training: Adam on the mean squared error over the free
 * vertices, hand-written forward and backward kernels.  Replaces any previous
 * network; leaves the corrector mode unchanged.  info may be NULL. */
int rm_corrector_train(rm_handle *h, const rm_train_options *o, int nrhs, const double *rhs,
                       rm_train_info *info);

/* Writes / reads the network (magic "RMCORR01", int32 dims[3], levels, width,
 * in_channels, int64 parameter count, FP32 parameters in the order of
 * rm_net_get_params).  Loading checks that the grid matches the handle's
 * coarse space. */
int rm_corrector_save(const rm_handle *h, const char *path);
int rm_corrector_load(rm_handle *h, const char *path);

typedef enum {
  RM_CORRECTOR_PLAIN = 0,   /* the plain coarse correction (default) */
  RM_CORRECTOR_LEARNED = 1, /* the network, judged by the plain correction */
  RM_CORRECTOR_OFF = 2      /* no coarse term (one-level relaxation), for comparison */
} rm_corrector_mode;

/* Selects the coarse term of later rm_precondition / rm_solve calls.
 * judge_every: judge calls 0, judge_every, 2 judge_every, ... of each solve
 * (0: never); judge_max: the largest eta accepted.  LEARNED needs a trained
 * or loaded network. */
int rm_corrector_use(rm_handle *h, int mode, int judge_every, double judge_max);

/* ---- the corrector's network on its own ----------------------------------------
 * Layers (levels L, width C, input channels c_in, grid D_0 = dims; level l has
 * the grid D_l = (D_{l-1} - 1)/2 + 1 and C 2^l channels; every conv 3x3x3
 * with zero padding, ReLU after all but the last):
 *   e0a = conv(x), e0 = conv(e0a); for l = 1..L: d_l = conv_stride2(e_{l-1}),
 *   e_l = conv(d_l); h_L = e_L; for l = L-1..0: u_l = up(h_{l+1}) (vertex-centred
 *   linear interpolation), a_l = conv(u_l), s_l = a_l + e_l, h_l = conv(s_l);
 *   y = conv(h_0) (one channel, no ReLU).
 * A stride-2 conv reads its input at 2 o + tap - 1.  Parameters: per conv in
 * that order W[c_out][27][c_in] (tap (dz * 3 + dy) * 3 + dx for the offset
 * (dx-1, dy-1, dz-1)), then b[c_out].  Tensors are channels-last FP32 on the
 * device, [batch][voxel][channel] with voxel (z * ny + y) * nx + x; the
 * kernels round activations and weights to BF16 and accumulate in FP32.
 * Errors: rm_net_last_error() (this thread). */
typedef struct rm_net rm_net;
int rm_net_create(rm_net **net, const int dims[3], int levels, int width, int in_channels,
                  int max_batch, unsigned long long seed, void *stream);
long long rm_net_num_params(const rm_net *net);
int rm_net_get_params(const rm_net *net, float *params);  /* host, FP32 master copy */
int rm_net_set_params(rm_net *net, const float *params);  /* host; resets Adam */
/* x: device [batch][voxel][in_channels]; y: device [batch][voxel] */
int rm_net_forward(rm_net *net, int batch, const float *x, float *y);
/* After rm_net_forward: gradients of sum(dy * y).  grad: device, num_params
 * (or NULL); dx: device, shaped like x (or NULL). */
int rm_net_backward(rm_net *net, const float *dy, float *grad, float *dx);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradients. */
int rm_net_adam(rm_net *net, float lr);
void rm_net_destroy(rm_net *net);
const char *rm_net_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RM_H */
