/*
 * xfft.h -- C-ABI of the GB300 (sm_103a) X-FFT solver for periodic 3D linear-elastic
 * homogenization with an X-FEM discretization (Gehrig & Schneider, arXiv 2601.02172).
 *
 * Problem statement (Sec. 2.1): find the periodic displacement fluctuation u_h in the X-FEM
 * space V_h (eq. X-FEM_space: standard P1 functions on six tetrahedra per voxel plus enriched
 * functions N_X^j = N_FE^j rho^m with the modified abs enrichment rho^m, eq.
 * modifiedabsEnrichment) such that  int_Y grad^s v : C : (eps_bar + grad^s u_h) dV = 0  for
 * all v in V_h (eq. discreteFormConti), with a mean-free standard part.  The enriched
 * functions are scaled to unit energy norm (eqs. scaledEnrichedFunction, XFFT_diagonal), and
 * the system is solved by linear CG (Algorithm 1) preconditioned with
 * P = diag(A0_11, I) (eq. scaledPreconditioner), A0_11 inverted by FFT (eq. GreenHermitian).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Grid: n[0] x n[1] x n[2] voxels on the cell [0,len[0]] x [0,len[1]] x [0,len[2]]; the
 *    periodic nodes are indexed  node = (i * n[1] + j) * n[2] + k  (C order, last axis
 *    fastest).  Voxel v has its lowest corner at node v.  Every n[a] must be even, of the form
 *    2^a 3^b 5^c, and between 4 and 1024.
 *  - Strains and stresses are Mandel 6-vectors, order (11, 22, 33, 23, 13, 12) with sqrt(2)
 *    on the shear entries; a 6x6 stiffness is stored row-major.
 *  - Phases: L < 0 is the "minus" phase, L > 0 the "plus" phase; each phase is isotropic and
 *    given by its Lame pair (lambda, mu).  An optional per-voxel factor s_v scales C in voxel v.
 *  - Field layouts (per right-hand side, contiguous, one RHS after the other):
 *      standard DOFs  u_std[rhs][c][node]    c = 0..2, node = 0..N-1   (N = n0 n1 n2)
 *      enriched DOFs  u_enr[rhs][c][j]       j = enriched id 0..nX-1 (increasing node index)
 *    Enriched values exchanged through this API are the *unscaled* coefficients u_X of
 *    eq. X-FEM_space (u_X = D^{-1/2} u~_X) unless a function says otherwise.
 *  - Pointers: every pointer argument is caller-owned.  ptrs_on_device = 1 means all array
 *    arguments of that call are device pointers (on the context's GPU); 0 means host memory
 *    (the call copies through pinned staging buffers).  Small fixed-size arguments (Lame
 *    pairs, eps_bar, C_eff, dL_dCeff, dL_dlame, stats) are always host memory.
 *  - Streams: all device work is enqueued on the stream given to xfft_create (0 = legacy
 *    default stream).  Calls that return host results synchronise that stream.
 *  - Errors: no function aborts, traps or exits; each returns an xfft_status and stores a
 *    message retrievable with xfft_last_error() (thread-local).  On XFFT_ENOTCONV the outputs
 *    hold the last iterate.
 *  - The library allocates its own device workspace with cudaMalloc and frees it in
 *    xfft_destroy.
 */
#ifndef XFFT_H
#define XFFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xfft_ctx xfft_ctx; /* opaque, library-owned */

typedef enum {
  XFFT_OK = 0,
  XFFT_EINVAL = 1,       /* invalid argument (sizes, NULL pointers, unsupported grid) */
  XFFT_ENOMEM = 2,       /* device or pinned allocation failed */
  XFFT_ECUDA = 3,        /* a CUDA runtime call failed; see xfft_last_error() */
  XFFT_ENOTCONV = 4,     /* maxit reached before the stopping rule held */
  XFFT_EBREAKDOWN = 5,   /* CG breakdown: <A d, d> <= 0 or a NaN/Inf scalar */
  XFFT_ETIMEOUT = 6,     /* a device-driven iteration loop reached spin_limit_ns */
  XFFT_EUNSUPPORTED = 7, /* valid request that the library does not implement */
  XFFT_ESTATE = 8        /* call order violated (e.g. solve before set_microstructure) */
} xfft_status;

/* Arithmetic of the kernels.  XFFT_DW (double-word, an unevaluated sum of two floats, about 48
 * significant bits, run on the FP32 units) is used by XFFT_FP32_REFINED for its residuals and
 * stress integrals; xfft_apply also accepts it directly. */
enum { XFFT_FP64 = 0, XFFT_FP32_REFINED = 1, XFFT_DW = 2 };
/* Preconditioner on the enriched DOFs.  XFFT_ENR_IDENTITY: the identity on the scaled DOFs,
 * P = diag(A0_11, I) (eq. scaledPreconditioner; the paper's choice).  XFFT_ENR_BLOCK3 (a variant,
 * not in the paper): per enriched node j the inverse of the 3x3 block
 *   B_j,kl = D0_jk^-1/2 D0_jl^-1/2 int sym(grad N_X^j (x) e_k) : sym(grad N_X^j (x) e_l)
 * of the scaled enriched reference Gram matrix (unit diagonal by eq. XFFT_diagonal), factorised
 * in FP64 at xfft_set_microstructure (XFFT_EBREAKDOWN if a block is not positive definite).
 * The discrete system and its solution do not depend on this choice; iteration counts do. */
enum { XFFT_ENR_IDENTITY = 0, XFFT_ENR_BLOCK3 = 1 };

typedef struct {
  int n[3];       /* voxels per axis */
  double len[3];  /* cell edge lengths */
} xfft_grid;

/* Iteration scheme on the same system and preconditioner (Sec. 2.3, next to Algorithm 1):
 * XFFT_SCHEME_CG the linear CG of Algorithm 1; XFFT_SCHEME_BASIC the basic scheme, a
 * preconditioned Richardson iteration u += s0 P^-1 f with s0 = 2 / (C_- + C_+) (eq. stepsize;
 * C_-, C_+ the smallest and largest eigenvalues 2 mu, 3 lambda + 2 mu of the phases' stiffness,
 * times the extreme voxel scales); XFFT_SCHEME_BB Barzilai-Borwein in the P metric, whose step
 * is the previous iteration's exact line-search step f^T P^-1 f / <d, A d> (s0 first);
 * XFFT_SCHEME_NLCG the nonlinear CG the paper compares (Sec. 2.3): the fixed step s0 without a
 * line search and the Fletcher-Reeves momentum beta = f_k^T P^-1 f_k / f_{k-1}^T P^-1 f_{k-1}. */
enum { XFFT_SCHEME_CG = 0, XFFT_SCHEME_BASIC = 1, XFFT_SCHEME_BB = 2, XFFT_SCHEME_NLCG = 3 };
/* Step rule of XFFT_SCHEME_BB.  The paper cites the Barzilai-Borwein scheme (Sec. 2.3) without
 * its formula, so every classical rule is offered; du = s d and dg = A du are the previous
 * iteration's changes of the iterate and of the gradient (d = P^-1 f, steepest descent):
 *   XFFT_BB1        <du, P du> / <du, dg>       (metric of P; equals the previous exact
 *                                                 line-search step; default)
 *   XFFT_BB2        <du, dg> / <dg, P^-1 dg>    (metric of P; from scalars already reduced)
 *   XFFT_BB_ALT     BB1 and BB2 in turn (BB2 first)
 *   XFFT_BB1_EUCLID <du, du> / <du, dg>         (Euclidean metric of the scaled DOFs)
 *   XFFT_BB2_EUCLID <du, dg> / <dg, dg>
 * The Euclidean rules are not invariant under a change of length unit (A scales like length,
 * P^-1 A does not); they need one more reduction pass per iteration. */
enum { XFFT_BB1 = 0, XFFT_BB2 = 1, XFFT_BB_ALT = 2, XFFT_BB1_EUCLID = 3, XFFT_BB2_EUCLID = 4 };

typedef struct {
  int precision;       /* XFFT_FP64 (all FP64) or XFFT_FP32_REFINED (FP32 CG; residuals of the
                          FP64 iterate in double-word arithmetic) */
  double tol;          /* stopping rule sqrt(r^T P^-1 r / |Y|) <= tol * ||<sigma>_Y|| (eqs.
                          stoppingCriterion, convergence) */
  int maxit;           /* CG iteration cap (FP64) or inner cap per refinement step */
  double snap_tau;     /* |L| < snap_tau counts as on the interface (Sec. 3); <= 0: 1e-6 * min h */
  int enr_precond;     /* XFFT_ENR_IDENTITY (the paper's choice) or XFFT_ENR_BLOCK3 */
  double inner_tol;    /* FP32_REFINED: smallest relative residual reduction asked of one FP32
                          inner solve (each inner solve aims at half the outer tolerance) */
  int max_refine;      /* FP32_REFINED: cap on FP64 refinement steps */
  int poll_every;      /* iterations between host checks of the device convergence flags */
  int scheme;          /* XFFT_SCHEME_CG (Algorithm 1, default), _BASIC, _BB or _NLCG */
  double step;         /* step of the basic / BB schemes; <= 0: s0 = 2 / (C_- + C_+) */
  int cut_cache;       /* FP32_REFINED: 1 caches each cut tet's scaled 24 x 24 element matrix
                          (FP32, packed upper triangle, 1200 bytes per cut tet) at
                          xfft_set_microstructure and applies it in the FP32 CG iterations (the
                          paper's caching strategy, Sec. 2.3); 0 (default) recomputes the element
                          action from the 32 per-side moments at every apply, which is about three
                          times faster on GB300 (the cached matrices make the kernel wait on
                          memory) */
  int bb_rule;         /* XFFT_SCHEME_BB: the step rule (XFFT_BB1 default) */
  int bb_cycle;        /* XFFT_SCHEME_BB: the step is renewed every bb_cycle iterations and kept
                          in between (cyclic BB; 1 = every iteration, the default) */
  int enrichment;      /* 1 (default): the X-FEM space of eq. X-FEM_space.  0: the P1 baseline of
                          the paper's discretization table (Sec. 4.1), voxel-segmented P1 elements
                          without enrichment: each voxel takes the phase of its centre, where the
                          level set is the mean of its eight corner values (several level sets:
                          the first one negative there), and nX = 0 */
  long long max_device_bytes; /* cap on the context's own device allocations (0 = none); a
                          request above it fails with XFFT_ENOMEM as a failed cudaMalloc would */
  long long spin_limit_ns; /* limit on the device time of one device-driven iteration loop (the
                          CG iterations between two residual checks run as one CUDA graph whose
                          while node repeats poll_every iterations until no right-hand side is
                          active); past it the loop stops, the outputs hold the last iterate and
                          the call returns XFFT_ETIMEOUT.  < 0 (default): no limit */
  int autotune;        /* FP32_REFINED: 1 (default) times candidate launch shapes of the cut-tet
                          kernel (grid size, right-hand sides per launch) and of the
                          preconditioner (right-hand sides per group of FFT passes) on the
                          microstructure at its first solve and keeps the fastest (cached per
                          grid and cut-tet count for the process; see xfft_get_tuning); 0 keeps
                          the defaults */
  int residual_update; /* FP32_REFINED (iterative refinement with a residual update, not in the
                          paper): 1 (default) recomputes the residual of the FP64 iterate in
                          double-word arithmetic until it is below 100 * tol (stopping-rule
                          measure), and from then on updates it, r_k = r_{k-1} - A delta_k and
                          <sigma>_k = <sigma>_{k-1} + <C grad^s delta_k>, with the FP32 operator
                          applied to the last inner solve's correction delta_k: the FP32 rounding
                          of A delta_k is far below the tolerance once delta_k is that small.
                          0: every residual recomputed in double-word arithmetic */
} xfft_options;

typedef struct {
  int n_rhs;
  int iters[64];        /* CG iterations per RHS (sum over refinement steps) */
  double final_res[64]; /* sqrt(r^T P^-1 r / |Y|) / ||<sigma>|| at exit, per RHS */
  int refine_steps;     /* FP64 residual evaluations after the first (FP32_REFINED) */
  int n_fe, n_x, n_cut_tets;
  double ms_setup, ms_solve;
} xfft_stats;

/* Fill *opt with the defaults: FP64, tol 1e-10, maxit 10000, snap_tau 0 (=> 1e-6 min h),
 * identity enriched block, inner_tol 1e-5, max_refine 20, poll_every 8, linear CG, cut_cache 0,
 * bb_rule XFFT_BB1, bb_cycle 1, enrichment 1, max_device_bytes 0, spin_limit_ns -1, autotune 1,
 * residual_update 1. */
xfft_status xfft_default_options(xfft_options* opt);

/* Create a context for one grid.  stream: a cudaStream_t (or NULL for the legacy stream).
 * Uses the current CUDA device.  Errors: EINVAL for an unsupported grid or options. */
xfft_status xfft_create(xfft_ctx** ctx, const xfft_grid* grid, const xfft_options* opt,
                        void* stream);

/* Load a microstructure (Sec. 2.1 level set, eq. levelset): nodal level set L (N doubles,
 * node order), phase Lame pairs, optional per-voxel scale (N floats, voxel order, or NULL).
 * Runs the setup on the GPU: snapping (Sec. 3), cut-tet classification and enriched-node
 * numbering (eq. X-FEM_space), per-side sub-tetrahedron moments of every cut tet (Sec. 3,
 * Fig. subdivision), the scaling factors D0 (eq. XFFT_diagonal, per DOF).
 * Errors: EINVAL (NULL L, non-positive mu), ECUDA, ENOMEM. */
xfft_status xfft_set_microstructure(xfft_ctx* ctx, const double* L, const double lame_minus[2],
                                    const double lame_plus[2], const float* voxel_scale,
                                    int ptrs_on_device);

/* Several interfaces (Sec. 4.2: the coated sphere of Hashin's neutral inclusion has an
 * inclusion, a coating and a matrix phase).  n_levelsets = K (1 .. XFFT_MAX_LEVELSETS) nodal
 * level sets L (K x N doubles, level set after level set, node order) and K + 1 phases, lame
 * ((K + 1) x 2 doubles, host: lambda, mu of phase 0, 1, ...).  A point lies in phase k if L_k is
 * the first level set that is negative there, in phase K if none is: for nested inclusions pass
 * the innermost first (coated sphere: L_0 = r - r_inclusion, L_1 = r - r_coating).  Each tet is
 * cut by at most one interface, the zero set of its first level set with a negative vertex, and
 * is enriched with the modified abs of that level set (eq. modifiedabsEnrichment); one
 * enrichment vector per node.  K = 1 with lame = {lambda_-, mu_-, lambda_+, mu_+} is
 * xfft_set_microstructure.  Errors as xfft_set_microstructure, and EINVAL if some tet is cut
 * by two interfaces (the two zero sets pass through one element).  Gradients: xfft_grad_phases. */
#define XFFT_MAX_LEVELSETS 2
xfft_status xfft_set_microstructure_phases(xfft_ctx* ctx, int n_levelsets, const double* L,
                                           const double* lame, const float* voxel_scale,
                                           int ptrs_on_device);

/* Solve the cell problem for n_rhs (1..64) macroscopic strains eps_bar (n_rhs x 6 Mandel,
 * host).  Outputs (each may be NULL): u_std (n_rhs x 3 x N), u_enr (n_rhs x 3 x nX, unscaled
 * u_X), voxel_stress (n_rhs x 6 x N: per-voxel average stress, voxel order),
 * mean_stress (n_rhs x 6, host: <sigma>_Y).  The solution is kept in the context (for
 * xfft_grad).  Returns ENOTCONV if some RHS hit maxit (outputs hold the last iterate). */
xfft_status xfft_solve(xfft_ctx* ctx, int n_rhs, const double* eps_bar, double* u_std,
                       double* u_enr, double* voxel_stress, double* mean_stress,
                       xfft_stats* stats, int ptrs_on_device);

/* Solve the six unit Mandel load cases and return the 6x6 effective stiffness (row-major,
 * C_eff[i*6+k] = <sigma_i> for eps_bar = E_k; Sec. 4.1 relation of <sigma> and C_eff).
 * The six converged fields stay in the context as the checkpoint for xfft_grad. */
xfft_status xfft_effective_stiffness(xfft_ctx* ctx, double C_eff[36], xfft_stats* stats);

/* Batch of microstructures (uneven grids allowed, at most 64): xfft_effective_stiffness on each of
 * the n contexts, all at once (the benchmark spec's batching of many microstructures; the paper
 * solves one at a time).  The contexts advance in lockstep: the residual phases of all contexts
 * run on their own streams, then every inner CG solve of every context still iterating runs as
 * ONE device-driven graph launch (a conditional while node whose body holds poll_every
 * iterations of each context, forked onto the contexts' streams, and a kernel that ends the
 * loop once no right-hand side of any context is active), so the host does not poll between
 * iterations.  Contexts need their own non-legacy streams and tracing off; otherwise (or where
 * conditional graphs are unavailable) each context runs from its own host thread.  spin_limit_ns:
 * the smallest limit of the contexts applies to the shared loop.  C_eff: n x 36 (host), stats: n
 * entries or NULL (ms_solve is the whole batch's device time).  The first error (or ENOTCONV /
 * ETIMEOUT) is returned with the context's index in the message; every context is solved. */
xfft_status xfft_batch_effective_stiffness(int n, xfft_ctx* const* ctxs, double* C_eff,
                                           xfft_stats* stats);

/* Gradient of a scalar loss through C_eff: given G = dLoss/dC_eff (6x6 row-major, host),
 * return dLoss/d(lambda_minus, mu_minus, lambda_plus, mu_plus) in dL_dlame[4] (host) and,
 * if dL_dscale != NULL, dLoss/ds_v (N floats, voxel order).  Uses the envelope identity
 * dC_kl/dtheta = (1/|Y|) int eps_k : dC/dtheta : eps_l on the six checkpointed load cases
 * of the last xfft_effective_stiffness call (not in the paper; App. A gives the identity's
 * ingredients).  C_energy (36, host, may be NULL) receives the energy-form C_eff.
 * Errors: ESTATE if no six-case solve is stored; EINVAL for a microstructure of more than two
 * phases (use xfft_grad_phases). */
xfft_status xfft_grad(xfft_ctx* ctx, const double dL_dCeff[36], double dL_dlame[4],
                      float* dL_dscale, double C_energy[36], int ptrs_on_device);

/* xfft_grad for any number of phases (xfft_set_microstructure_phases): dL_dlame receives
 * 2 (K + 1) values, dLoss/d(lambda_0, mu_0, lambda_1, mu_1, ...) (host).  Two phases: the
 * same values and order as xfft_grad. */
xfft_status xfft_grad_phases(xfft_ctx* ctx, const double dL_dCeff[36], double* dL_dlame,
                             float* dL_dscale, double C_energy[36], int ptrs_on_device);

/* Step-level entry points (each is one piece of Algorithm 1 and is what the parity tests
 * call).  Vectors here use the *scaled* enriched coefficients u~_X of eq. scaledEnrichedU and
 * the full DOF layout [std (3N) | enr (3 nX)] per RHS.
 *   xfft_apply:        q = A d  (+ b(eps_bar) when eps_bar != NULL), i.e. the residual map of
 *                      eq. resVector with the sign of eq. linearSystem; also returns, per RHS,
 *                      int_Y C (eps_bar + grad^s d) in sigma_int (n_rhs x 6, host, may be NULL).
 *                      With eps_bar and sigma_int both NULL and XFFT_FP32_REFINED it runs the
 *                      kernels of the FP32 CG iterations (cached cut-tet matrices if cut_cache).
 *   xfft_precondition: z = P^{-1} f with P = diag(A0_11, I) (eqs. scaledPreconditioner,
 *                      GreenHermitian); the standard part of f must have zero mean per
 *                      component.  rr (n_rhs, host, may be NULL) receives f^T z.
 * precision: XFFT_FP64, XFFT_FP32_REFINED (= 1, the FP32 kernels) or XFFT_DW (xfft_apply only:
 * double-word kernels); inputs and outputs stay double.  Other values: XFFT_EINVAL. */
xfft_status xfft_apply(xfft_ctx* ctx, int n_rhs, const double* d, const double* eps_bar,
                       double* q, double* sigma_int, int precision, int ptrs_on_device);
xfft_status xfft_precondition(xfft_ctx* ctx, int n_rhs, const double* f, double* z,
                              double* rr, int precision, int ptrs_on_device);

/* Setup results for inspection: enr_nodes (nX ints), D0 (nX x 3 doubles, eq. XFFT_diagonal
 * per DOF), tet_code (N uint16: 2 bits per Kuhn tet t = 0..5 in itertools.permutations order
 * of the axes: 0 = minus phase, 1 = plus phase, 2 = cut).  Host pointers; each may be NULL. */
xfft_status xfft_get_setup(xfft_ctx* ctx, int* enr_nodes, double* D0, unsigned short* tet_code);

/* Tracing (not in the paper; per-kernel timing for roofline reports).  While enabled, every
 * group of kernel launches is bracketed by CUDA events recorded on the context's stream.
 * xfft_profile_read returns per group k (the XFFT_PROF_* values): the summed device time in ms,
 * the number of kernel launches, and the number of right-hand sides processed (counted on the
 * device by the apply and preconditioner kernels, 0 for the other groups).  Arrays have 16
 * entries (host).  xfft_profile(ctx, 1) enables and resets; xfft_profile(ctx, 0) disables.
 * Reading synchronises the stream.  Errors: ECUDA. */
enum {
  XFFT_PROF_APPLY_UNCUT_F32 = 0, XFFT_PROF_APPLY_CUT_F32 = 1, XFFT_PROF_APPLY_UNCUT_F64 = 2,
  XFFT_PROF_APPLY_CUT_F64 = 3, XFFT_PROF_PREC_F32 = 4, XFFT_PROF_PREC_F64 = 5,
  XFFT_PROF_VECTOR = 6, XFFT_PROF_FINALIZE = 7, XFFT_PROF_SETUP = 8, XFFT_PROF_GRAD = 9,
  XFFT_PROF_POST = 10, XFFT_PROF_APPLY_UNCUT_DW = 11, XFFT_PROF_APPLY_CUT_DW = 12,
  XFFT_PROF_COUNT = 13
};
xfft_status xfft_profile(xfft_ctx* ctx, int enable);
xfft_status xfft_profile_read(xfft_ctx* ctx, double ms[16], long long launches[16],
                              long long units[16]);

/* Allocation-free stiffness apply.  The paper has no counterpart: this is a service for
 * callers that must not allocate device memory once they are running, for example an
 * application that hands all device memory to its own pool allocator at start-up, or one
 * whose other work cannot tolerate the device-wide synchronisation a cudaMalloc/cudaFree
 * may cause.  It computes the same q = A d as xfft_apply in FP64 (scaled enriched DOFs,
 * layout [std (3N) | enr (3 nX)] per RHS), all arrays on the device and caller-owned:
 *   d        n_rhs x 3 (N + nX) doubles (input),
 *   q        n_rhs x 3 (N + nX) doubles (output),
 *   dAd_sig  n_rhs x 7 doubles (output, may be NULL): <d, A d> followed by
 *            int_Y C grad^s d (Mandel 6) per RHS.
 * Its reduction scratch is a fixed array in the library's device memory (about 1.8 MB,
 * present on every GPU that loads the library until the process exits), so it serves at most
 * XFFT_NOALLOC_MAX_RHS right-hand sides and grids whose apply launches at most
 * XFFT_NOALLOC_MAX_PARTS blocks, each writing one partial sum per value: the stencil's
 * ceil(n2 / 15) ceil(n1 / 15) ceil(n0 / 32) blocks plus the cut-tet kernel's blocks (at most
 * a few waves of the GPU's SMs).  With the default tiling 256^3 grids fit and 384^3 grids do
 * not; larger requests return XFFT_EINVAL and touch nothing.  The scratch address of a device
 * is looked up once, by the first xfft_set_microstructure (or xfft_apply_noalloc) on that
 * device; a first lookup attempted while the context's stream is being captured returns
 * XFFT_ESTATE instead.
 * Every call shares the one scratch array: calls that overlap on the GPU (other streams,
 * other threads, other contexts on the same device) race and must be serialised by the
 * caller.  The context must exist with its microstructure set (those calls do allocate). */
#define XFFT_NOALLOC_MAX_RHS 8
#define XFFT_NOALLOC_MAX_PARTS 4096
xfft_status xfft_apply_noalloc(xfft_ctx* ctx, int n_rhs, const double* d, double* q,
                               double* dAd_sig);

/* Launch shapes in use (not in the paper), as picked by the tuner (option autotune) or the
 * defaults: the FP32 cut-tet kernel's grid in blocks and right-hand sides per launch (default 8,
 * i.e. all of a six-case solve), and the FP32 preconditioner's right-hand sides per group of FFT
 * passes (default 64, i.e. all at once; smaller groups keep a group's spectrum in L2 between the
 * passes).  Errors: EINVAL (NULL), ESTATE (no microstructure). */
xfft_status xfft_get_tuning(const xfft_ctx* ctx, int* cut_blocks, int* cut_rhs_per_launch,
                            int* prec_rhs_per_group);

/* Measured FMA throughput of the current GPU in FLOP/s (2 per FMA; not in the paper: the
 * denominator of the ALU roofline reported for the FP64 kernels, precision XFFT_FP64, and for the
 * double-word kernels on the FP32 pipes, XFFT_FP32_REFINED).  A probe kernel of independent FMA
 * chains over 8 blocks per SM, timed with CUDA events on `stream` (a cudaStream_t or NULL);
 * about a millisecond.  Errors: EINVAL, ECUDA. */
xfft_status xfft_fma_rate(int precision, double* flops_per_s, void* stream);

int xfft_num_enriched(const xfft_ctx* ctx);   /* nX, or -1 before set_microstructure */
int xfft_num_cut_tets(const xfft_ctx* ctx);   /* number of cut tetrahedra, or -1 */
const char* xfft_status_string(xfft_status s);
const char* xfft_last_error(void);
void xfft_destroy(xfft_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* XFFT_H */
