/*
 * ch.h -- C ABI of the GB300 solver for the per-time-step saddle-point systems of
 * the ternary Cahn-Hilliard model of Bergermann, Stoll et al., "Preconditioning for
 * a Phase-Field Model with Application to Morphology Evolution in Organic
 * Semiconductors" (arXiv 2204.03575).
 *
 * The model (Section 2) evolves the polymer and NFA volume fractions phi_p, phi_nfa
 * with phi_s = 1 - phi_p - phi_nfa (Eq. (2)).  P1 finite elements and the
 * semi-implicit scheme of Eq. (12) give, per time step and per species, the
 * symmetric saddle-point system of Eq. (14)
 *
 *     [ M     a K ] [phi^{k+1}]   [ M phi^k + tau g_bd ]
 *     [ a K  -c M ] [ mu^{k+1}] = [ -c f^{k}           ],   a = tau*mob, c = a/eps,
 *
 * with the same matrix for both species.  It is solved by flexible GMRES (FP64)
 * right-preconditioned by Algorithm 1 (block-diagonal: AMG for M, and the matching
 * Schur-complement approximation S~ = H M^-1 H with H = a K + sqrt(c) M, Section 3).
 *
 * Conventions (all entry points):
 *  - Every pointer argument named as a vector is a DEVICE pointer owned by the caller,
 *    unless the comment says "host".  Work is enqueued on the caller's CUDA stream
 *    (`stream` is a cudaStream_t; NULL = legacy default stream).  Entry points that
 *    return data to host memory (stats, info) synchronise that stream.
 *  - Opaque handles are created and owned by the library and released with the
 *    matching *_destroy call (NULL is accepted and ignored).  A handle created from
 *    another (system from mesh, preconditioner from system, state from both) borrows
 *    it: the borrowed handle must outlive the borrower.
 *  - Node-major vectors: index i is the node number i + (nx+1)(j + (ny+1)k) of the
 *    grid point (i,j,k).  "N x 4" vectors store, per node, the four unknowns of the
 *    two systems as (phi_p, phi_nfa, mu_p, mu_nfa) -- the first block of both
 *    species, then the second block of both species.
 *  - Errors come back only as return codes; ch_last_error() gives a message for the
 *    calling thread.  No entry point aborts or throws.  A handle stays valid after an
 *    error return unless the code is CH_ERR_CUDA (the CUDA context may be unusable).
 *  - Handles are not thread-safe: one thread at a time per handle.
 */
#ifndef CH_H
#define CH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CH_OK = 0,
  CH_ERR_ARG = 1,            /* invalid argument (NULL handle, bad size or parameter) */
  CH_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  CH_ERR_OOM = 3,            /* device allocation failed */
  CH_ERR_NOT_CONVERGED = 4,  /* FGMRES hit max_iter; the best iterate is still written */
  CH_ERR_BREAKDOWN = 5,      /* Krylov breakdown before convergence */
  CH_ERR_NONFINITE = 6,      /* NaN/Inf met in a residual norm or the right-hand side */
  CH_ERR_STATE = 7,          /* call out of order (e.g. step before the state was set) */
  CH_ERR_INTERNAL = 8        /* a device-side capacity or consistency check failed */
} ch_status;

/* Parameters.  ch_params_default() fills the paper's values (Section 4; Fig. 1 caption). */
typedef struct ch_params {
  int32_t dim;               /* 2 (triangles) or 3 (Kuhn tetrahedra) */
  int32_t nx, ny, nz;        /* cells per axis; nz ignored in 2D.  y is the film height */
  double Lx, Ly, Lz;         /* box [0,Lx]x[0,Ly](x[0,Lz]) */
  double tau;                /* time step (scaled), default 1e-4 */
  double eps;                /* interface parameter eps_p = eps_nfa, default 1e-3 */
  double mobility;           /* M_p = M_nfa, default 1 */
  int32_t bc_mode;           /* 0: zero flux on the whole boundary; 1: Eq. (10) fluxes */
  int32_t evap_sign;         /* +1: evaporation adds polymer/NFA at y=Ly (text); -1: Eq. (10) literally */
  int32_t potential;         /* 0: f of Eq. (15), chain rule through phi_s; 1: without the phi_s term; 2: f' = 0;
                                3: the Flory-Huggins f of Section 2 (logarithmic), also through phi_s, with
                                the chi_* / N_* below; its load is defined by the collapsed 3-point
                                Gauss-Legendre product rule on each simplex (9 points in 2D, 27 in 3D) */
  int32_t precision;         /* 0: FP64 everywhere; 1: FP32 AMG V-cycles inside FP64 FGMRES */
  double k_evap;             /* evaporation rate k, default 5e-3 */
  double g_p, g_nfa;         /* substrate energy g of Eq. (5), default 0.01 */
  double h_p, h_nfa;         /* substrate energy h of Eq. (5), default 0 */
  double rtol;               /* stop when ||b - A x||_2 <= rtol ||b||_2 per species, default 1e-8 */
  int32_t restart;           /* FGMRES restart length m (1..64), default 30 */
  int32_t max_iter;          /* total FGMRES iterations per step, default 300 */
  int32_t cheb_degree;       /* Chebyshev smoothing steps before and after coarse correction on the
                                finest level; 0 (default): 5 */
  int32_t coarse_max;        /* AMG: coarsest level is solved densely at or below this size (<= 4096);
                                0 (default): 512 rows for FP64 V-cycles, 2048 for FP32 */
  double amg_theta;          /* AMG strength threshold, default 0.08 */
  int32_t vcycles_M;         /* V-cycles per application of M~^-1 (Algorithm 1, step 1), default 1 */
  int32_t vcycles_H;         /* V-cycles per application of H~^-1 (Algorithm 1, steps 2 and 4), default 2 */
  int32_t autotune;          /* SpMV lanes per row: 0 = fixed rule, 1 = timed at set-up (cached per process), default 1 */
  double cheb_lower;         /* Chebyshev interval [cheb_lower, 1] x 1.1 lambda_max(D^-1 A), default 0.3 */
  int32_t graphs;            /* 1 (default): FGMRES's convergence loop runs on the device -- a plain
                                step (ch_step) is one CUDA graph launch (conditional while / switch
                                nodes: Arnoldi steps and restart cycles chosen by the flags of every
                                run and species) and one host synchronisation, a step with a guess
                                launches its solve as one graph; 0: the host drives the loop with
                                direct launches, reading the flags after every Arnoldi step.  Both
                                give bitwise the same steps.  Per-launch event timing
                                (ch_profile_enable) and MINRES (krylov = 1) use the host loop */
  int32_t cheb_degree_coarse; /* Chebyshev steps on the levels below the finest; 0 (default): 2 (at
                                most cheb_degree) */
  int32_t cheb_degree_M;     /* finest-level Chebyshev degree of M's hierarchy (Algorithm 1, step 1);
                                0 (default): min(3, cheb_degree) -- M is close to its diagonal */
  int32_t krylov;            /* 0 (default): flexible GMRES(restart); 1: preconditioned MINRES, the
                                paper's method (Algorithm 1 with fixed V-cycles is symmetric positive
                                definite; work vectors use the basis storage, so restart >= 5) */
  int32_t pattern;           /* substrate preference on y = 0 (Eq. (5), Section 4): 0 (default) p_p =
                                p_nfa = 1; 1: p_p = 1 on the 1st, 3rd and 5th sixth of [0, Lx] (each
                                run's own Lx), p_nfa = 1 on the others.  Integrated exactly: facets
                                are cut where they cross a breakpoint */
  int32_t precond_M;         /* Algorithm 1, step 1 (M~^-1 v_1): 0 (default) AMG V-cycles of M's
                                hierarchy; 1: the Chebyshev semi-iteration Section 3 names instead --
                                cheb_M_steps steps on D^-1 M from a zero guess over Wathen's bounds of
                                its eigenvalues, [1/2, 2] (triangles) or [1/2, 5/2] (tetrahedra) */
  int32_t cheb_M_steps;      /* steps of that semi-iteration (1..16); 0 (default): 5 */
  double chi_pn, chi_ps, chi_ns; /* Flory-Huggins interaction parameters (potential = 3); default
                                1, 0.3, 0.3 (Section 4) */
  double N_p, N_nfa, N_s;    /* degrees of polymerisation (potential = 3); default 20, 20, 1 (Section 4) */
  double fh_delta;           /* potential = 3: each logarithm is taken at max(phi, fh_delta) (a
                                positivity guard; concentrations may dip below 0), default 1e-10 */
  int32_t pdl;               /* 1 (default): the V-cycle and Krylov kernels are launched as programmatic
                                dependents -- each kernel's blocks are scheduled while its predecessor
                                drains and wait on the device for its results (griddepcontrol), which
                                hides the launch gap between the many short kernels of a step; 0: plain
                                stream-ordered launches.  Same arithmetic, bitwise the same results */
  int32_t gs_reorth;         /* FGMRES's Gram-Schmidt: 0 (default) classical Gram-Schmidt twice at every
                                Arnoldi step; 1 selective reorthogonalisation -- one projection, and the
                                second only for a species whose vector lost more than half its squared
                                norm to it (||w'|| < ||w|| / sqrt(2)).  On the 512 x 512 workload the
                                second pass is still needed on ~72 % of the steps, which makes 1 slightly
                                slower than 0; ch_step_stats.reorth counts the second passes */
} ch_params;

/* Per-step statistics (host struct). */
typedef struct ch_step_stats {
  int32_t iters[2];          /* FGMRES iterations (polymer, NFA) */
  int32_t restarts;          /* FGMRES: restart cycles used; MINRES: true-residual checks after the first */
  int32_t status;            /* ch_status of this step */
  double relres[2];          /* true final ||b - A x|| / ||b|| per species, FP64 */
  double mass[2];            /* int phi_h = 1^T M phi^{k+1} per species */
  double ms;                 /* wall time of the step (ms, CUDA events) */
  int32_t warm[2];           /* ch_step_guess: 1 if the caller's guess was used as initial iterate */
  int32_t reorth[2];         /* FGMRES: Arnoldi steps that took the second Gram-Schmidt pass (all of them
                                with gs_reorth = 0) */
} ch_step_stats;

typedef struct ch_mesh_s ch_mesh_t;
typedef struct ch_system_s ch_system_t;
typedef struct ch_precond_s ch_precond_t;
typedef struct ch_state_s ch_state_t;
typedef struct ch_ws_s ch_ws_t;

const char* ch_status_str(ch_status s);
const char* ch_last_error(void);
void ch_params_default(ch_params* p);

/* ---------------------------------------------------------------- mesh (Section 4)
 * Uniform simplicial mesh of the box: 2 triangles per cell (diagonal from (i,j) to
 * (i+1,j+1)) or the 6 Kuhn tetrahedra per hexahedron.  Gamma_b = {y = 0} (substrate),
 * Gamma_t = {y = Ly} (evaporation).  Built on the device. */
ch_status ch_mesh(const ch_params* p, void* stream, ch_mesh_t** out);
/* Batched runs: the disjoint union of nruns box meshes (runs[r] gives run r's dim, nx, ny, nz,
 * Lx, Ly, Lz; all runs share dim).  Run r owns the node range [off[r], off[r+1]) (ch_mesh_runs),
 * its own boundaries Gamma_b, Gamma_t and its own initial state; the model parameters come from
 * the params given to ch_assemble (whose cell counts are then ignored) and are the same for every run.  Every later call (assembly,
 * AMG set-up, V-cycles, FGMRES steps) then advances all runs together, with the Krylov scalars
 * and convergence tests kept per run and species. */
ch_status ch_mesh_batch(int32_t nruns, const ch_params* runs, void* stream, ch_mesh_t** out);
/* host outputs: number of runs and (if run_offsets != NULL) nruns+1 node offsets */
ch_status ch_mesh_runs(const ch_mesh_t* m, int32_t* nruns, int32_t* run_offsets);
/* host outputs, any may be NULL */
ch_status ch_mesh_info(const ch_mesh_t* m, int64_t* n_nodes, int64_t* n_elems,
                       int64_t* n_bottom, int64_t* n_top);
/* copies to caller device buffers: coords N x dim (fp64), elems E x (dim+1), facets F x dim (int32); any may be NULL */
ch_status ch_mesh_copy(const ch_mesh_t* m, double* coords, int32_t* elems, int32_t* bottom,
                       int32_t* top, void* stream);
void ch_mesh_destroy(ch_mesh_t* m);

/* ---------------------------------------------------------------- assembly (Section 3)
 * P1 mass M and stiffness K ("standard ... with appropriate constants", below Eq. (12)) in
 * one shared CSR pattern (sorted column indices), and H = a K + sqrt(c) M, on the device.
 * The system also holds a scratch for the explicit loads (one entry per element vertex):
 * calls that use one system -- ch_loads, ch_rhs and the steps of states built on it -- must
 * not overlap on the GPU. */
ch_status ch_assemble(const ch_mesh_t* m, const ch_params* p, void* stream, ch_system_t** out);
ch_status ch_system_info(const ch_system_t* s, int64_t* n, int64_t* nnz);   /* host outputs */
/* copies to caller device buffers (rowptr N+1, col nnz int32; values nnz fp64); any may be NULL */
ch_status ch_system_copy(const ch_system_t* s, int32_t* rowptr, int32_t* col, double* valM,
                         double* valK, double* valH, void* stream);
void ch_system_destroy(ch_system_t* s);

/* Explicit loads of one step (Eq. (12), right-hand sides): F_s[i] = int f_s'(phi_h) lambda_i,
 * exact for the polynomial potential Eq. (15), and the boundary loads g_s of the flux
 * conditions Eq. (10), with Section 4's substrate pattern when the system's pattern = 1 (its
 * per-facet weights are formed once by ch_assemble).  Inputs N fp64; outputs N fp64 (any output
 * may be NULL). */
ch_status ch_loads(const ch_system_t* s, const double* phi_p, const double* phi_nfa,
                   double* F_p, double* F_nfa, double* g_p, double* g_nfa, void* stream);
/* Right-hand sides of Eq. (14) for both species, b (N x 4) = (M phi_p + tau g_p, M phi_nfa + tau g_nfa,
 * -c F_p, -c F_nfa) per node. */
ch_status ch_rhs(const ch_system_t* s, const double* phi_p, const double* phi_nfa, double* b,
                 void* stream);
/* y = A x for both species at once (Eq. (14)); x, y are N x 4 fp64, must not alias. */
ch_status ch_apply_A(const ch_system_t* s, const double* x, double* y, void* stream);

/* ---------------------------------------------------------------- preconditioner (Algorithm 1)
 * Builds, on the device, smoothed-aggregation AMG hierarchies for M and H (strength of
 * connection, MIS(2) aggregation, Jacobi-smoothed prolongator, Galerkin coarse operators,
 * dense inverse of the coarsest level), Chebyshev smoother bounds per level and, when
 * precision = 1, FP32 copies of every level.  On a uniform mesh (one run or a batch of them) the
 * finest level is also stored by lattice diagonals.  The preconditioner owns a non-blocking
 * CUDA stream and two events on the current device: ch_precond_apply runs step 1 of Algorithm 1
 * on that stream, forked from and joined back into the caller's stream. */
ch_status ch_precond_setup(const ch_system_t* s, void* stream, ch_precond_t** out);
/* which: 0 = M hierarchy, 1 = H hierarchy.  Host outputs; level-wise sizes for level < nlevels. */
ch_status ch_precond_info(const ch_precond_t* pc, int32_t which, int32_t level, int32_t* nlevels,
                          int64_t* rows, int64_t* nnz);
/* Level `level` of hierarchy `which` as the V-cycle uses it, for checking the V-cycle against an
 * independent implementation.  Host outputs (any may be NULL): rows and nnz of A_l, nnz of P_l,
 * the Chebyshev interval [lo, hi] of D^-1 A_l and the level's smoothing degree (the coarsest
 * level has nnz_P = 0, lo = hi = 0 and degree 0: it is solved by its dense inverse).  Device
 * outputs (any may be NULL; caller-owned, sized from a first call's host outputs): the FP64
 * set-up matrices A_l (rowptr rows + 1, col nnz, val nnz) and P_l (rowptr rows + 1, col and val
 * nnz_P; columns index level l + 1), copied on `stream`.  Precision 1 smooths with FP32 copies of
 * these matrices. */
ch_status ch_precond_level(const ch_precond_t* pc, int32_t which, int32_t level, int64_t* rows,
                           int64_t* nnz, int64_t* nnz_P, double* lo, double* hi, int32_t* degree,
                           int32_t* A_rowptr, int32_t* A_col, double* A_val, int32_t* P_rowptr,
                           int32_t* P_col, double* P_val, void* stream);
/* Lanes per row chosen for the level's A (smoothing, residual), R (restriction) and P
 * (prolongation) SpMVs (host outputs; R and P are 0 on the coarsest level). */
ch_status ch_precond_tiles(const ch_precond_t* pc, int32_t which, int32_t level, int32_t* tpr_A,
                           int32_t* tpr_R, int32_t* tpr_P);
/* Algorithm 1 on both species: w_1 ~ M^-1 v_1 and w_2 ~ H^-1 M H^-1 v_2 (AMG V-cycles); the
 * w_1 branch runs concurrently on the preconditioner's own stream and is joined back into
 * `stream` before the call's work ends (stream order for the caller is unchanged).
 * v, w: N x 4 fp64, must not alias. */
ch_status ch_precond_apply(ch_precond_t* pc, const double* v, double* w, void* stream);
/* The V-cycles' finest-level smoother on its own (Section 3's AMG relaxation): `passes` passes of
 * `degree` Chebyshev steps on D^-1 A x = D^-1 b over the V-cycle's interval of D^-1 A (as
 * ch_precond_level exports it), each pass continuing from the previous one's x, as the V-cycle's
 * post-smoothing does, in the hierarchy's working precision; A = M (which = 0) or H (which = 1).
 * b, x: N x 2 fp64 device arrays, 16-byte aligned, not aliased; x is the initial iterate on entry
 * and the result on exit.  The steps are the solver's own fine-level kernels, launched as it
 * launches them (a caller may capture the call in a CUDA graph).  CH_ERR_ARG for degree outside
 * [1, 16], passes < 1, which outside {0, 1}, NULL, aliased or misaligned arrays, and for a
 * hierarchy of one level (solved directly by the V-cycle: it has no smoother). */
ch_status ch_smooth(ch_precond_t* pc, int32_t which, int32_t degree, int32_t passes, const double* b, double* x,
                    void* stream);
/* vcycles V-cycles (zero initial guess) on M (which = 0) or H (which = 1) for two right-hand
 * sides stored N x 2 (fp64): x ~ A^-1 b.  b, x must not alias. */
ch_status ch_vcycle(ch_precond_t* pc, int32_t which, int32_t vcycles, const double* b, double* x,
                    void* stream);
/* Algorithm 1's step 1 alone (Section 3: "approximately solve M w_1 = v_1") for two right-hand
 * sides stored N x 2 (fp64): x = M~^-1 b, by the vcycles_M V-cycles of M's hierarchy
 * (precond_M = 0) or the Chebyshev semi-iteration (precond_M = 1: cheb_M_steps steps on D^-1 M
 * from zero over Wathen's bounds [1/2, 2] for triangles, [1/2, 5/2] for tetrahedra), in the
 * preconditioner's working precision.  b, x must not alias and must be 16-byte aligned. */
ch_status ch_mass_solve(ch_precond_t* pc, const double* b, double* x, void* stream);
void ch_precond_destroy(ch_precond_t* pc);

/* Allocation-free V-cycles.  The paper has no counterpart to this call: it exists for callers
 * that must not allocate device memory while they run -- for example code recorded into a CUDA
 * graph by stream capture (where cudaMalloc is not allowed), applications whose device memory is
 * owned by a framework's caching allocator with a fixed budget, or latency-critical loops that
 * cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * It computes exactly what ch_vcycle computes (the same arithmetic in the same order; ch_vcycle
 * merges some of these launches, which leaves the results unchanged; strides 2), but every
 * per-level work vector lives in one static device array of 8 MiB that each GPU loading the
 * library reserves until the process exits.  The only other device memory it touches is the
 * caller's b and x and the hierarchy built earlier by ch_precond_setup (read only).
 *  - Limit: 5 work vectors x 2 right-hand sides per level must fit in 8 MiB, i.e. the level
 *    sizes summed over the hierarchy may not exceed about 104,000 rows with precision 0 (FP64)
 *    or 209,000 with precision 1 (FP32); larger hierarchies return CH_ERR_ARG with a message.
 *  - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream capture on the device.
 *  - All calls share the one array and keep the last call's contents (nothing in it needs to
 *    start at zero).  Calls that overlap on the GPU -- different streams or threads at the same
 *    time -- race and give wrong results: issue them in order on one stream. */
ch_status ch_vcycle_noalloc(ch_precond_t* pc, int32_t which, int32_t vcycles, const double* b,
                            double* x, void* stream);

/* ---------------------------------------------------------------- time stepping (Eq. (12)-(14))
 * A state holds (phi_p, phi_nfa, mu_p, mu_nfa) on the device plus all FGMRES work space, so
 * ch_step allocates no work vectors; with graphs on, the first step of each kind captures and
 * instantiates the state's CUDA graph (kept until ch_state_destroy). */
ch_status ch_state_create(const ch_system_t* s, ch_precond_t* pc, void* stream, ch_state_t** out);
/* Set the state from caller device buffers (N fp64 each); mu_* may be NULL (zero). */
ch_status ch_state_set(ch_state_t* st, const double* phi_p, const double* phi_nfa,
                       const double* mu_p, const double* mu_nfa, void* stream);
/* Seeded initial state (Section 4): phi = base + noise (2u - 1), u from SplitMix64 on the counter
 * seed ^ (field << 40) ^ node, field 0 = polymer, 1 = NFA; mu = 0.  For a batch, every run uses
 * these bases and run r the stream seed + r over its local node index. */
ch_status ch_state_init_seeded(ch_state_t* st, double phi_p0, double phi_nfa0, double noise,
                               uint64_t seed, void* stream);
/* Seeded initial state of a batch: run r gets bases phi_p0[r], phi_nfa0[r] (host arrays of nruns)
 * and the generator stream seed + r over its local node index. */
ch_status ch_state_init_seeded_batch(ch_state_t* st, const double* phi_p0, const double* phi_nfa0,
                                     double noise, uint64_t seed, void* stream);
/* Statistics of run `run` for the last ch_step (host output); ch_step itself reports run 0. */
ch_status ch_state_run_stats(const ch_state_t* st, int32_t run, ch_step_stats* out);
/* Copy fields to caller device buffers (N fp64 each); any may be NULL.  phi_s = 1 - phi_p - phi_nfa. */
ch_status ch_state_get(const ch_state_t* st, double* phi_p, double* phi_nfa, double* phi_s,
                       double* mu_p, double* mu_nfa, void* stream);
/* Checkpoint / resume.  ch_state_save writes the state (phi_p, phi_nfa, mu_p, mu_nfa of every
 * node, FP64) to a file at `path`: an 8-byte tag "CHSTATE1", the node count and the run count
 * (int64 each), then the N x 4 values node by node, in the host's byte order.  ch_state_load reads
 * such a file into a state built on a system of the same node and run counts (CH_ERR_ARG
 * otherwise, or when the file is missing, truncated or not a state file); the loaded state then
 * steps exactly as the saved one would (the learned-step history starts afresh).  Both block the
 * stream; save needs a set state (CH_ERR_STATE). */
ch_status ch_state_save(const ch_state_t* st, const char* path, void* stream);
ch_status ch_state_load(ch_state_t* st, const char* path, void* stream);
/* One time step: loads, right-hand sides, FGMRES + Algorithm 1 for both species with the
 * previous step as initial guess, state update.  stats (host) may be NULL.  On
 * CH_ERR_NOT_CONVERGED the best iterate is stored in the state. */
ch_status ch_step(ch_state_t* st, void* stream, ch_step_stats* stats);
/* One time step as ch_step, but with a candidate initial iterate `guess` (N x 4 fp64 device, the
 * state layout): for each run and species FGMRES starts from the guess if its true FP64 residual
 * ||b - A guess|| is smaller than that of the previous step's state, else from the previous state
 * (stats->warm records which).  The right-hand side is always built from the previous state. */
ch_status ch_step_guess(ch_state_t* st, const double* guess, void* stream, ch_step_stats* stats);
/* nsteps steps; per_step (host, nsteps entries) may be NULL.  Stops at the first error. */
ch_status ch_run(ch_state_t* st, int32_t nsteps, void* stream, ch_step_stats* per_step);
void ch_state_destroy(ch_state_t* st);

/* ---------------------------------------------------------------- learned warm start
 * A 3-layer convolutional network on the nodal image of a 2D structured mesh (H = ny+1 rows,
 * W = nx+1 columns, node i + W j = pixel (j, i)) that predicts the next step's state from the last
 * three, used as the guess of ch_step_guess.  The paper has no counterpart (this extension is one
 * of the build's own).  The prediction is a learned second-order extrapolation:
 *   pred = s + d + theta * D,  d = s - q,  D = s - 2 q + q2,  theta = y * out_scale,
 * with s = s_k, q = s_{k-1}, q2 = s_{k-2} (phi_p, phi_nfa, mu_p, mu_nfa) and y the network's output:
 * the zero network is linear extrapolation, theta = 1 quadratic extrapolation, and the network
 * only scales the second difference pixel by pixel.
 * Layers: 3x3 convolutions with zero padding, 12 -> 32 (ReLU) -> 32 (ReLU) -> 4; BF16 weights and
 * activations, FP32 accumulation on the tensor cores, FP32 master weights with Adam.
 * Input channels, with r1[c], r2[c] the RMS over the image of channel c of d and D:
 * (s - mean[0:4]) * inv_std[0:4], (d / r1 - mean[4:8]) * inv_std[4:8], D / r2.
 * Parameters (ch_ws_nparams() floats, host arrays), in order: w1[9][16][32] (tap = 3 ky + kx,
 * input channel padded to 16, output channel), b1[32], w2[9][32][32], b2[32], w3[9][32][8]
 * (output channel padded to 8), b3[8]; padded entries are ignored. */
int32_t ch_ws_nparams(void);
ch_status ch_ws_create(int32_t H, int32_t W, int32_t max_batch, ch_ws_t** out);
void ch_ws_destroy(ch_ws_t* w);
/* The tensor-core path of the network's convolutions (host setting, applies to later calls):
 * 0: mma.sync, each warp 16 pixels x the output channels with fragments gathered from the image;
 * 1 (default): tcgen05 -- persistent blocks of 128 threads stage the weights once, then per tile
 * (a segment of <= 128 pixels of one image row) the three input row bands its taps read; one
 * thread issues the MMAs, whose A operands are descriptors into the bands, into a tensor-memory
 * accumulator, and the warps read it back for the epilogue.  Measured on a 257 x 257 image:
 * 16.0 against 22.6 us per convolution (prediction), 97 against 48 TFLOP/s (training batch of 8).  Both compute the same convolutions (FP32 accumulation, in
 * a different order).  A tcgen05 block whose wait for its MMAs runs out records it; the next
 * training call or learned step that synchronises returns CH_ERR_INTERNAL.  CH_ERR_ARG for an
 * engine other than 0 or 1. */
ch_status ch_ws_set_engine(ch_ws_t* w, int32_t engine);
/* Test of the failure path of the tcgen05 convolutions (host setting): with on = 1 their blocks
 * issue and commit no MMA, so each block's bounded wait on its mbarrier runs out (after a short
 * limit), the block records the timeout, frees its tensor memory and writes nothing; the next
 * training call or learned step that synchronises returns CH_ERR_INTERNAL and clears the record.
 * The device context stays usable: with on = 0 the network computes as before. */
ch_status ch_ws_inject_mma_timeout(ch_ws_t* w, int32_t on);
ch_status ch_ws_set_params(ch_ws_t* w, const float* params, void* stream);     /* host; resets Adam */
/* host outputs, either may be NULL; grads are those of the last ch_ws_train_step */
ch_status ch_ws_get_params(const ch_ws_t* w, float* params, float* grads, void* stream);
/* host: mean[8], inv_std[8], out_scale[4] */
ch_status ch_ws_set_norm(ch_ws_t* w, const float* norm20, void* stream);
/* Normalisation of a training set, computed on the device and set on the network (as
 * ch_ws_set_norm): the states x = s_k of nsamples samples, a device array of nsamples x N x 4
 * (fp64, or fp32 when fp32 = 1).  mean[0:4] and inv_std[0:4] are the mean and 1 / standard
 * deviation of the four fields over the set (n - 1 divisor, floor 1e-30); mean[4:8] = 0,
 * inv_std[4:8] = 1 (the change is already in units of its RMS); out_scale = 1 (theta = y).  Sums in
 * a fixed order (reproducible).  norm20 (host, 20 doubles) receives (mean[8], inv_std[8],
 * out_scale[4]).  Allocates and frees its own small scratch. */
ch_status ch_ws_fit_norm(ch_ws_t* w, const void* x, int32_t nsamples, int32_t fp32, double* norm20, void* stream);
/* pred (N x 4 fp64 device): the prediction of the next state from the state and its two
 * predecessors (N x 4 fp64 device each); pred must not alias them */
ch_status ch_ws_predict(ch_ws_t* w, const double* state, const double* prev, const double* prev2, double* pred,
                        void* stream);
/* One training step on B <= max_batch samples (device fp32, B x N x 4 each): states x = s_k, their
 * predecessors q = s_{k-1}, q2 = s_{k-2} and successors n = s_{k+1}.  With E = (theta D - e) / r1
 * (the prediction's error in units of the change's RMS; e = n - 2 x + q) and G the graph Laplacian
 * of the pixel grid ((G E)_p = sum over the 4-neighbours q of p in the image of E_q - E_p), the
 * loss is (sum E^2 + lap * sum (G E)^2) / (4 B N): lap >= 0 weighs rough errors, which dominate the
 * step's residual through its stiffness rows.  Computes the gradients (ch_ws_get_params); lr > 0
 * also takes an Adam step.  *loss (host) may be NULL.  CH_ERR_ARG: B outside [1, max_batch],
 * lap < 0 or not finite. */
ch_status ch_ws_train_step(ch_ws_t* w, const float* x, const float* q, const float* q2, const float* n, int32_t B,
                           float lap, float lr, float* loss, void* stream);

/* One training step against the residual of Eq. (14) (the quantity FGMRES's stopping test
 * measures), on B <= max_batch samples of consecutive states (device fp64, B x N x 4 each:
 * x = s_k, q = s_{k-1}, q2 = s_{k-2}) of the 2D single-run mesh of `sys` (N = H W).  Per sample and
 * species, with b the right-hand side of the step from s_k and c = theta D the network's change of
 * the linear extrapolation, r_ex = b - A (2 s_k - s_{k-1}) and r = r_ex - A c, measured in the norm
 * of the preconditioner `pc` (<r, P^-1 r>, Algorithm 1 built on `sys`) or, if pc is NULL, the
 * Euclidean norm.  The loss is the mean over samples and species of ln(|r|^2 / |r_ex|^2): 0 for
 * linear extrapolation, negative where the prediction beats it; Krylov iteration counts grow with
 * the logarithm of the initial residual, so each sample's relative gain counts alike.  Computes
 * the gradients; lr > 0 also
 * takes an Adam step.  *loss (host) may be NULL.  CH_ERR_ARG: B outside [1, max_batch], a system
 * that is not a single-run 2D mesh of H x W nodes, or a preconditioner of another system. */
ch_status ch_ws_train_residual(ch_ws_t* w, const ch_system_t* sys, ch_precond_t* pc, const double* x,
                               const double* q, const double* q2, int32_t B, float lr, float* loss, void* stream);

/* One time step whose candidate guess is the network's prediction from the state and its two
 * predecessors, which the state keeps on the device across consecutive ch_step_learned calls; the
 * choice between guess and previous state is that of ch_step_guess.  Until three steps have been
 * taken since the state was set (the first sets up the chemical potentials), and until two learned
 * steps in a row have recorded the history, the step starts from the previous state.
 * stats->ms includes the prediction.  CH_ERR_ARG: a network sized for another mesh, or a state
 * of several runs. */
ch_status ch_step_learned(ch_state_t* st, ch_ws_t* w, void* stream, ch_step_stats* stats);

/* ---------------------------------------------------------------- morphology projection (Section 5)
 * Section 5 passes a simulated morphology to a device model on a finite-difference grid: the field
 * is thresholded into a binary image, and each grid point is classified by the parity of the
 * number of object faces crossed by a ray from the point.  Here the image has one pixel per node of
 * a 2D nx x ny mesh of [0,Lx]x[0,Ly] (node i + (nx+1) j; pixel (i, j) is the half-open cell
 * [(i-1/2)hx, (i+1/2)hx) x [(j-1/2)hy, (j+1/2)hy) clipped to the box), set where phi_p > phi_nfa
 * (use_threshold = 0) or phi_p > threshold (use_threshold = 1; phi_nfa may then be NULL); the
 * grid points are the centres of a uniform gx x gy cell grid of the box (point k + gx l at
 * ((k+1/2) Lx/gx, (l+1/2) Ly/gy)); each point's ray runs upward and crosses the horizontal pixel
 * faces between vertically adjacent pixels of different value and the top edge above a set
 * top-row pixel.  Device inputs: phi_p, phi_nfa ((nx+1)(ny+1) fp64, e.g. from ch_state_get).
 * Device outputs (gx gy each, any may be NULL): polymer (1 inside the polymer phase, else 0), and
 * Section 5's mobilities: mu_e = 1e-10, mu_h = 0.1 m^2/(V s) in the polymer phase, the other way
 * round elsewhere.  CH_ERR_ARG for sizes < 1, a non-positive box, a NULL field. */
ch_status ch_morphology_project(const double* phi_p, const double* phi_nfa, int32_t nx, int32_t ny, double Lx,
                                double Ly, int32_t use_threshold, double threshold, int32_t gx, int32_t gy,
                                uint8_t* polymer, double* mu_e, double* mu_h, void* stream);

/* ---------------------------------------------------------------- launch accounting
 * Every kernel launch of the library is counted per kernel and working precision, with the
 * algorithmic bytes (each operand once) and FMAs of that launch.  With timing on, CUDA events
 * are recorded around each launch on its stream and the elapsed times summed (adds a small
 * host overhead per launch).  Process-wide; thread-safe. */
typedef struct ch_prof_entry {
  char name[40];             /* kernel name and precision, e.g. "cheb_step_f32" */
  int64_t launches;
  double ms;                 /* summed event time (0 unless timing was on) */
  double bytes;              /* summed algorithmic bytes */
  double fmas;               /* summed fused multiply-adds */
} ch_prof_entry;
ch_status ch_profile_enable(int32_t on);
/* Waits for pending events, then copies up to cap entries (host array) and sets *n to the
 * number of kernels seen; out may be NULL to query n.  reset != 0 clears the counters. */
ch_status ch_profile_read(ch_prof_entry* out, int32_t cap, int32_t* n, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* CH_H */
