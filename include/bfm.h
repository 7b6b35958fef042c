/*
 * bfm.h -- C ABI of the GB300 back-and-forth optimal-transport library.
 *
 * The back-and-forth method (BFM) of Jacobs & Leger, "A fast approach to
 * optimal transport: the back-and-forth method" (arXiv 1905.12154) solves the
 * quadratic-cost Kantorovich dual problem (Section 3, eq. (dual)) between two
 * densities mu and nu on a regular grid over [0,1]^d (Section 4.3), by
 * alternating H1-dot gradient ascent steps on J (phi-space) and I (psi-space)
 * with c-transforms in between (Algorithm 1) and the step-size rule of
 * Section 4.2.
 *
 * Conventions shared by every entry point
 *   grid      cell-centred, n[a] cells on axis a (2 <= n[a]), ndim in {2, 3};
 *             cell i of axis a has centre (i + 1/2) / n[a].
 *   layout    a field is N = n[0]*n[1]*n[2] contiguous elements with axis 0
 *             fastest: index = (k*n[1] + j)*n[0] + i.  A map is ndim fields
 *             stored one after the other (component a at offset a*N).
 *   precision BFM_FP32: fields are float, all reductions, the dual value,
 *             the residual and the step-size test are FP64.  BFM_FP64: fields
 *             are double.
 *   densities non-negative density values; a density of unit mass has
 *             mean 1 over the grid.  The transport cost C (Section 4.3) is
 *             half the squared Wasserstein distance: W2^2 = 2 C.
 *   memory    every field pointer is DEVICE memory owned by the caller unless
 *             the argument says "host".  The library never allocates device
 *             memory: scratch comes from a caller-provided device workspace
 *             of at least the size the matching *_workspace_bytes() returns
 *             (256-byte aligned).  Work is stream-ordered on `stream`
 *             (a cudaStream_t passed as void*, NULL = legacy default stream);
 *             functions that return results to host memory synchronise that
 *             stream before returning.
 *   errors    every call returns a bfm_status; on BFM_ERR_INVALID_ARG /
 *             BFM_ERR_UNSUPPORTED nothing was launched; on BFM_ERR_CUDA the
 *             CUDA error string is available from bfm_last_error().
 *   sizes     FFT-based steps need every n[a] of the form 2^p 3^q with
 *             2 <= n[a] <= 8192 (4096 in FP64); other sizes give
 *             BFM_ERR_UNSUPPORTED.  The c-transform accepts any 2 <= n[a] <= 8192.
 */
#ifndef BFM_H
#define BFM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFM_OK = 0,
    BFM_NOT_CONVERGED = 1,      /* max_iter reached; results are filled */
    BFM_ERR_INVALID_ARG = -1,   /* bad pointer, size, density (negative, NaN, zero mass) */
    BFM_ERR_NONFINITE = -2,     /* a reduction produced Inf/NaN during the solve */
    BFM_ERR_CUDA = -3,          /* a CUDA call failed; see bfm_last_error() */
    BFM_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up */
    BFM_ERR_UNSUPPORTED = -5,   /* grid size / cost / precision not supported */
    BFM_ERR_WORKSPACE = -6      /* workspace NULL, misaligned or too small */
} bfm_status;

typedef enum { BFM_FP32 = 0, BFM_FP64 = 1 } bfm_precision;

/* Costs: the quadratic cost |x-y|^2/2 of Section 4.3, and the separable power
 * costs of Section 5 (eq. p_costs), c(x,y) = sum_a |y_a - x_a|^{p_a} / p_a with
 * 1 < p_a <= 16 given in bfm_options.cost_p (axis 0 first). */
typedef enum { BFM_COST_QUADRATIC = 0, BFM_COST_POWER = 1 } bfm_cost;

typedef struct {
    int ndim;       /* 2 or 3 */
    int n[3];       /* cells per axis; n[2] ignored when ndim == 2 */
} bfm_grid;

/* The iteration.  BFM_BACK_AND_FORTH is Algorithm 1 (the default).
 * BFM_GRADIENT_ASCENT is the plain H1-dot gradient ascent on J that Section 5
 * compares it with (Tables 5 and 6): phi_{n+1/2} = phi_n + sigma grad J(phi_n),
 * phi_{n+1} = (phi_{n+1/2})^{cc}; two c-transforms and one Poisson solve per
 * iteration (phi_{n+1}^c = (phi_{n+1/2})^c is kept for the next gradient), the
 * step rule of Section 4.2 applied to J(phi_{n+1/2}) - J(phi_n), and the
 * residual, logs and outputs of Algorithm 1 (dual[n] = J(phi_n)). */
typedef enum { BFM_BACK_AND_FORTH = 0, BFM_GRADIENT_ASCENT = 1 } bfm_method;

/* Step-size rule of Section 4.2 and loop control.  bfm_default_options()
 * fills the paper's values: beta1 = 1/4, beta2 = 3/4, alpha1 = 5/4,
 * alpha2 = 4/5, sigma0 <= 0 meaning 8 min(1/|mu|_inf, 1/|nu|_inf),
 * sigma_min = 0.01, method = BFM_BACK_AND_FORTH and cost_p = {0, 0, 0}. */
typedef struct {
    double beta1, beta2, alpha1, alpha2;
    double sigma0;
    double sigma_min;
    int poll_every;          /* host reads the device convergence flag every k iterations (default 4) */
    int warm_start;          /* nonzero: result->phi holds the initial phi on entry (else phi_0 = 0) */
    int method;              /* bfm_method */
    double cost_p[3];        /* BFM_COST_POWER: the exponents p_a (axis 0 first); all 0 for
                                the quadratic cost */
} bfm_options;

typedef struct {
    /* outputs the caller provides (DEVICE, precision of the call):
     *   phi  N elements    the final phi_n (nu side potential)
     *   psi  N elements    phi_n^c (mu side potential)
     *   map  ndim*N        T(x) = x - grad psi(x) in [0,1] coordinates (may be NULL) */
    void *phi, *psi, *map;
    /* per-iteration logs the caller provides (HOST, length max_iter+1, may be NULL):
     *   dual[n]  = J(phi_n)  (eq. (defJ)), resid[n] = relative H^-1 residual
     *   ||nu - T_phi_n # mu|| / ||nu - 1||, sigma[n] = step size at iteration n */
    double *dual, *resid, *sigma;
    /* filled by the call */
    double w2sq;             /* 2 J(phi_final) */
    double mass_mu, mass_nu; /* input masses (mean * 1): the solve uses mu/mass_mu, nu/mass_nu */
    double max_mu, max_nu;   /* |mu|_inf, |nu|_inf after normalisation (max density ratio) */
    double sigma_final;
    int iters;               /* completed back-and-forth iterations */
    int converged;
} bfm_result;

/* ----------------------------------------------------------------------- */

/* Fills `opt` with the paper's step-rule constants (Section 4.2). */
void bfm_default_options(bfm_options *opt);

/* Human-readable name of a status code (static string). */
const char *bfm_status_string(bfm_status s);

/* Text of the last CUDA error seen by this thread's calls (static buffer). */
const char *bfm_last_error(void);

/* Device workspace bytes bfm_solve needs for this grid, precision and
 * max_iter (log arrays are max_iter+1 long).  0 for an invalid grid. */
size_t bfm_workspace_bytes(const bfm_grid *grid, bfm_precision prec, int max_iter);

/*
 * Algorithm 1 (the back-and-forth method) with the step-size rule of
 * Section 4.2 (or opt->method's gradient ascent).  cost: BFM_COST_QUADRATIC
 * (opt->cost_p all 0), or BFM_COST_POWER with the exponents in opt->cost_p;
 * for a power cost T(x) = x - (grad h)^{-1}(grad psi~) and the c-transforms
 * are those of bfm_ctransform_power.  Per iteration n (4 c-transforms and 2
 * Poisson solves, as counted in Section 4.3):
 *   phi-half: psi~ = phi^c; J(phi) (eq. (defJ)); rho = T_phi # mu with
 *             T(x) = x - grad psi~ (Lemma 2.2(ii), Lemma 3.1); g =
 *             (-Delta)^{-1}(nu - rho) (eq. (gradients_J_I)); residual r_n;
 *             stop if r_n < tol; phi += sigma g; psi = phi^c; step rule.
 *   psi-half: the same with mu <-> nu, phi <-> psi, J -> I (eq. (defI)).
 * mu, nu: DEVICE, N elements each, non-negative, finite, positive mass (not
 * modified).  tol: stop when the residual drops below it (0 = run max_iter).
 * out->phi/psi/map: DEVICE outputs (see bfm_result).  opt may be NULL.
 * Returns BFM_OK (converged), BFM_NOT_CONVERGED (max_iter reached), or an
 * error.  Synchronises `stream` before returning.
 */
bfm_status bfm_solve(const void *mu, const void *nu, const bfm_grid *grid, bfm_cost cost,
                     bfm_precision prec, double tol, int max_iter, const bfm_options *opt,
                     void *workspace, size_t workspace_bytes, void *stream, bfm_result *out);

/*
 * The same solve driven step by step by the caller (Algorithm 1 as above);
 * all solver state lives in the workspace and the host keeps nothing between
 * calls.  Each call takes the same grid, precision, max_iter and workspace.
 *   bfm_solver_init     validates and normalises mu, nu (DEVICE, N each), fills
 *                       the tables, measures ||nu - 1||^2_{H^-1} and sets
 *                       phi_0 = 0 (or keeps phi when opt->warm_start) in `phi`;
 *                       `phi`, `psi` are DEVICE fields of N elements that hold
 *                       the iterates.  Synchronises once to check the inputs.
 *   bfm_solver_iterate  enqueues `iterations` iterations of opt->method (opt:
 *                       the options given to bfm_solver_init, NULL for the
 *                       defaults) on `stream` without synchronising; once the
 *                       device has converged (or reached max_iter) further
 *                       iterations do no work.  With BFM_GRADIENT_ASCENT the
 *                       `psi` field is written by bfm_solver_finish only.
 *   bfm_solver_finish   measures the current phi_n if the loop has not
 *                       stopped, then fills `out` exactly as bfm_solve does
 *                       (out->phi and out->psi must be the `phi`, `psi` of the
 *                       earlier calls).  Synchronises the stream.
 */
bfm_status bfm_solver_init(const void *mu, const void *nu, const bfm_grid *grid, bfm_cost cost,
                           bfm_precision prec, double tol, int max_iter, const bfm_options *opt,
                           void *workspace, size_t workspace_bytes, void *stream,
                           void *phi, void *psi);
bfm_status bfm_solver_iterate(const bfm_grid *grid, bfm_precision prec, int max_iter,
                              int iterations, const bfm_options *opt, void *workspace,
                              size_t workspace_bytes, void *stream, void *phi, void *psi);
bfm_status bfm_solver_finish(const bfm_grid *grid, bfm_precision prec, int max_iter,
                             void *workspace, size_t workspace_bytes, void *stream,
                             bfm_result *out);

/*
 * Per-launch timing of the library's kernels with CUDA events (this host
 * thread only; the paper has no counterpart, it is measurement support).
 * bfm_profile_begin(k) creates 2k events and starts recording one event pair
 * around every kernel group the solver enqueues; bfm_profile_end waits for
 * the recorded events and fills, for each kind 0..nkinds-1 (names from
 * bfm_profile_kind_name), the summed milliseconds and the number of kernel
 * launches; *dropped counts groups beyond k that were not recorded.
 */
int bfm_profile_kinds(void);
const char *bfm_profile_kind_name(int kind);
bfm_status bfm_profile_begin(int max_records);
bfm_status bfm_profile_end(double *ms_by_kind, int *launches_by_kind, int nkinds, int *dropped);

/*
 * Many independent problems of uneven sizes (Algorithm 1 on each, as in
 * bfm_solve), solved together: problem p has grid grids[p], DEVICE inputs
 * mu[p], nu[p] and the outputs/logs of outs[p] (see bfm_result).  Each problem
 * keeps its own step size, logs and convergence flag; a problem that has
 * converged (or reached max_iter) does no further work while the others
 * continue.  Problems of equal grid shape share each kernel launch; a chunk of
 * opt->poll_every iterations is captured once as a CUDA graph and replayed
 * until every problem has stopped.  Returns BFM_OK when all converged,
 * BFM_NOT_CONVERGED when some reached max_iter (outs[p].converged says which).
 * opt->warm_start, the gradient-ascent method and power costs are not
 * supported here (BFM_ERR_UNSUPPORTED).  Synchronises `stream`.
 */
size_t bfm_workspace_bytes_batched(int nprob, const bfm_grid *grids, bfm_precision prec,
                                   int max_iter);
bfm_status bfm_solve_batched(int nprob, const void *const *mu, const void *const *nu,
                             const bfm_grid *grids, bfm_cost cost, bfm_precision prec, double tol,
                             int max_iter, const bfm_options *opt, void *workspace,
                             size_t workspace_bytes, void *stream, bfm_result *outs);

/*
 * Backward of the loss W2^2(mu_p, nu_p) for a batch of converged solves.  By
 * the envelope theorem on the dual problem (eq. (symmetric_dual)) at its
 * optimum, dC/dnu = phi and dC/dmu = psi, so along mass-preserving
 * perturbations of the density values
 *     grad_mu[p] = grad_out[p] * 2 hd (psi[p] - mean psi[p]) / mass_mu[p],
 *     grad_nu[p] = grad_out[p] * 2 hd (phi[p] - mean phi[p]) / mass_nu[p],
 * hd = 1/N.  phi, psi: DEVICE potentials from the forward solves (N each);
 * mass_mu, mass_nu: HOST, the masses bfm_solve reported; grad_out: DEVICE,
 * nprob elements of the call's precision; grad_mu, grad_nu: DEVICE outputs
 * (N each), either array (or an entry of it) may be NULL to skip it.
 * Synchronises `stream`.
 */
size_t bfm_w2_backward_workspace_bytes(int nprob);
bfm_status bfm_w2_backward(int nprob, const bfm_grid *grids, bfm_precision prec,
                           const void *const *phi, const void *const *psi,
                           const double *mass_mu, const double *mass_nu, const void *grad_out,
                           void *const *grad_mu, void *const *grad_nu, void *workspace,
                           size_t workspace_bytes, void *stream);

/* Workspace bytes for bfm_solve_host: bfm_workspace_bytes plus device room
 * for mu, nu, phi, psi and the map. */
size_t bfm_workspace_bytes_host(const bfm_grid *grid, bfm_precision prec, int max_iter);

/*
 * bfm_solve with HOST inputs and outputs: copies mu, nu (host, N elements)
 * into the device workspace, solves, and copies phi, psi (N each) and map
 * (ndim*N, may be NULL) back to the host arrays given in out->phi/psi/map.
 * Same algorithm and return values as bfm_solve.
 */
bfm_status bfm_solve_host(const void *mu, const void *nu, const bfm_grid *grid, bfm_cost cost,
                          bfm_precision prec, double tol, int max_iter, const bfm_options *opt,
                          void *workspace, size_t workspace_bytes, void *stream, bfm_result *out);

/*
 * The grid c-transform for the quadratic cost (Definition 2.1; Section 4.1):
 *     out(x) = min over grid points y of |x - y|^2 / 2 - phi(y),
 * computed by dimension splitting into exact 1-D lower envelopes along each
 * axis in turn (Section 4.1).  phi, out: DEVICE, N elements; out may equal
 * phi (in place).  Needs no workspace.
 */
bfm_status bfm_ctransform(const void *phi, void *out, const bfm_grid *grid,
                          bfm_precision prec, void *stream);

/* Workspace bytes for bfm_poisson (twiddle and eigenvalue tables, partial sums). */
size_t bfm_poisson_workspace_bytes(const bfm_grid *grid, bfm_precision prec);

/*
 * Neumann Poisson solve of Lemma 2.3 / eq. (gradients_J_I):
 *     g = (-Delta_h)^{-1} (f - mean f),
 * Delta_h the 5/7-point Laplacian with reflected ghost cells, diagonalised by
 * DCT-II along every axis (Section 4.3 inverts the Laplacian by FFT); the
 * zero mode is set to 0.  f, g: DEVICE, N elements (g may equal f).
 * G_out (HOST, may be NULL) receives ||f - mean f||^2_{H^-1} = ||g||^2_{H1-dot}
 * (eq. (defHm1dot)) in FP64; when it is non-NULL the stream is synchronised.
 */
bfm_status bfm_poisson(const void *f, void *g, const bfm_grid *grid, bfm_precision prec,
                       double *G_out, void *workspace, size_t workspace_bytes, void *stream);

/*
 * bfm_poisson without a workspace, for callers that cannot allocate device
 * memory (their device memory is owned by another allocator, or allocating
 * after start-up is forbidden because cudaMalloc/cudaFree synchronise the
 * device).  The paper has no counterpart: it is a memory-management variant of
 * bfm_poisson and computes the same g and G (same arguments, same meaning).
 * Its scratch is a 1 MiB array built into the library (one per device, kept
 * until the process exits), which holds every 2D or 3D grid with at most 4096
 * cells per axis in either precision; a grid that needs more scratch returns
 * BFM_ERR_UNSUPPORTED.  The call allocates no device memory.
 * The first call on a device (with that device current) looks up the array's
 * device address; make that first call before any stream capture begins.
 * Every call on a device uses the same array: calls whose GPU work overlaps
 * (different streams or host threads) race and must be serialised by the
 * caller.  The looked-up address is kept per device for the life of the
 * process; cudaDeviceReset rebuilds the device's context and module, after
 * which the kept address is stale, so do not call this entry point on a
 * device after resetting it.
 */
bfm_status bfm_poisson_noalloc(const void *f, void *g, const bfm_grid *grid, bfm_precision prec,
                               double *G_out, void *stream);

/*
 * The map of Lemma 2.2(ii) for the quadratic cost, T(x) = x - grad psi(x),
 * with grad psi by central differences (one-sided at the first and last cell
 * of each line) and T clamped to the box of cell centres.
 * psi: DEVICE, N elements; map: DEVICE, ndim*N elements ([0,1] coordinates).
 */
bfm_status bfm_map(const void *psi, void *map, const bfm_grid *grid, bfm_precision prec,
                   void *stream);

/*
 * The c-transform (Definition 2.1) and the map (Lemma 2.2(ii)) of the
 * separable power cost c(x,y) = sum_a |y_a - x_a|^{p_a}/p_a (Section 5, eq.
 * p_costs; the fast c-transform of Section 4.1): phi^c by dimension splitting,
 * each 1-D pass by the divide-and-conquer over the monotone minimiser, and
 * T_a(x) = x_a - sign(w_a)|w_a|^{1/(p_a - 1)} with w = grad psi by central
 * differences (one-sided at the first and last cell), clamped as in bfm_map.
 * p: HOST, ndim exponents with 1 < p_a <= 16 (axis 0 first); other arguments
 * as bfm_ctransform and bfm_map.  A line must fit in shared memory (up to
 * 8192 FP32 or 4096 FP64 cells); longer lines return BFM_ERR_UNSUPPORTED.
 */
bfm_status bfm_ctransform_power(const void *phi, void *out, const bfm_grid *grid,
                                bfm_precision prec, const double *p, void *stream);
bfm_status bfm_map_power(const void *psi, void *map, const bfm_grid *grid, bfm_precision prec,
                         const double *p, void *stream);

/*
 * Pushforward rho = T # mu (Section 2.1; the first variation of Lemma 3.1)
 * with T(x) = x - grad psi(x) as in bfm_map, discretised by depositing the
 * mass of every cell with mu != 0 onto the 2^d cell centres around T(x) with
 * bilinear / trilinear weights.  psi, mu: DEVICE, N elements; rho: DEVICE,
 * N elements, overwritten (density values: mass is conserved).
 */
bfm_status bfm_pushforward(const void *psi, const void *mu, void *rho, const bfm_grid *grid,
                           bfm_precision prec, void *stream);

/*
 * Displacement interpolation of Section 4.3 (images):
 *     rho_t = (S_t) # mu,   S_t(x) = t T(x) + (1 - t) x,
 * deposited as in bfm_pushforward.  map: DEVICE, ndim*N ([0,1] coordinates,
 * as bfm_map / bfm_solve write it); mu, rho: DEVICE, N elements; 0 <= t <= 1.
 */
bfm_status bfm_interpolate(const void *map, const void *mu, double t, void *rho,
                           const bfm_grid *grid, bfm_precision prec, void *stream);

/*
 * Launch shapes of the line c-transform (Section 4.1 computes the transform
 * line by line; here a thread takes K consecutive cells of a line and a CTA
 * W lines) and the autotuner that chooses them by timing.  The paper has no
 * counterpart: its transform is a sequential sweep.  Kinds of line kernel
 * (kind): 0 = tile rows (axis 0, lines of at most 256 cells), 1 = tile
 * columns (axes > 0, W neighbouring lines interleaved), 2 = the row kernel
 * (axis 0, rows of more than 256 cells), 3 = the row kernel on interleaved
 * tiles (axes > 0, lines of more than 256 cells where a tile of the default
 * shape spans at least 32 bytes per element position; longer lines along
 * axis 1 of a 2-D grid are swept as rows of a transposed copy by the solver,
 * and take kind 1 in the batched solver and in bfm_ctransform).  A shape is
 * (K, W) with W = 0 for "as many lines as fit" (512 threads, about 110 KB of
 * shared memory).
 * Every shape computes the same exact discrete envelope; shapes differ in
 * speed only (and in rounding order where hidden-parabola tests tie).
 * The table of chosen shapes is process-wide, read whenever a pass is
 * planned (bfm_solve captures its plan once per call); set shapes before a
 * solve starts, not while one runs in another thread.
 *
 * bfm_tune_candidates: the shapes the tuner tries for lines of n cells of
 *   this kind, into K[i], W[i] (HOST, cap entries; may be NULL to count).
 *   Returns their number, or -1 for an unknown kind or n < 2.
 * bfm_tune_default: the hand-picked shape (-1 as above).
 * bfm_tune_set: store a shape (BFM_ERR_INVALID_ARG unless it is a candidate).
 * bfm_tune_get: the shape plans take now; returns 1 if stored, 0 if default.
 * bfm_tune_clear: forget every stored shape.
 * bfm_tune_pick: the tuner's choice among timings ms[0..ncand) (ms <= 0:
 *   not measured): the fastest, unless the default (default_index, or -1)
 *   is within a factor 1 + margin of it, when the default stays.
 * bfm_tune_passes: the (kind, n) pairs the c-transforms of a solve on this
 *   grid read (batched != 0: of the batched solver), into kinds[i], ns[i]
 *   (HOST, cap entries); returns their number, -1 for an unsupported grid.
 * bfm_autotune_scratch_bytes: device scratch bfm_autotune needs (two fields
 *   of about 8 M cells of lines of n cells), 0 for an unknown kind or n.
 * bfm_autotune: time every candidate of (kind, n) on a synthetic field in
 *   `scratch` (DEVICE, caller-owned, 256-byte aligned, at least
 *   bfm_autotune_scratch_bytes) on `stream` (CUDA events, median of five
 *   launches after two untimed ones), store the pick (margin 2%) and return
 *   it in K_out, W_out (HOST, may be NULL); ms_out (HOST, may be NULL)
 *   receives up to ms_cap candidate times in the order of
 *   bfm_tune_candidates.  Synchronises the stream.  Errors:
 *   BFM_ERR_INVALID_ARG (kind/n), BFM_ERR_WORKSPACE (scratch), BFM_ERR_CUDA;
 *   on an error the table entry of (kind, n) is left as it was.
 */
int bfm_tune_candidates(int kind, int n, bfm_precision prec, int *K, int *W, int cap);
int bfm_tune_default(int kind, int n, bfm_precision prec, int *K, int *W);
bfm_status bfm_tune_set(int kind, int n, bfm_precision prec, int K, int W);
int bfm_tune_get(int kind, int n, bfm_precision prec, int *K, int *W);
void bfm_tune_clear(void);
int bfm_tune_pick(const double *ms, int ncand, int default_index, double margin);
int bfm_tune_passes(const bfm_grid *grid, bfm_precision prec, int batched, int *kinds, int *ns,
                    int cap);
size_t bfm_autotune_scratch_bytes(int kind, int n, bfm_precision prec);
bfm_status bfm_autotune(int kind, int n, bfm_precision prec, void *scratch, size_t scratch_bytes,
                        void *stream, int *K_out, int *W_out, double *ms_out, int ms_cap);

#ifdef __cplusplus
}
#endif

#endif /* BFM_H */
