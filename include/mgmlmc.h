/*
 * mgmlmc.h -- C ABI of the GB300 (sm_103a) deflated multigrid multilevel
 * Monte Carlo library: stochastic estimation of tr(D^{-1}) for the 2D
 * Wilson-Schwinger operator D (Frommer & Ramirez-Hidalgo, "Deflated Multigrid
 * Multilevel Monte Carlo", Lattice 2022).
 *
 * General conventions
 *  - Every call returns an int status (mgmlmc_status); no exception, abort or
 *    exit crosses the ABI.  After a failure mgmlmc_last_error(ctx) holds text.
 *  - Complex numbers are interleaved (re, im) doubles.  Host arrays are owned
 *    by the caller and only read or written during the call.
 *  - Device state (gauge links, hierarchy, deflation space, Krylov work space)
 *    is owned by the context and released by mgmlmc_destroy.  Device memory is
 *    taken from the caller's allocator callback when one is given (the Python
 *    binding passes PyTorch's caching allocator), else from cudaMalloc.
 *  - All GPU work runs on the CUDA stream given to mgmlmc_create.  Calls that
 *    return host data synchronise that stream.  A context is not thread safe.
 *  - Vectors of level l have n_l = sites_l * d_l complex entries ordered
 *    site-major (site = x + lx * t), then dof; d_1 = 2 (spin), d_l = 2 nvec_{l-1}
 *    on coarse levels, whose first nvec dof form spin block 0 (Gamma5 = +1) and
 *    the next nvec spin block 1 (Gamma5 = -1).
 *  - Multi-vector host arrays are [vector][n_l] (one vector after another).
 */
#ifndef MGMLMC_H
#define MGMLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGMLMC_MAX_LEVELS 6

typedef enum {
    MGMLMC_OK = 0,
    MGMLMC_EINVAL = -1,          /* invalid argument                                  */
    MGMLMC_ENOMEM = -2,          /* device or host allocation refused                 */
    MGMLMC_ENOTCONVERGED = -3,   /* an iteration hit its cap; partial results marked   */
    MGMLMC_ETIMEOUT = -4,        /* a bounded device wait gave up                      */
    MGMLMC_ECUDA = -5,           /* CUDA runtime error                                 */
    MGMLMC_ENOTIMPL = -6,        /* combination not implemented                        */
    MGMLMC_ENAN = -7,            /* NaN/Inf met in the data                            */
    MGMLMC_ESTATE = -8,          /* call out of order (e.g. estimate before hierarchy) */
    MGMLMC_ECANCELLED = -9,      /* a served request was cancelled                     */
    MGMLMC_PENDING = 1           /* mgmlmc_poll / mgmlmc_wait: request not finished    */
} mgmlmc_status;

typedef struct mgmlmc_ctx mgmlmc_ctx;

/* Device allocator hooks: alloc returns a device pointer (NULL = refused). */
typedef void* (*mgmlmc_alloc_fn)(void* user, size_t bytes);
typedef void (*mgmlmc_free_fn)(void* user, void* ptr);

typedef struct {
    int mg_precision;     /* 64: FP64 multigrid preconditioner ("plain FP64 path");
                             32: FP32 V-cycle with a BF16 tensor-core coarsest solve
                             (mixed); 16: as 32, and the coarse-level smoother's
                             block stencil (d = 16) on the tensor cores in BF16.
                             The outer FGMRES, its residuals and every sample are
                             FP64 in all cases.                                [64]    */
    double solve_tol;     /* relative residual ||b - D x|| / ||b|| of every solve;
                             Sect. 4.3 uses 1e-12.                             [1e-12] */
    int fgmres_restart;   /* Krylov basis size m of the outer FGMRES(m).       [24]    */
    int max_iters;        /* cap on outer iterations of one solve.             [2000]  */
    int nu_pre;           /* pre-smoothing MR steps per level (Eq. two_level_mg). [0]  */
    int nu_post;          /* post-smoothing MR steps per level.                [4]     */
    int max_block_rhs;    /* most right-hand sides solved together.            [256]   */
    int verbose;          /* 1: iteration counts on stderr.                    [0]     */
    int kcycle_iters;     /* coarse-grid correction of the multigrid cycle (Sect. 3.1,
                             Eq. two_level_mg_method applied recursively): 0 = one
                             cycle on the next level (V-cycle); k > 0 = k steps of
                             flexible GMRES on the next level preconditioned by its
                             own cycle (K-cycle), wherever that level is not the
                             coarsest.  The steps run entirely on the device.  0..16.
                                                                               [0]     */
} mgmlmc_options;

/* Per-term statistics of the samples drawn so far (FP64, Sect. 3.2). */
typedef struct {
    int64_t nsamples;     /* N_l                                   */
    double sum_re, sum_im;/* sum of samples s_j                    */
    double sum_abs2;      /* sum of |s_j|^2                         */
    double mean_re, mean_im;
    double variance;      /* unbiased E|s - mean|^2                 */
    double seconds;       /* device time spent on this term         */
    int64_t iters;        /* outer FGMRES iterations, summed        */
} mgmlmc_level_stats;

typedef struct {
    double trace_re, trace_im;   /* sum of term means + deflated part          */
    double rel_err;              /* sqrt(sum_l V_l / N_l) / |trace|             */
    double deflated_part;        /* tr(V Sigma^{-1} U^H) term (real part)       */
    int nterms;
    int converged;               /* rel_err <= rel_tol                          */
    int rounds;
    mgmlmc_level_stats term[MGMLMC_MAX_LEVELS];
} mgmlmc_trace_result;

/* Operators for mgmlmc_apply. */
typedef enum {
    MGMLMC_OP_D = 0,      /* y = D_l x                       (l = 1..L)           */
    MGMLMC_OP_PH = 1,     /* y = P_l^H x   (level l -> l+1)   (l = 1..L-1)         */
    MGMLMC_OP_P = 2,      /* y = P_l x     (level l+1 -> l)   (l = 1..L-1)         */
    MGMLMC_OP_G5 = 3,     /* y = Gamma5^l x                                         */
    MGMLMC_OP_PREC = 4,   /* y = one multigrid cycle from level l applied to x      */
    MGMLMC_OP_DINV_C = 5, /* y = stored inverse of the coarsest D_L applied to x    */
    MGMLMC_OP_SMOOTH = 6  /* y = D_l M_l^{-1} x, M_l the block diagonal (self blocks)
                             of D_l: the operator the coarse-level smoother iterates
                             on (l = 2..L-1; BF16 tensor cores when mg_precision = 16) */
} mgmlmc_opkind;

/* Fill *opt with the defaults shown in brackets above. */
void mgmlmc_default_options(mgmlmc_options* opt);

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream).  alloc/free may be NULL (then cudaMalloc and
 * cudaFree).  opt may be NULL (defaults).  On success *out owns all state. */
int mgmlmc_create(mgmlmc_ctx** out, const mgmlmc_options* opt, void* cuda_stream,
                  mgmlmc_alloc_fn alloc, mgmlmc_free_fn free_fn, void* alloc_user);

/* A second context holding device copies of src's state: gauge field, mass,
 * options, hierarchy (test vectors, prolongators, coarse operators, smoother and
 * coarsest data), term list and deflations (Sects. 2, 3.1) — none of the setup
 * is computed again.  It runs on cuda_stream with its own work space and
 * statistics; the intended use is one context per term for
 * mgmlmc_estimate_concurrent / mgmlmc_estimate_trace_concurrent.  src's stream is
 * synchronised first.  On failure *out is NULL and src holds the message. */
int mgmlmc_create_copy(mgmlmc_ctx** out, mgmlmc_ctx* src, void* cuda_stream, mgmlmc_alloc_fn alloc,
                       mgmlmc_free_fn free_fn, void* alloc_user);

/* Replace the solver options of a context: block width, restart length, iteration
 * cap, smoothing steps, coarse-grid correction, solve tolerance, verbosity (the
 * setting mgmlmc_autotune makes, or a caller's).  mg_precision must stay what the
 * context was created with (MGMLMC_EINVAL otherwise): it decides which operator
 * copies the hierarchy holds.  Later calls use the new options. */
int mgmlmc_set_options(mgmlmc_ctx* ctx, const mgmlmc_options* opt);

/* Release every device allocation of the context, then the context. */
void mgmlmc_destroy(mgmlmc_ctx* ctx);

/* Text of the last error of this context ("" if none).  Valid until the next call. */
const char* mgmlmc_last_error(const mgmlmc_ctx* ctx);

/* Gauge field (Sect. 1: U(1) links of the Schwinger model).  theta is a host
 * array [t][x][mu] of Lt*Lx*2 link angles, U_mu(x) = exp(i theta); mu = 0 is
 * space (periodic), mu = 1 is time (antiperiodic fermion boundary).  Lx, Lt
 * even and >= 2.  Invalidates any hierarchy and deflation. */
int mgmlmc_set_gauge(mgmlmc_ctx* ctx, int Lx, int Lt, const double* theta);

/* Wilson mass m0: D = (m0 + 2) - 1/2 sum_mu [(1 - sigma_mu) U_mu(x) T_{+mu}
 * + (1 + sigma_mu) U_mu^*(x - mu) T_{-mu}] with sigma_0 = sigma_1, sigma_1 =
 * sigma_2 (Pauli), Gamma5 = sigma_3.  Invalidates hierarchy and deflation. */
int mgmlmc_set_mass(mgmlmc_ctx* ctx, double m0);

/* Multigrid hierarchy (Sect. 3.1; spin-preserving aggregation, Sect. 4.2).
 * nlevels = L in 1..MGMLMC_MAX_LEVELS; for l = 1..L-1 aggregates of
 * agg_x[l-1] x agg_t[l-1] sites of level l and nvec[l-1] test vectors.
 * start_vectors[l-1] is a host array [nvec][n_l] of complex start vectors;
 * the setup runs setup_iters rounds of inverse iteration v <- D_l^{-1} v
 * (solved to relative residual setup_tol), v <- v/||v||, then orthonormalises
 * each vector's restriction to an (aggregate, spin block) in vector order
 * (modified Gram-Schmidt) to form P_l, and D_{l+1} = P_l^H D_l P_l.
 * setup_iters = 0 uses the start vectors as they are.  Returns
 * MGMLMC_EINVAL if a block has fewer rows than nvec or a vector block is
 * rank deficient.  Invalidates deflation. */
int mgmlmc_set_hierarchy(mgmlmc_ctx* ctx, int nlevels, const int* agg_x, const int* agg_t,
                         const int* nvec, int setup_iters, double setup_tol,
                         const double* const* start_vectors);

/* Terms of the telescoping sum (Eq. mgmlmc).  nskip levels listed in skip
 * (2..L) are left out of the sum, giving Eq. skip_level for skip = {2}, and
 * plain (deflated) Hutchinson on D_1 (Sect. 2) for skip = {2..L}:
 * tr(D^{-1}) = tr(D_1^{-1} - P_1 P_2 D_3^{-1} P_2^H P_1^H) + ... .  nskip = 0
 * restores the plain sum.  Term t (0-based) then has fine level
 * term_level[t] and coarse level term_level[t+1] (none for the last term).
 * Skipping the last levels (e.g. skip = {4, 5} with L = 5) ends the sum at a
 * level above the coarsest: the levels below it then serve only the solver
 * (the multigrid cycle recurses through them down to the stored inverse of
 * D_L), and the last term is tr(D_c^{-1}) of that level c. */
int mgmlmc_set_terms(mgmlmc_ctx* ctx, int nskip, const int* skip);
int mgmlmc_num_terms(const mgmlmc_ctx* ctx, int* nterms, int* term_level /* [MGMLMC_MAX_LEVELS] */);

/* Exact deflation of the last term (Sect. 2), whose operator D_L is the
 * coarsest level of the sum (the hierarchy's last level unless mgmlmc_set_terms
 * ended the sum above it; then D_L below means that level's operator): the k
 * smallest singular triplets of D_L from the eigenpairs of Q_L = Gamma5^L D_L (U = Gamma5 X
 * sign(Lambda), Sigma = |Lambda|, V = X), found by subspace iteration on
 * Q_L^{-1} with Rayleigh-Ritz until every residual ||Q x - lambda x|| <=
 * tol |lambda| (Sect. 4.3 uses tol = 1e-9), at most max_iters iterations.
 * Each iteration's solves run to max(solve_tol, min(1e-6, 1e-3 tol)): any
 * vectors leave the estimator unbiased, since tau below comes from the stored
 * factors.
 * k = 0 removes deflation.  Also computes tau = tr(V Sigma^{-1} U^H) (Eq.
 * small_trace_term) in FP64 from the stored factors. */
int mgmlmc_compute_deflation(mgmlmc_ctx* ctx, int k, double tol, int max_iters);

/* Host copies of the deflation: lambda[k], sigma[k], U and V as [k][n_L]
 * complex (n_L of the deflated level), tau (2 doubles).  Any pointer may be NULL. */
int mgmlmc_get_deflation(mgmlmc_ctx* ctx, double* lambda, double* sigma, double* U,
                         double* V, double* tau);

/* Exact deflation of term t (0-based).  For the last (coarsest) term this is
 * mgmlmc_compute_deflation.  For a difference term with fine level a and coarse
 * level b (Sect. 4.2, exact deflation on difference levels): the k largest
 * singular triplets of M = D_a^{-1} - P D_b^{-1} P^H (P = P_a ... P_{b-1}) from the
 * eigenpairs of the Hermitian J = M Gamma5^a = Q_a^{-1} - P Q_b^{-1} P^H,
 * J = X Lambda X^H -> U = X sign(Lambda), S = |Lambda|, V = Gamma5^a X (Eq.
 * hermitian_diff_lev_op), by subspace iteration on J (two FP64-accurate solves
 * per application) with Rayleigh-Ritz until ||J x - lambda x|| <= tol |lambda|
 * for the k wanted pairs (Sect. 4.3 uses 1e-9), at most max_iters iterations.
 * The term's samples then subtract x^H U S V^H x and the estimate adds
 * tr(U S V^H) = sum_i lambda_i x_i^H Gamma5 x_i.  k = 0 removes it.  A later
 * mgmlmc_set_terms that changes the term's coarse level disables it. */
int mgmlmc_compute_term_deflation(mgmlmc_ctx* ctx, int term, int k, double tol, int max_iters);

/* Inexact deflation of term t (Sect. 3.2/4.3: loosely converged vectors, the
 * paper uses eigensolver tolerance 1e-1 and inner solves at 1e-3): the same
 * eigensolver as mgmlmc_compute_term_deflation run to eig_tol with its solves at
 * inner_tol gives approximate vectors V (Gamma5 X); the term is then deflated by
 * the orthogonal projector V V^H with the deflated part computed from V by k
 * extra solves at opt.solve_tol ("the computation of tr(D^{-1} Pi) requires k
 * extra inversions"): samples subtract x^H (A V) V^H x, the estimate adds
 * tr(V^H A V), A the term's traced operator.  Unbiased for any V. */
int mgmlmc_compute_term_deflation_inexact(mgmlmc_ctx* ctx, int term, int k, double eig_tol, double inner_tol,
                                          int max_iters);

/* Deflation of term t by caller-supplied vectors V (host, [k][n_a] complex; the
 * projector V V^H is orthogonal when V has orthonormal columns): the library
 * computes A V with k FP64-accurate solves, as in the inexact deflation. */
int mgmlmc_set_term_deflation_vectors(mgmlmc_ctx* ctx, int term, int k, const double* V);

/* Host copies of term t's deflation: *k, lambda[k] (eigenvalues of the Hermitian
 * operator), the traced operator's left vectors L and right vectors R as [k][n_a]
 * complex (L = V, R = U for the coarsest term; L = U, R = V for a difference
 * term), tau (2 doubles) = its deflated trace part.  Pointers may be NULL. */
int mgmlmc_get_term_deflation(mgmlmc_ctx* ctx, int term, int* k, double* lambda, double* L, double* R,
                              double* tau);

/* The deflated trace part that the estimate adds for term t (0-based; 2 doubles,
 * zero without deflation).  With mg_precision 64 or 32 it is the tau of the
 * stored FP64 factors (mgmlmc_get_term_deflation).  With mg_precision 16 the
 * samples form the deflation projections on the tensor cores from the factors
 * rounded to BF16 (FP64 -> FP32 -> BF16, to nearest) with FP32 accumulation, and
 * this part is the trace over exactly those rounded factors, computed in FP64 —
 * so the estimate stays unbiased for the factors it uses (Sect. 2, Eq.
 * splitting_defl_trace holds for any fixed factors). */
int mgmlmc_term_deflated_part(mgmlmc_ctx* ctx, int term, double* tau);

/* nsamples Hutchinson samples of term t (0-based; Sect. 3.2):
 *   s_j = x_j^H D_a^{-1} x_j - (P^H x_j)^H D_b^{-1} (P^H x_j)   (difference term)
 *   s_j = x_j^H D_L^{-1} x_j - (V^H x_j)^H Sigma^{-1} (U^H x_j) (deflated coarsest)
 * with P = P_{a->b} the prolongation between the term's levels and x_j the Z2
 * vector j = first_sample + i drawn on the device: entry k is +1 or -1 by the
 * low bit of sm(sm(sm(seed ^ a) ^ j) ^ k), sm = one splitmix64 step.  Solves to
 * opt.solve_tol in blocks of at most opt.max_block_rhs.  samples_out (host,
 * 2*nsamples doubles, may be NULL) receives s_j; *stats (may be NULL) receives
 * this call's statistics, and the context adds them to the term's running
 * totals.  MGMLMC_ENOTCONVERGED if a solve hit opt.max_iters. */
int mgmlmc_estimate_level(mgmlmc_ctx* ctx, int term, int64_t first_sample, int nsamples,
                          uint64_t seed, double* samples_out, mgmlmc_level_stats* stats);

/* Same as mgmlmc_estimate_level but with caller-supplied real probe vectors:
 * probes is a host array [nsamples][n_a] of signed bytes (the entries of x_j,
 * e.g. +-1 for Z2 noise), copied to the device inside the call. */
int mgmlmc_estimate_level_probes(mgmlmc_ctx* ctx, int term, int nsamples, const int8_t* probes,
                                 double* samples_out, mgmlmc_level_stats* stats);

/* Several terms at once: the terms of the telescoping sum are independent
 * (Sect. 3.2), so entry i runs mgmlmc_estimate_level (probes NULL or probes[i]
 * NULL) or mgmlmc_estimate_level_probes (probes[i] a host array [nsamples][n_a])
 * for term terms[i] on contexts[i], each entry on its own host thread (entry 0
 * on the calling one).  The contexts must be distinct (MGMLMC_EINVAL otherwise),
 * built from the same gauge field, mass and hierarchy inputs if their samples
 * are to be combined, and each created on its own CUDA stream: their kernels
 * then overlap on the GPU, and the host round trips of one term (convergence
 * checks) are covered by the others' work.  first_sample and seed apply to the
 * device-noise entries.  samples_out (may be NULL; so may each samples_out[i])
 * receives 2*nsamples doubles per entry; stats (may be NULL) n statistics.
 * Returns MGMLMC_OK, or the status of the first entry that failed (that
 * context holds its message); every entry runs to completion either way. */
int mgmlmc_estimate_concurrent(mgmlmc_ctx* const* contexts, int n, const int* terms, int64_t first_sample,
                               int nsamples, uint64_t seed, const int8_t* const* probes,
                               double* const* samples_out, mgmlmc_level_stats* stats);

/* Running totals of term t since the last mgmlmc_reset_stats. */
int mgmlmc_get_stats(mgmlmc_ctx* ctx, int term, mgmlmc_level_stats* stats);
int mgmlmc_reset_stats(mgmlmc_ctx* ctx);

/* Multilevel Monte Carlo estimate of tr(D^{-1}) (Eq. mgmlmc, with deflation
 * of the coarsest term when computed): pilot of 16 samples per term, then
 * rounds that raise N_l towards eps^-2 sqrt(V_l/C_l) sum_m sqrt(V_m C_m)
 * (eps = rel_tol |estimate|; at most doubling per round) until
 * sqrt(sum_l V_l/N_l) <= rel_tol |estimate| or max_samples in total.
 * costs[t] gives fixed per-sample costs C_l (NULL: measured device seconds).
 * Sample indices of term t run 0, 1, 2, ... on the noise stream of seed. */
int mgmlmc_estimate_trace(mgmlmc_ctx* ctx, double rel_tol, int64_t max_samples, uint64_t seed,
                          const double* costs, mgmlmc_trace_result* out);

/* mgmlmc_estimate_trace with the terms drawn at once: contexts[t] (n = the number
 * of terms, distinct contexts built from the same inputs, each created on its own
 * CUDA stream) draws the samples of term t, on one host thread per term within
 * each round of the loop; the allocation and the stopping rule see all terms'
 * statistics, as in mgmlmc_estimate_trace.  Errors are reported in contexts[0]. */
int mgmlmc_estimate_trace_concurrent(mgmlmc_ctx* const* contexts, int n, double rel_tol, int64_t max_samples,
                                     uint64_t seed, const double* costs, mgmlmc_trace_result* out);

/* Test hook: y = op(x) for nrhs host vectors [nrhs][n_in] -> [nrhs][n_out]. */
int mgmlmc_apply(mgmlmc_ctx* ctx, int op, int level, int nrhs, const double* x, double* y);

/* Solve D_l x = b for nrhs host vectors [nrhs][n_l] with the outer FGMRES to
 * opt.solve_tol; *iters (may be NULL) receives the outer iteration count. */
int mgmlmc_solve(mgmlmc_ctx* ctx, int level, int nrhs, const double* b, double* x, int* iters);

/* Test hook: the Z2 vectors of mgmlmc_estimate_level as doubles [nsamples][n_l]. */
int mgmlmc_noise(mgmlmc_ctx* ctx, int level, int64_t first_sample, int nsamples, uint64_t seed,
                 double* x);

/* Test hook: the test vectors after the setup iteration, [nvec][n_l] complex. */
int mgmlmc_get_test_vectors(mgmlmc_ctx* ctx, int level, double* v);

/* Per-operation timing (Sect. 4.3 times D_l, deflations, P_l, P_l^H and axpy
 * separately): with enable = 1 every launch of a kernel class is bracketed by
 * CUDA events on the context's stream and its algorithmic bytes and flops are
 * recorded; reset = 1 clears the totals.  Classes: "D<l>.<prec>" operator
 * applications, "PH<l>", "P<l>" restriction/prolongation, "Dinv.<prec>"
 * coarsest solve, "mr<l>" smoother updates, "orth" Gram-Schmidt, "defl"
 * deflation projections. */
int mgmlmc_profile(mgmlmc_ctx* ctx, int enable, int reset);

/* JSON object {class: {"count", "ms", "bytes", "flops"}} of the totals so far,
 * written to buf (capacity cap, NUL-terminated); *needed receives the length. */
int mgmlmc_profile_report(mgmlmc_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* Measurement helper (no counterpart in the paper): achieved fused
 * multiply-add throughput of the current device in FLOP/s for precision 64 or
 * 32, from a kernel of independent FMA chains on every SM (best of 3). */
int mgmlmc_fma_peak(int precision, double* flops_per_s);

/* Allocation-free coarsest solve (the paper has no counterpart; this is a service
 * for callers that must not allocate device memory while they run, e.g. code
 * running under a host framework that owns a fixed device-memory budget, or a
 * real-time loop that cannot take the synchronisation that cudaMalloc/cudaFree
 * imply).
 * y = D_L^{-1} x with the stored BF16 inverse on the tensor cores: the computation
 * of mgmlmc_apply(MGMLMC_OP_DINV_C) in the mixed modes.  The results agree with
 * that call within FP32 accumulation rounding, not bit for bit: this call sums
 * over the whole of n_L in one pass, the context path may split the sum.  x and y
 * are caller-owned device arrays of nrhs FP32 complex vectors laid out
 * [n_L][nrhs] (row-major, rhs fastest, interleaved re/im); y must not alias x,
 * y must be 16-byte aligned and x 8-byte aligned (MGMLMC_EINVAL otherwise).
 * Needs mg_precision 32 or 16 and n_L % 128 == 0 (MGMLMC_ESTATE otherwise); nrhs
 * a multiple of 32 with n_L * nrhs <= 2^20 (MGMLMC_EINVAL otherwise).
 * Work space: a file-scope 8 MiB device array, present on every GPU that loads
 * the library until the process exits; every call overwrites it entirely (no
 * part needs to start at zero), so calls that overlap on the GPU (different
 * streams or threads) race and must be serialised by the caller.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture begins.  The
 * call runs on `stream` (a
 * cudaStream_t, NULL = default stream) and synchronises it before returning, to
 * read the kernel's status; MGMLMC_ETIMEOUT if a bounded wait inside the kernel
 * gave up. */
int mgmlmc_coarse_inverse_noalloc(mgmlmc_ctx* ctx, int nrhs, const float* x, float* y, void* stream);

/* One timed setting of mgmlmc_autotune. */
#define MGMLMC_TUNE_LOG 16
typedef struct {
    int block_rhs, fgmres_restart, nu_post, kcycle_iters;
    double samples_per_s;
} mgmlmc_tune_trial;

/* Result of mgmlmc_autotune. */
typedef struct {
    int block_rhs;        /* chosen opt.max_block_rhs                                  */
    int fgmres_restart;   /* chosen opt.fgmres_restart                                 */
    int nu_post;          /* chosen opt.nu_post                                        */
    int kcycle_iters;     /* chosen opt.kcycle_iters                                   */
    double samples_per_s; /* measured rate of the chosen setting: one block per term   */
    size_t footprint;     /* modelled device bytes of the chosen setting               */
    size_t budget;        /* the budget the candidates were held to                    */
    int trials;           /* settings timed                                            */
    mgmlmc_tune_trial log[MGMLMC_TUNE_LOG];   /* the first trials, in order             */
} mgmlmc_tune_result;

/* Autotuner (no counterpart in the paper): chooses the block width, the FGMRES
 * restart length, the post-smoothing steps and the coarse-grid correction of this
 * context for this GPU.  Candidates whose modelled device footprint (the model of
 * mgmlmc_request_footprint for the context's own shape) exceeds hbm_budget bytes
 * (0: 90 % of the free device memory plus what the context holds) are skipped; at
 * most max_trials others are timed on one block of samples of every term (a fixed
 * Z2 noise block; the context's statistics are not touched): the three widest blocks
 * that fit with a restart of at most 16, then restart length (8, 16, 24), smoother
 * steps (2, 6) and, with four levels or more, the other coarse-grid correction.
 * The fastest becomes the context's setting; its work space is released.  Needs a
 * hierarchy (and the deflation, if any, already computed).  MGMLMC_ENOMEM if no
 * block width fits the budget. */
int mgmlmc_autotune(mgmlmc_ctx* ctx, size_t hbm_budget, int max_trials, mgmlmc_tune_result* out);

/* Level geometry: sites per direction, dof per site, n_l. */
int mgmlmc_level_info(const mgmlmc_ctx* ctx, int level, int* lx, int* lt, int* d, int64_t* n);

/* Device bytes the context holds now (*live) and has held at most (*peak) through
 * its allocator (either may be NULL).  Pinned host scratch is not counted. */
int mgmlmc_memory(const mgmlmc_ctx* ctx, size_t* live, size_t* peak);

/* ---- Serving: trace requests admitted continuously on one GPU ----------------
 * A server takes whole trace problems (gauge field, mass, hierarchy, deflation,
 * target relative error: the estimation of tr(D^{-1}) of Sect. 3.2 with the
 * deflated coarsest term of Sect. 2, one request each) and runs them on the current
 * CUDA device.  A request is admitted when a slot is free and its estimated device
 * footprint fits in the server's HBM budget beside the requests already admitted;
 * each admitted request gets its own context (hierarchy, deflation space and Krylov
 * work space stay on the device until it finishes) and CUDA stream, and its work
 * overlaps on the device with that of the other admitted requests.  Inside a
 * request all samples of a term in one round are solved as multi-rhs blocks of
 * up to opt.max_block_rhs right-hand sides.  Queued requests are admitted in
 * arrival order; a request that does not fit may be overtaken by later ones that
 * do, at most max_bypass times, after which nothing behind it is admitted before
 * it.  Device memory of the requests comes from a stream-ordered pool owned by the
 * server (no device-wide synchronisation when a request frees its memory).
 * All server calls are thread safe.  Results do not depend on what else runs:
 * with fixed costs a request's rounds, sample counts and estimate are those it
 * gets alone. */
typedef struct mgmlmc_server mgmlmc_server;

typedef struct {
    size_t hbm_budget;    /* device bytes the admitted requests may reserve together
                             (0: 3/4 of the free device memory at creation)    [0]  */
    int max_active;       /* most requests admitted at once (1..64)            [4]  */
    int max_bypass;       /* times a queued request may be overtaken           [4]  */
} mgmlmc_server_options;

typedef struct {
    int Lx, Lt;           /* lattice (as mgmlmc_set_gauge)                          */
    const double* theta;  /* host link angles [Lt][Lx][2]; copied by mgmlmc_submit  */
    double m0;            /* Wilson mass                                            */
    int nlevels;          /* multigrid levels (1..MGMLMC_MAX_LEVELS)                */
    int agg_x[MGMLMC_MAX_LEVELS], agg_t[MGMLMC_MAX_LEVELS], nvec[MGMLMC_MAX_LEVELS];
                          /* aggregates and test vectors per spin of levels
                             1..nlevels-1 (as mgmlmc_set_hierarchy)                 */
    const double* start_vectors[MGMLMC_MAX_LEVELS];
                          /* host [nvec][n_l] complex start vectors of levels
                             1..nlevels-1 (as mgmlmc_set_hierarchy); copied          */
    int setup_iters;      /* inverse-iteration steps of the hierarchy setup         */
    double setup_tol;     /* solve tolerance of those steps                          */
    int k;                /* smallest triplets of the coarsest operator deflated (0: none) */
    double defl_tol;      /* eigensolver tolerance (as mgmlmc_compute_deflation)     */
    int defl_max_iters;
    double rel_tol;       /* target relative error of the estimate (> 0)             */
    int64_t max_samples;  /* cap on samples over all terms                           */
    uint64_t seed;        /* noise seed of the estimate                              */
    double costs[MGMLMC_MAX_LEVELS]; /* per-sample cost of each term for the sample
                             allocation, > 0 for each of the terms; all zero:
                             measured device time (then the allocation depends on
                             the load)                                               */
    mgmlmc_options opt;   /* context options (mgmlmc_default_options for defaults)  */
    int sum_levels;       /* levels 1..sum_levels start the terms of the sum and the
                             deflation acts on level sum_levels; the levels below
                             serve only the solver (as mgmlmc_set_terms with the last
                             levels skipped).  0: all nlevels                        */
} mgmlmc_request;

typedef struct {
    int status;           /* MGMLMC_OK, the failing call's status, or MGMLMC_ECANCELLED */
    mgmlmc_trace_result result;
    double queued_s;      /* submission -> admission                                 */
    double setup_s;       /* admission -> hierarchy and deflation ready              */
    double estimate_s;    /* the MLMC loop                                           */
    double total_s;       /* submission -> result: the time to trace                 */
    size_t reserved_bytes;/* footprint reserved at admission                         */
    size_t peak_bytes;    /* device bytes the request's context held at most         */
    int retries;          /* re-admissions after a refused device allocation         */
    char error[160];      /* text of the failure ("" if none)                        */
    int deflation_converged; /* 1: the deflation eigensolver reached defl_tol; 0: it
                             stopped at defl_max_iters and the request went on with the
                             factors it had (the estimate adds their own deflated
                             trace, so it stays unbiased), or k = 0                    */
} mgmlmc_request_result;

typedef struct {
    int queued, active;   /* requests waiting / admitted now                        */
    int64_t completed;    /* requests finished (any status) since creation           */
    int max_active_seen;  /* most requests admitted at once so far                   */
    size_t budget;        /* the HBM budget in force                                 */
    size_t reserved;      /* bytes reserved by the admitted requests now             */
    size_t max_reserved;  /* most bytes reserved at once so far (<= budget)          */
} mgmlmc_server_stats;

/* Upper estimate of the device bytes a request's context holds at most: the
 * operators of every level, the dense coarsest inverse in each precision used, the
 * deflation space and eigensolver blocks, and the Krylov, refinement, V-cycle and
 * estimator blocks of opt.max_block_rhs right-hand sides.  MGMLMC_EINVAL if the
 * lattice, hierarchy or options are malformed (as mgmlmc_set_gauge /
 * mgmlmc_set_hierarchy / mgmlmc_create),
 * MGMLMC_ENOTIMPL if the coarsest level has more than 16384 unknowns.  Host only:
 * needs no device.  (The same model, for a context's own shape, bounds the
 * candidates of mgmlmc_autotune.) */
int mgmlmc_request_footprint(const mgmlmc_request* req, size_t* bytes);

/* Create a server on the current CUDA device (opt NULL: defaults).  MGMLMC_ECUDA
 * without a device; MGMLMC_EINVAL for a bad option. */
int mgmlmc_server_create(mgmlmc_server** out, const mgmlmc_server_options* opt);

/* Cancel queued requests, stop running ones at their next check, wait for them,
 * release the pool and the server.  Results not yet polled are lost.  No other call
 * on this server may be in progress or follow (a thread blocked in mgmlmc_wait
 * must have returned first). */
void mgmlmc_server_destroy(mgmlmc_server* srv);

/* Queue a request (the struct, theta and the start vectors are copied; the caller
 * may free them on return).  *id identifies it for poll, wait and cancel.  The footprint reserved
 * for it is mgmlmc_request_footprint while no request of the same shape (lattice,
 * hierarchy, k, precision, block width, restart length) has finished, then 1.1 x
 * the largest device peak of those that have.  MGMLMC_EINVAL for a malformed
 * request, MGMLMC_ENOMEM if that footprint exceeds the whole budget. */
int mgmlmc_submit(mgmlmc_server* srv, const mgmlmc_request* req, uint64_t* id);

/* MGMLMC_OK and *out filled once the request has finished (its own outcome is
 * out->status); the id is released then.  MGMLMC_PENDING while it is queued or
 * running, MGMLMC_EINVAL for an unknown id. */
int mgmlmc_poll(mgmlmc_server* srv, uint64_t id, mgmlmc_request_result* out);

/* mgmlmc_poll after waiting at most timeout_s seconds (< 0: no limit) for the
 * request to finish. */
int mgmlmc_wait(mgmlmc_server* srv, uint64_t id, double timeout_s, mgmlmc_request_result* out);

/* Cancel a request: a queued one finishes at once, a running one at its next check
 * (between setup steps and between rounds of the MLMC loop), with status
 * MGMLMC_ECANCELLED.  MGMLMC_EINVAL for an unknown or already finished id. */
int mgmlmc_cancel(mgmlmc_server* srv, uint64_t id);

/* Counters of the server (queue, admitted requests, reserved bytes). */
int mgmlmc_get_server_stats(mgmlmc_server* srv, mgmlmc_server_stats* out);

/* Text of the last server call that failed on the calling thread ("" if none). */
const char* mgmlmc_server_last_error(const mgmlmc_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* MGMLMC_H */
