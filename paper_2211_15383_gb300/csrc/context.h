// Context of the library: device-resident gauge field, multigrid hierarchy,
// deflation space, per-term statistics and a named work-space pool.
#pragma once

#include <atomic>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

struct mgmlmc_ctx;

namespace mg {

struct Level {
    int lx = 0, lt = 0, d = 0;       // sites per direction, dof per site
    int nsites = 0;
    long long n = 0;                 // nsites * d
    // operator as 5-point block stencil [site][5][d][d] (level 0: d = 2, used by the
    // Galerkin product; the fine solve uses the link-based Wilson kernel)
    double2* A64 = nullptr;
    float2* A32 = nullptr;
    // block-Jacobi smoother (coarse levels above the coarsest): Minv[s] = A[s][0]^{-1},
    // Ahat = block stencil of D M^{-1}
    double2* Minv64 = nullptr;
    float2* Minv32 = nullptr;
    double2* Ahat64 = nullptr;
    float2* Ahat32 = nullptr;
    // mg_precision 16, d = 16: Ahat as BF16 real 32 x 32 operands of the tensor-core stencil
    __nv_bfloat16* Ahat16 = nullptr;
    __nv_bfloat16* A16 = nullptr;    // the same for D_l itself (the V-cycle residual)
    // prolongation to the next level: [site][d][nvec]
    int ax = 0, at = 0, nvec = 0;
    double2* P64 = nullptr;
    float2* P32 = nullptr;
    double2* tv = nullptr;           // test vectors [nvec][n]
    // coarsest level: dense inverse [n][n]
    double2* Dinv64 = nullptr;
    float2* Dinv32 = nullptr;
    __nv_bfloat16* Dinv16 = nullptr;  // [Re | Im] BF16 embedding for the tensor-core solve
};

struct Deflation {
    int k = 0;
    int fine = -1;                   // fine level (0-based) of the term it belongs to
    int coarse = -1;                 // coarse level of that term (-1: last term)
    bool inexact = false;            // vectors from a loose eigensolve, L = A R computed
    double2* Lv = nullptr;           // [n][k] left vectors of the traced operator (V)
    double2* Rv = nullptr;           // [n][k] right vectors (U)
    double* a = nullptr;             // [k] 1/sigma
    std::vector<double> lambda;      // eigenvalues of Q_L
    double tau_re = 0, tau_im = 0;   // tr(V Sigma^{-1} U^H)
    // mg_precision 16: the factors rounded to BF16 for the tensor-core projections
    // (W^T = [Re R | -Im R | Re L | -Im L]^T, pre-tiled) and the deflated trace of
    // exactly those rounded factors, which the estimate then adds
    __nv_bfloat16* W16 = nullptr;
    double tau16_re = 0, tau16_im = 0;
    double tau_used_re() const { return W16 ? tau16_re : tau_re; }
    double tau_used_im() const { return W16 ? tau16_im : tau_im; }
};

struct TermStats {
    long long n = 0;
    double sum_re = 0, sum_im = 0, sum_abs2 = 0;
    double seconds = 0;
    long long iters = 0;
};

// CUDA-event timing of kernel classes with their algorithmic bytes and flops
// per launch (the per-operation timing of Sect. 4.3: D_l, P_l, P_l^H,
// deflations, axpy-type updates).
struct ProfStat {
    long long count = 0;
    double ms = 0, bytes = 0, flops = 0;
    double impl_bytes = 0;           // bytes the implementation moves (>= the algorithmic bytes)
};
struct Profiler {
    bool on = false;
    std::map<std::string, ProfStat> stats;
    struct Pending {
        std::string key;
        cudaEvent_t a, b;
        double bytes, flops, impl_bytes;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    long long launch_base = 0;       // launch_counter() at the last reset
    cudaEvent_t take();
    void resolve();      // call after the stream is synchronised
    void clear();
    ~Profiler();
};

struct Ctx;
// Brackets the launches issued during its lifetime with events (when enabled);
// the entry joins the profiler's pending list only once both events are
// recorded, so a synchronisation inside the scope is harmless.
struct ProfScope {
    Ctx* c;
    bool active;
    Profiler::Pending p;
    // impl_bytes < 0: the implementation moves the algorithmic bytes
    ProfScope(Ctx& ctx, const std::string& key, double bytes, double flops, double impl_bytes = -1);
    ~ProfScope();
};

struct Ctx {
    mgmlmc_options opt{};
    Profiler prof;
    cudaStream_t stream = nullptr;
    mgmlmc_alloc_fn alloc = nullptr;
    mgmlmc_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string err;
    double* hbuf = nullptr;          // pinned host scratch for scalar read-backs
    int* dev_err = nullptr;          // device error flag of kernels with bounded waits
    size_t hbuf_bytes = 0;

    int Lx = 0, Lt = 0;
    bool have_gauge = false, have_mass = false, have_hier = false;
    double m0 = 0;
    double2* U64 = nullptr;          // links [site][2]
    float2* U32 = nullptr;

    int L = 0;
    Level lev[MGMLMC_MAX_LEVELS];
    int nterms = 0;
    int term_level[MGMLMC_MAX_LEVELS + 1] = {0};   // 0-based fine level of each term
    std::vector<int> skip;
    Deflation defl;                  // coarsest term: k smallest triplets of D_L (Sect. 2)
    Deflation ddefl[MGMLMC_MAX_LEVELS];   // difference terms, by fine level: largest triplets of M_l (Sect. 4.2)
    TermStats stats[MGMLMC_MAX_LEVELS];
    long long last_iters = 0;        // outer iterations of the last solve
    // iterations of the last inner FGMRES cycle, by level, rhs count and decade of its
    // tolerance
    std::map<long long, int> cycle_hint;
    // the refinement loop may take its residuals from FP32 products between FP64 ones
    // (the estimator's solves: Z2 right-hand sides, no strong cancellation in D e)
    bool fp32_residual_updates = false;

    // ---- memory
    struct Buf { void* p = nullptr; size_t bytes = 0; };
    std::map<std::string, Buf> ws;
    std::unordered_map<void*, size_t> owned;   // device allocations and their sizes
    size_t live_bytes = 0, peak_bytes = 0;     // device bytes held now and at most

    void* dev_alloc(size_t bytes);
    void dev_free(void* p);
    template <typename T> T* alloc_n(size_t count) { return reinterpret_cast<T*>(dev_alloc(count * sizeof(T))); }
    // Named scratch that grows on demand; contents are undefined after growth.
    void* scratch_bytes(const std::string& name, size_t bytes);
    template <typename T> T* scratch(const std::string& name, size_t count) {
        return reinterpret_cast<T*>(scratch_bytes(name, count * sizeof(T)));
    }
    void release_all();
    // Frees the named work space whose names start with one of the prefixes.
    void free_scratch(const std::vector<std::string>& prefixes);
    void free_hierarchy();
    void free_deflation();
    void sync();
};

// ---- solver layer (solver.cu)
template <typename C> void apply_D(Ctx& c, int l, C* y, const C* x, const C* b, int N, int mode, double2* dots);
template <typename C> void apply_restrict(Ctx& c, int l, C* xc, const C* x, int N);
template <typename C> void apply_prolong(Ctx& c, int l, C* x, const C* xc, int N, bool accumulate);
template <typename C> void mg_cycle(Ctx& c, int l, C* e, const C* r, int N);
// y = D_l M_l^{-1} x, the operator of the block-Jacobi smoother (coarse levels
// above the coarsest); dots (2N, may be null) receive conj(y).x and |y|^2 per rhs.
template <typename C> void apply_smoother_operator(Ctx& c, int l, C* y, const C* x, int N, double2* dots);
// FGMRES(m) in precision C on level l; x holds the initial guess (zero if x_zero).
// At most max_cycles restart cycles.  Returns outer iterations; *ok = 1 if the
// relative residual reached tol (or the cycle budget ended, for inner solves).
template <typename C>
long long fgmres(Ctx& c, int l, const C* b, C* x, int N, double tol, long long maxit, bool x_zero, int* ok,
                 int max_cycles);
// FP64-accurate solve D_l x = b (plain FP64 FGMRES, or mixed iterative refinement).
long long solve(Ctx& c, int l, const double2* b, double2* x, int N, double tol, int* ok);
// One FGMRES cycle (restart length m) in the multigrid precision: x ~ D_l^{-1} b.
void approx_inverse(Ctx& c, int l, const double2* b, double2* x, int N);
void column_norms(Ctx& c, double* out, const double2* x, long long n, int N);
// Throws MGMLMC_ETIMEOUT if a kernel with bounded waits recorded a timeout.
void check_device_error(Ctx& c);
// The context's device flag that kernels with bounded waits set when they give up.
int* device_error_flag(Ctx& c);
// d receives device copies of s's gauge field, mass, hierarchy, terms and deflations.
void copy_state(Ctx& d, Ctx& s);
// Throws MGMLMC_EINVAL for options outside their documented ranges.
void check_options(const mgmlmc_options& o);
// The MLMC loop of mgmlmc_estimate_trace(_concurrent): term t draws its samples on
// ctx_of[t] (one host thread per term with `concurrent`); when *cancel becomes true
// the loop stops at its next round with MGMLMC_ECANCELLED.
void mlmc_loop(const std::vector<Ctx*>& ctx_of, bool concurrent, double rel_tol, int64_t max_samples, uint64_t seed,
               const double* costs, mgmlmc_trace_result* out, const std::atomic<bool>* cancel = nullptr);

// ---- setup (setup.cu)
void build_hierarchy(Ctx& c, int nlevels, const int* ax, const int* at, const int* nvec, int setup_iters,
                     double setup_tol, const double* const* start_vectors);
// Exact deflation of the last term (fine level a): k smallest triplets of D_a.
// With inexact, the vectors come from the eigensolver as they are and the
// deflated part is recomputed from them (see store_deflation).
// eig_solve_tol: tolerance of the eigensolver's solves (0: 1e-3 tol, within
// [solve_tol, 1e-6]).
void compute_deflation(Ctx& c, int a, int k, double tol, int max_iters, bool inexact = false,
                       double eig_solve_tol = 0);
// Exact deflation of the difference term with fine level a and coarse level b
// (0-based): k largest singular triplets of M from eigenpairs of J = M Gamma5^a.
void compute_difference_deflation(Ctx& c, int a, int b, int k, double tol, int max_iters, bool inexact = false,
                                  double eig_solve_tol = 0);
// Deflation of term (a, b) by given right vectors R [n_a][k] (device): L = A R with
// A the term's traced operator (FP64-accurate solves), a_i = 1.
void set_deflation_vectors(Ctx& c, int a, int b, const double2* R, int k);
// The deflation that applies to the term (a, b), or nullptr.
const Deflation* term_deflation(const Ctx& c, int a, int b);
// With mg_precision 16 and a supported level size: the BF16 copy of the factors and
// the deflated trace over them (called whenever a deflation is stored).
void prepare_tc_deflation(Ctx& c, Deflation& D);
void upload_links(Ctx& c, const double* theta);

}  // namespace mg

struct mgmlmc_ctx {
    mg::Ctx c;
};
