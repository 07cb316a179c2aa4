// Context memory management, gauge upload, multigrid hierarchy setup
// (Sect. 3.1, spin-preserving aggregation of Sect. 4.2) and the exact deflation
// of the coarsest operator (Sect. 2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "context.h"

namespace mg {

// ------------------------------------------------------------------ memory
void* Ctx::dev_alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (alloc) {
        p = alloc(alloc_user, bytes);
        if (!p) throw Error(MGMLMC_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes refused");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(MGMLMC_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        }
    }
    owned[p] = bytes;
    live_bytes += bytes;
    peak_bytes = std::max(peak_bytes, live_bytes);
    return p;
}

void Ctx::dev_free(void* p) {
    if (!p) return;
    auto it = owned.find(p);
    if (it == owned.end()) return;
    live_bytes -= it->second;
    owned.erase(it);
    if (free_fn) free_fn(alloc_user, p);
    else cudaFree(p);
}

void* Ctx::scratch_bytes(const std::string& name, size_t bytes) {
    Buf& b = ws[name];
    if (b.p && b.bytes >= bytes) return b.p;
    if (b.p) dev_free(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = ((bytes + 255) / 256) * 256;
    b.p = dev_alloc(want);
    b.bytes = want;
    return b.p;
}

void Ctx::free_scratch(const std::vector<std::string>& prefixes) {
    sync();
    for (auto it = ws.begin(); it != ws.end();) {
        bool hit = false;
        for (const auto& p : prefixes) hit |= it->first.compare(0, p.size(), p) == 0;
        if (hit) {
            dev_free(it->second.p);
            it = ws.erase(it);
        } else {
            ++it;
        }
    }
}

void Ctx::release_all() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& kv : owned) {
        if (free_fn) free_fn(alloc_user, kv.first);
        else cudaFree(kv.first);
    }
    owned.clear();
    live_bytes = 0;
    ws.clear();
    dev_err = nullptr;
    for (auto& L : lev) L = Level();
    U64 = nullptr;
    U32 = nullptr;
    defl = Deflation();
}

static void free_one_deflation(Ctx& c, Deflation& d) {
    c.dev_free(d.Lv);
    c.dev_free(d.Rv);
    c.dev_free(d.a);
    c.dev_free(d.W16);
    d = Deflation();
}

void Ctx::free_deflation() {
    free_one_deflation(*this, defl);
    for (auto& d : ddefl) free_one_deflation(*this, d);
}

const Deflation* term_deflation(const Ctx& c, int a, int b) {
    if (b < 0) return (c.defl.k > 0 && c.defl.fine == a) ? &c.defl : nullptr;
    const Deflation& d = c.ddefl[a];
    return (d.k > 0 && d.coarse == b) ? &d : nullptr;
}

void Ctx::free_hierarchy() {
    sync();
    for (int l = 0; l < MGMLMC_MAX_LEVELS; ++l) {
        Level& L = lev[l];
        dev_free(L.A64); dev_free(L.A32); dev_free(L.P64); dev_free(L.P32); dev_free(L.tv);
        dev_free(L.Minv64); dev_free(L.Minv32); dev_free(L.Ahat64); dev_free(L.Ahat32); dev_free(L.Ahat16); dev_free(L.A16);
        dev_free(L.Dinv64); dev_free(L.Dinv32); dev_free(L.Dinv16);
        L = Level();
    }
    free_deflation();
    L = 0;
    have_hier = false;
    for (auto& s : stats) s = TermStats();
}

void Ctx::sync() {
    MG_CUDA(cudaStreamSynchronize(stream));
    if (!prof.pending.empty()) prof.resolve();
}

// ------------------------------------------------------------------ profiler
std::atomic<long long>& launch_counter() {
    static std::atomic<long long> n{0};
    return n;
}

cudaEvent_t Profiler::take() {
    if (pool.empty()) {
        cudaEvent_t e;
        MG_CUDA(cudaEventCreate(&e));
        return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
}
void Profiler::resolve() {
    for (auto& p : pending) {
        float ms = 0;
        MG_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        ProfStat& s = stats[p.key];
        s.count += 1;
        s.ms += ms;
        s.bytes += p.bytes;
        s.flops += p.flops;
        s.impl_bytes += p.impl_bytes;
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}
void Profiler::clear() {
    stats.clear();
    launch_base = launch_counter();
}
Profiler::~Profiler() {
    for (auto& p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}
ProfScope::ProfScope(Ctx& ctx, const std::string& key, double bytes, double flops, double impl_bytes)
    : c(&ctx), active(ctx.prof.on) {
    if (!active) return;
    p = Profiler::Pending{key, c->prof.take(), c->prof.take(), bytes, flops, impl_bytes < 0 ? bytes : impl_bytes};
    MG_CUDA(cudaEventRecord(p.a, c->stream));
}
ProfScope::~ProfScope() {
    if (!active) return;
    cudaEventRecord(p.b, c->stream);
    c->prof.pending.push_back(p);
}

// ------------------------------------------------------------------ gauge
// ------------------------------------------------------------------ copy of a context
template <typename T>
static T* dup(Ctx& d, const T* p, size_t count) {
    if (!p) return nullptr;
    T* q = d.alloc_n<T>(count);
    MG_CUDA(cudaMemcpyAsync(q, p, count * sizeof(T), cudaMemcpyDeviceToDevice, d.stream));
    return q;
}

static void dup_deflation(Ctx& d, const Ctx& s, const Deflation& from, Deflation& to) {
    to = Deflation();
    if (!from.Lv) return;
    const size_t n = (size_t)s.lev[from.fine].n, k = (size_t)from.k;
    to.k = from.k;
    to.fine = from.fine;
    to.coarse = from.coarse;
    to.inexact = from.inexact;
    to.lambda = from.lambda;
    to.tau_re = from.tau_re;
    to.tau_im = from.tau_im;
    to.Lv = dup(d, from.Lv, n * k);
    to.Rv = dup(d, from.Rv, n * k);
    to.a = dup(d, from.a, k);
    to.W16 = from.W16 ? dup(d, from.W16, (size_t)tc_deflation_rows(from.k) * n) : nullptr;
    to.tau16_re = from.tau16_re;
    to.tau16_im = from.tau16_im;
}

// d (fresh, on its own stream) receives s's gauge field, mass, hierarchy, term list
// and deflations: device copies of every array, no setup computation repeated.
void copy_state(Ctx& d, Ctx& s) {
    MG_CUDA(cudaStreamSynchronize(s.stream));
    d.Lx = s.Lx;
    d.Lt = s.Lt;
    d.have_gauge = s.have_gauge;
    d.have_mass = s.have_mass;
    d.have_hier = s.have_hier;
    d.m0 = s.m0;
    const size_t V = (size_t)s.Lx * s.Lt;
    d.U64 = dup(d, s.U64, 2 * V);
    d.U32 = dup(d, s.U32, 2 * V);
    d.L = s.L;
    for (int l = 0; l < s.L; ++l) {
        const Level& b = s.lev[l];
        Level& a = d.lev[l];
        a = Level();
        a.lx = b.lx;
        a.lt = b.lt;
        a.d = b.d;
        a.nsites = b.nsites;
        a.n = b.n;
        a.ax = b.ax;
        a.at = b.at;
        a.nvec = b.nvec;
        const size_t nb = (size_t)b.nsites * b.d * b.d;
        a.A64 = dup(d, b.A64, 5 * nb);
        a.A32 = dup(d, b.A32, 5 * nb);
        a.Minv64 = dup(d, b.Minv64, nb);
        a.Minv32 = dup(d, b.Minv32, nb);
        a.Ahat64 = dup(d, b.Ahat64, 5 * nb);
        a.Ahat32 = dup(d, b.Ahat32, 5 * nb);
        a.Ahat16 = dup(d, b.Ahat16, 5 * nb * 4);
        a.A16 = dup(d, b.A16, 5 * nb * 4);
        a.P64 = dup(d, b.P64, (size_t)b.n * b.nvec);
        a.P32 = dup(d, b.P32, (size_t)b.n * b.nvec);
        a.tv = dup(d, b.tv, (size_t)b.n * b.nvec);
        a.Dinv64 = dup(d, b.Dinv64, (size_t)b.n * b.n);
        a.Dinv32 = dup(d, b.Dinv32, (size_t)b.n * b.n);
        a.Dinv16 = dup(d, b.Dinv16, (size_t)b.n * 2 * b.n);
    }
    d.nterms = s.nterms;
    for (int t = 0; t <= MGMLMC_MAX_LEVELS; ++t) d.term_level[t] = s.term_level[t];
    d.skip = s.skip;
    dup_deflation(d, s, s.defl, d.defl);
    for (int l = 0; l < MGMLMC_MAX_LEVELS; ++l) dup_deflation(d, s, s.ddefl[l], d.ddefl[l]);
    MG_CUDA(cudaStreamSynchronize(d.stream));
}

void upload_links(Ctx& c, const double* theta) {
    const int V = c.Lx * c.Lt;
    std::vector<double2> U((size_t)2 * V);
    for (int i = 0; i < 2 * V; ++i) {
        const double th = theta[i];
        MG_REQUIRE(std::isfinite(th), MGMLMC_ENAN, "set_gauge: non-finite link angle");
        U[i] = make_double2(std::cos(th), std::sin(th));
    }
    c.dev_free(c.U64);
    c.dev_free(c.U32);
    c.U64 = c.alloc_n<double2>((size_t)2 * V);
    c.U32 = c.alloc_n<float2>((size_t)2 * V);
    MG_CUDA(cudaMemcpyAsync(c.U64, U.data(), sizeof(double2) * 2 * V, cudaMemcpyHostToDevice, c.stream));
    launch_convert<float2, double2>(c.U32, c.U64, 2LL * V, c.stream);
    c.sync();
}

// ------------------------------------------------------------------ small kernels
__global__ void k_scale_cols_rsqrt(double2* W, const double* lam, int b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int col = e % b;
    const double l = lam[col];
    const double f = (l > 0.0) ? 1.0 / sqrt(l) : 0.0;
    W[e] = make_double2(W[e].x * f, W[e].y * f);
}
__global__ void k_hermitize(double2* G, int b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e / b, j = e % b;
    if (i > j) return;
    const double2 a = G[i * b + j], t = G[j * b + i];
    const double2 h = make_double2(0.5 * (a.x + t.x), 0.5 * (a.y - t.y));
    G[i * b + j] = h;
    G[j * b + i] = make_double2(h.x, -h.y);
}
__global__ void k_resid_cols(double2* R, const double2* QX, const double2* X, const double* lam, long long n, int b) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * b) return;
    const int col = (int)(e % b);
    R[e] = make_double2(QX[e].x - lam[col] * X[e].x, QX[e].y - lam[col] * X[e].y);
}
__global__ void k_reciprocal(double* v, int b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b) v[i] = (v[i] != 0.0) ? 1.0 / v[i] : 1e300;
}
__global__ void k_sign_cols(double2* Y, const double* lam, long long n, int b) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n * b) return;
    if (lam[(int)(e % b)] < 0.0) Y[e] = make_double2(-Y[e].x, -Y[e].y);
}
__global__ void k_inv_abs(double* a, const double* lam, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) a[i] = 1.0 / fabs(lam[i]);
}
__global__ void k_abs(double* a, const double* lam, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) a[i] = fabs(lam[i]);
}
// tau = sum_i a_i t_i  (t_i = u_i^H v_i), fixed order, one thread.
__global__ void k_weighted_sum(double2* out, const double2* t, const double* a, int k) {
    if (threadIdx.x || blockIdx.x) return;
    double2 s = make_double2(0, 0);
    for (int i = 0; i < k; ++i) s = make_double2(s.x + a[i] * t[i].x, s.y + a[i] * t[i].y);
    *out = s;
}

static void small_launch_check() { MG_LAUNCHED(); }

void prepare_tc_deflation(Ctx& c, Deflation& D) {
    c.dev_free(D.W16);
    D.W16 = nullptr;
    const long long n = c.lev[D.fine].n;
    if (c.opt.mg_precision != 16 || D.k < 1 || !tc_deflation_supported(n, D.k)) return;
    D.W16 = c.alloc_n<__nv_bfloat16>((size_t)tc_deflation_rows(D.k) * n);
    launch_embed_deflation_bf16(D.W16, D.Rv, D.Lv, n, D.k, c.stream);
    double2* t = c.scratch<double2>("tcd_t", D.k);
    double2* tau = c.scratch<double2>("tcd_tau", 1);
    launch_deflation_tau_bf16(t, D.Rv, D.Lv, n, D.k, c.stream);
    k_weighted_sum<<<1, 1, 0, c.stream>>>(tau, t, D.a, D.k);
    small_launch_check();
    double2 h;
    MG_CUDA(cudaMemcpyAsync(&h, tau, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    D.tau16_re = h.x;
    D.tau16_im = h.y;
}


void column_norms(Ctx& c, double* out, const double2* x, long long n, int N);   // solver.cu
// Rounds of the preconditioner bootstrap: two, plus one per level beyond three (the
// deeper the hierarchy, the more its coarse levels built from random vectors weaken
// the first cycles).
static int bootstrap_rounds(int nlevels) { return 2 + std::max(0, nlevels - 3); }
constexpr int kSetupRestart = 64;
constexpr int kRefreshRounds = 2;
// Subspace iterations between Rayleigh-Ritz projections (and convergence checks).
constexpr int kRayleighRitzEvery = 4;

// ------------------------------------------------------------------ hierarchy
static void coarsest_inverse(Ctx& c) {
    Level& L = c.lev[c.L - 1];
    const long long n = L.n;
    MG_REQUIRE(n <= 16384, MGMLMC_ENOTIMPL, "coarsest level above 16384 unknowns (dense inverse) not supported");
    double2* Dd = c.scratch<double2>("dense_D", (size_t)n * n);
    launch_dense_from_blocks(Dd, L.A64, L.lx, L.lt, L.d, c.stream);
    void* work = c.scratch_bytes("gj_work", gauss_jordan_work_bytes((int)n));
    int* status = reinterpret_cast<int*>(reinterpret_cast<double2*>(work) + n) + n;
    if (c.opt.mg_precision == 64) {
        if (!L.Dinv64) L.Dinv64 = c.alloc_n<double2>((size_t)n * n);
        MG_CUDA(cudaMemcpyAsync(L.Dinv64, Dd, sizeof(double2) * n * n, cudaMemcpyDeviceToDevice, c.stream));
        ProfScope ps(c, "setup.gauss_jordan.f64", 2.0 * n * n * 16 * std::ceil(n / 16.0), 8.0 * n * n * n);
        launch_gauss_jordan<double2>(L.Dinv64, (int)n, work, c.stream);
    } else {
        if (!L.Dinv32) L.Dinv32 = c.alloc_n<float2>((size_t)n * n);
        launch_convert<float2, double2>(L.Dinv32, Dd, n * n, c.stream);
        ProfScope ps(c, "setup.gauss_jordan.f32", 2.0 * n * n * 8 * std::ceil(n / 32.0), 8.0 * n * n * n);
        launch_gauss_jordan<float2>(L.Dinv32, (int)n, work, c.stream);
        if (tc_coarse_supported((int)n)) {
            if (!L.Dinv16) L.Dinv16 = c.alloc_n<__nv_bfloat16>((size_t)n * 2 * n);
            launch_embed_bf16(L.Dinv16, L.Dinv32, (int)n, c.stream);
        }
    }
    int hs = 0;
    MG_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    MG_REQUIRE(hs == 0, MGMLMC_EINVAL, "coarsest operator is singular (zero pivot)");
}

// Block-Jacobi smoother of coarse level l: M = block diagonal of D_l (the self
// blocks), smoothing on the right-preconditioned operator D_l M^{-1}.
static void block_jacobi_setup(Ctx& c, int l) {
    Level& L = c.lev[l];
    const size_t nb = (size_t)L.nsites * L.d * L.d;
    if (!L.Minv64) {
        L.Minv64 = c.alloc_n<double2>(nb);
        L.Minv32 = c.alloc_n<float2>(nb);
        L.Ahat64 = c.alloc_n<double2>(nb * 5);
        L.Ahat32 = c.alloc_n<float2>(nb * 5);
    }
    int* status = c.scratch<int>("status_bj", 4);
    double2* work = c.scratch<double2>("bj_work", nb);
    MG_CUDA(cudaMemsetAsync(status, 0, sizeof(int), c.stream));
    launch_block_diag_inverse(L.Minv64, work, L.A64, L.nsites, L.d, status, c.stream);
    launch_precondition_blocks(L.Ahat64, L.A64, L.Minv64, L.lx, L.lt, L.d, c.stream);
    launch_convert<float2, double2>(L.Minv32, L.Minv64, (long long)nb, c.stream);
    launch_convert<float2, double2>(L.Ahat32, L.Ahat64, (long long)nb * 5, c.stream);
    if (c.opt.mg_precision == 16 && tc_stencil_supported(L.d, 2)) {
        if (!L.Ahat16) L.Ahat16 = c.alloc_n<__nv_bfloat16>((size_t)L.nsites * 5 * 4 * L.d * L.d);
        if (!L.A16) L.A16 = c.alloc_n<__nv_bfloat16>((size_t)L.nsites * 5 * 4 * L.d * L.d);
        launch_embed_stencil_bf16(L.Ahat16, L.Ahat32, L.nsites, c.stream);
        launch_embed_stencil_bf16(L.A16, L.A32, L.nsites, c.stream);
    }
    int hs = 0;
    MG_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    MG_REQUIRE(hs == 0, MGMLMC_EINVAL, "set_hierarchy: singular diagonal block on level " + std::to_string(l + 1));
}

static void rebuild_from(Ctx& c, int l0) {
    int* status = c.scratch<int>("status", 4);
    for (int l = l0; l < c.L - 1; ++l) {
        Level& L = c.lev[l];
        Level& Lc = c.lev[l + 1];
        MG_CUDA(cudaMemsetAsync(status, 0, sizeof(int), c.stream));
        launch_build_prolongator(L.P64, L.tv, L.lx, L.lt, L.d, L.ax, L.at, L.nvec, status, c.stream);
        int hs = 0;
        MG_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        MG_REQUIRE(hs == 0, MGMLMC_EINVAL,
                   "set_hierarchy: rank-deficient test vectors on an aggregate of level " + std::to_string(l + 1));
        launch_convert<float2, double2>(L.P32, L.P64, L.n * L.nvec, c.stream);
        double2* T = c.scratch<double2>("galerkin_T", galerkin_scratch_count(L.lx, L.lt, L.d, L.nvec));
        ProfScope ps(c, "setup.galerkin", 0, 0);
        launch_galerkin(Lc.A64, L.A64, L.P64, L.lx, L.lt, L.d, L.ax, L.at, L.nvec, T, c.stream);
        launch_convert<float2, double2>(Lc.A32, Lc.A64, (long long)Lc.nsites * 5 * Lc.d * Lc.d, c.stream);
        if (l + 1 < c.L - 1) block_jacobi_setup(c, l + 1);
    }
    coarsest_inverse(c);
}

void build_hierarchy(Ctx& c, int nlev, const int* ax, const int* at, const int* nvec, int setup_iters,
                     double setup_tol, const double* const* sv) {
    MG_REQUIRE(c.have_gauge && c.have_mass, MGMLMC_ESTATE, "set_hierarchy: gauge field and mass must be set first");
    MG_REQUIRE(nlev >= 1 && nlev <= MGMLMC_MAX_LEVELS, MGMLMC_EINVAL, "set_hierarchy: 1 <= nlevels <= 6");
    MG_REQUIRE(setup_iters >= 0 && setup_iters <= 100, MGMLMC_EINVAL, "set_hierarchy: 0 <= setup_iters <= 100");
    MG_REQUIRE(nlev == 1 || (ax && at && nvec && sv), MGMLMC_EINVAL, "set_hierarchy: NULL argument");
    int lx = c.Lx, lt = c.Lt, d = 2;
    for (int l = 0; l < nlev - 1; ++l) {
        MG_REQUIRE(ax[l] >= 1 && at[l] >= 1 && lx % ax[l] == 0 && lt % at[l] == 0, MGMLMC_EINVAL,
                   "set_hierarchy: aggregate extents must divide the lattice of level " + std::to_string(l + 1));
        MG_REQUIRE(nvec[l] >= 1 && nvec[l] <= 32, MGMLMC_EINVAL, "set_hierarchy: 1 <= nvec <= 32");
        MG_REQUIRE(nvec[l] <= ax[l] * at[l] * d / 2, MGMLMC_EINVAL,
                   "set_hierarchy: more test vectors than rows of an aggregate block on level " + std::to_string(l + 1));
        MG_REQUIRE(sv[l] != nullptr, MGMLMC_EINVAL, "set_hierarchy: missing start vectors");
        lx /= ax[l];
        lt /= at[l];
        d = 2 * nvec[l];
    }
    MG_REQUIRE((long long)lx * lt * d <= 16384, MGMLMC_ENOTIMPL,
               "set_hierarchy: coarsest level above 16384 unknowns (dense inverse) not supported");
    c.free_hierarchy();
    c.L = nlev;
    lx = c.Lx; lt = c.Lt; d = 2;
    for (int l = 0; l < nlev; ++l) {
        Level& L = c.lev[l];
        L.lx = lx; L.lt = lt; L.d = d;
        L.nsites = lx * lt;
        L.n = (long long)L.nsites * d;
        L.A64 = c.alloc_n<double2>((size_t)L.nsites * 5 * d * d);
        if (l > 0) L.A32 = c.alloc_n<float2>((size_t)L.nsites * 5 * d * d);
        if (l < nlev - 1) {
            L.ax = ax[l]; L.at = at[l]; L.nvec = nvec[l];
            L.P64 = c.alloc_n<double2>((size_t)L.n * L.nvec);
            L.P32 = c.alloc_n<float2>((size_t)L.n * L.nvec);
            L.tv = c.alloc_n<double2>((size_t)L.n * L.nvec);
            MG_CUDA(cudaMemcpyAsync(L.tv, sv[l], sizeof(double2) * L.n * L.nvec, cudaMemcpyHostToDevice, c.stream));
            lx /= ax[l]; lt /= at[l]; d = 2 * nvec[l];
        }
    }
    launch_materialize_wilson(c.lev[0].A64, c.U64, c.m0, c.Lx, c.Lt, c.stream);
    rebuild_from(c, 0);
    if (setup_iters > 0) {
        // The setup solves run nvec right-hand sides only, so their Krylov bases are
        // small: they use a restart length of at least kSetupRestart, which keeps the
        // low modes a hierarchy built from rough vectors still misses (a short restart
        // stagnates on them near the critical mass).
        struct RestartScope {
            Ctx& c;
            int keep;
            ~RestartScope() { c.opt.fgmres_restart = keep; }
        } restart_scope{c, c.opt.fgmres_restart};
        c.opt.fgmres_restart = std::max(c.opt.fgmres_restart, kSetupRestart);
        // Keep the start vectors: the test vectors are defined by exact inverse
        // iteration from them.
        std::vector<double2*> raw(nlev - 1);
        for (int l = 0; l < nlev - 1; ++l) {
            const Level& L = c.lev[l];
            raw[l] = c.scratch<double2>("setup_raw" + std::to_string(l), (size_t)L.n * L.nvec);
            MG_CUDA(cudaMemcpyAsync(raw[l], L.tv, sizeof(double2) * L.n * L.nvec, cudaMemcpyDeviceToDevice,
                                    c.stream));
        }
        // Preconditioner bootstrap: a hierarchy built from random vectors is too weak
        // for the near-critical solves of the inverse iteration, so first improve the
        // vectors of levels from..L-1 by rounds of approximate inverse iteration (one
        // FGMRES cycle each) on their current operators.  This only shapes the
        // preconditioner of the setup solves; the final test vectors come from the
        // exact iteration below.
        auto bootstrap = [&](int from, int rounds) {
            for (int round = 0; round < rounds; ++round)
                for (int l = from; l < nlev - 1; ++l) {
                    Level& L = c.lev[l];
                    const int nv = L.nvec;
                    double2* B = c.scratch<double2>("setup_B", (size_t)L.n * nv);
                    double2* X = c.scratch<double2>("setup_X", (size_t)L.n * nv);
                    double* nrm = c.scratch<double>("setup_nrm", nv);
                    launch_transpose(B, L.tv, nv, (int)L.n, c.stream);
                    approx_inverse(c, l, B, X, nv);
                    column_norms(c, nrm, X, L.n, nv);
                    launch_scale_rhs<double2, double2>(X, X, nrm, true, L.n, nv, c.stream);
                    launch_transpose(L.tv, X, L.n, nv, c.stream);
                    rebuild_from(c, l);
                }
        };
        bootstrap(0, bootstrap_rounds(nlev));
        // Inverse iteration v <- D_l^{-1} v / ||.|| from the start vectors, level by
        // level top-down, each solve to setup_tol.
        for (int l = 0; l < nlev - 1; ++l) {
            // the exact vectors of the levels above changed D_l and everything below it:
            // adapt level l's preconditioner (its vectors and the levels under it) to
            // those operators first
            if (l > 0) bootstrap(l, kRefreshRounds);
            Level& L = c.lev[l];
            const int nv = L.nvec;
            double2* B = c.scratch<double2>("setup_B", (size_t)L.n * nv);
            double2* X = c.scratch<double2>("setup_X", (size_t)L.n * nv);
            double* nrm = c.scratch<double>("setup_nrm", nv);
            launch_transpose(B, raw[l], nv, (int)L.n, c.stream);
            for (int it = 0; it < setup_iters; ++it) {
                int ok = 0;
                const long long its = solve(c, l, B, X, nv, setup_tol, &ok);
                if (c.opt.verbose)
                    fprintf(stderr, "[mgmlmc] setup level %d inverse iteration %d: %lld iterations%s\n", l + 1, it,
                            its, ok ? "" : " (not converged)");
                MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED,
                           "set_hierarchy: inverse-iteration solve on level " + std::to_string(l + 1) +
                               " did not converge");
                column_norms(c, nrm, X, L.n, nv);
                launch_scale_rhs<double2, double2>(B, X, nrm, true, L.n, nv, c.stream);
            }
            launch_transpose(L.tv, B, L.n, nv, c.stream);
            rebuild_from(c, l);
        }
    }
    c.sync();
    c.have_hier = true;
    c.nterms = nlev;
    for (int t = 0; t < nlev; ++t) c.term_level[t] = t;
    c.skip.clear();
}

// ------------------------------------------------------------------ deflation
// Block products of the eigensolvers.  On large levels with a loose tolerance they
// run with FP32 arithmetic on the FP64 vectors (fast = true): FP64 runs at 1/64 of
// the FP32 rate on this GPU, and n b^2 products at n = 262144, b = 1024 would take
// seconds each.  The Ritz residuals are still formed in FP64; FP32 rounding of the
// Ritz vectors limits them to about 1e-6 ||Q|| / |lambda| (hence the tolerance bound).
static bool fast_block_products(long long n, int b, double tol) {
    return (double)n * b * b * 8.0 > 2e11 && tol >= 1e-4;
}
static void block_hn(Ctx& c, bool fast, double2* G, const double2* A, const double2* B, long long n, int ka, int kb,
                     const char* part_name) {
    if (fast) {
        const int groups = gemm_hn_fp32_groups(n, ka, kb);
        double2* part = c.scratch<double2>(part_name, (size_t)groups * ka * kb);
        launch_gemm_hn_fp32(G, A, B, n, ka, kb, part, groups, c.stream);
        return;
    }
    const int groups = gemm_hn_groups(n, ka, kb);
    double2* part = c.scratch<double2>(part_name, (size_t)groups * ka * kb);
    launch_gemm_hn<double2>(G, A, B, n, ka, kb, part, groups, c.stream);
}
static void block_nn(Ctx& c, bool fast, double2* Y, const double2* X, const double2* W, long long n, int b, int kb) {
    if (fast) launch_gemm_nn_fp32(Y, X, W, (int)n, b, kb, c.stream);
    else launch_gemm_nn<double2>(Y, X, W, (int)n, b, kb, false, c.stream);
}

// Loewdin orthonormalisation X <- X G^{-1/2} (G = X^H X via the Jacobi eigensolver),
// twice: robust for nearly dependent columns, used as the fallback.
static void orthonormalize_loewdin(Ctx& c, double2*& X, double2*& Y, long long n, int b, bool fast) {
    double2* G = c.scratch<double2>("df_G", (size_t)b * b);
    double2* W = c.scratch<double2>("df_W", (size_t)b * b);
    double* lam = c.scratch<double>("df_lamG", b);
    for (int pass = 0; pass < 2; ++pass) {
        block_hn(c, fast, G, X, X, n, b, b, "df_part");
        k_hermitize<<<(b * b + 127) / 128, 128, 0, c.stream>>>(G, b);
        small_launch_check();
        {
            ProfScope ps(c, "setup.jacobi", 0, 0);
            launch_jacobi_eig(G, W, lam, b, 40, c.scratch_bytes("jacobi_work", jacobi_work_bytes(b)),
                              device_error_flag(c), c.stream);
        }
        k_scale_cols_rsqrt<<<(b * b + 127) / 128, 128, 0, c.stream>>>(W, lam, b);
        small_launch_check();
        block_nn(c, fast, Y, X, W, n, b, b);
        std::swap(X, Y);
    }
}

// CholQR2: X <- X R^{-1} with G = X^H X = R^H R, twice; falls back to the
// Loewdin form if a Gram matrix is not numerically positive definite.
static void orthonormalize(Ctx& c, double2*& X, double2*& Y, long long n, int b, bool fast) {
    double2* G = c.scratch<double2>("df_G", (size_t)b * b);
    double2* Ri = c.scratch<double2>("df_Ri", (size_t)b * b);
    int* st = c.scratch<int>("df_st", 4);
    double2* keep = c.scratch<double2>("df_Xkeep", (size_t)n * b);
    MG_CUDA(cudaMemcpyAsync(keep, X, sizeof(double2) * n * b, cudaMemcpyDeviceToDevice, c.stream));
    MG_CUDA(cudaMemsetAsync(st, 0, sizeof(int), c.stream));
    for (int pass = 0; pass < 2; ++pass) {
        block_hn(c, fast, G, X, X, n, b, b, "df_part");
        {
            ProfScope ps(c, "setup.cholqr", 0, 0);
            launch_cholesky_inv(G, Ri, b, c.scratch_bytes("chol_work", cholesky_work_bytes(b)), st,
                                device_error_flag(c), c.stream);
        }
        block_nn(c, fast, Y, X, Ri, n, b, b);
        std::swap(X, Y);
    }
    int hs = 0;
    MG_CUDA(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    if (hs) {
        MG_CUDA(cudaMemcpyAsync(X, keep, sizeof(double2) * n * b, cudaMemcpyDeviceToDevice, c.stream));
        orthonormalize_loewdin(c, X, Y, n, b, fast);
    }
}

// Block of the subspace iteration on level l (per-level names: a coarser level's
// iteration runs while the finer level's block is held).
struct Subspace {
    double2 *X, *Y, *T, *T2, *H, *W;
    double *lam, *res;
};
static Subspace subspace_buffers(Ctx& c, int l, int b) {
    const size_t n = (size_t)c.lev[l].n;
    const std::string sfx = "_" + std::to_string(l);
    Subspace S;
    S.X = c.scratch<double2>("df_X" + sfx, n * b);
    S.Y = c.scratch<double2>("df_Y" + sfx, n * b);
    S.T = c.scratch<double2>("df_T" + sfx, n * b);
    S.T2 = c.scratch<double2>("df_T2" + sfx, n * b);
    S.H = c.scratch<double2>("df_H" + sfx, (size_t)b * b);
    S.W = c.scratch<double2>("df_WR" + sfx, (size_t)b * b);
    S.lam = c.scratch<double>("df_lam" + sfx, b);
    S.res = c.scratch<double>("df_res" + sfx, b);
    return S;
}

// Subspace iteration on Q_l^{-1} = D_l^{-1} Gamma5^l from the orthonormal block S.X
// (FP64-accurate solves to solve_tol), with Rayleigh-Ritz after the first iteration,
// every kRayleighRitzEvery and after the last; stops once every one of the k wanted
// Ritz pairs has ||Q x - lambda x|| <= tol |lambda|.  S.X holds the Ritz vectors (by
// increasing |lambda|) and h_lam their values after the last Rayleigh-Ritz step.
//
// The Rayleigh-Ritz step projects the iterated operator Q^{-1}, not Q: H = X^H Q^{-1} X
// = X^H Y with the block Y = Q^{-1} X the solves just formed.  The wanted pairs (the
// smallest |lambda| of Q) are the extremal ones of Q^{-1}, and extremal Ritz values are
// never spurious.  Q itself is indefinite: on a block that still mixes eigenvectors of
// +lambda and -lambda (a slow gap after the block's last eigenvalue) its Ritz values can
// fall anywhere in the spectral gap around 0, below the wanted ones, and hold the
// iteration there.
static bool subspace_iteration(Ctx& c, int l, int k, int b, double tol, int max_iters, double solve_tol, Subspace& S,
                               std::vector<double>& h_lam) {
    const Level& L = c.lev[l];
    const long long n = L.n;
    const bool fast = fast_block_products(n, b, tol);
    std::vector<double> h_res(b);
    h_lam.assign(b, 0.0);
    bool conv = false;
    for (int it = 0; it < max_iters && !conv; ++it) {
        // Y = Q^{-1} X = D^{-1} Gamma5 X (FP64-accurate solves)
        launch_gamma5<double2>(S.T, S.X, L.nsites, L.d, b, c.stream);
        int ok = 0;
        solve(c, l, S.T, S.Y, b, solve_tol, &ok);
        MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED, "deflation eigensolver: a solve did not converge");
        if (it > 0 && (it + 1) % kRayleighRitzEvery != 0 && it + 1 < max_iters) {
            std::swap(S.X, S.Y);
            orthonormalize(c, S.X, S.Y, n, b, fast);
            continue;
        }
        // Rayleigh-Ritz with Q^{-1} on span(X): Ritz values mu = 1/lambda by decreasing |mu|
        block_hn(c, fast, S.H, S.X, S.Y, n, b, b, "df_partR");
        k_hermitize<<<(b * b + 127) / 128, 128, 0, c.stream>>>(S.H, b);
        small_launch_check();
        {
            ProfScope ps(c, "setup.jacobi", 0, 0);
            launch_jacobi_eig(S.H, S.W, S.lam, b, 40, c.scratch_bytes("jacobi_work", jacobi_work_bytes(b)),
                              device_error_flag(c), c.stream, true);
        }
        k_reciprocal<<<(b + 127) / 128, 128, 0, c.stream>>>(S.lam, b);
        small_launch_check();
        block_nn(c, fast, S.T, S.X, S.W, n, b, b);    // Ritz vectors x = X w
        block_nn(c, fast, S.T2, S.Y, S.W, n, b, b);   // Q^{-1} x: the next block
        // residuals with Q itself: Y = Q x - lambda x
        apply_D<double2>(c, l, S.X, S.T, nullptr, b, 0, nullptr);
        launch_gamma5<double2>(S.X, S.X, L.nsites, L.d, b, c.stream);
        k_resid_cols<<<(unsigned)((n * b + 255) / 256), 256, 0, c.stream>>>(S.Y, S.X, S.T, S.lam, n, b);
        small_launch_check();
        column_norms(c, S.res, S.Y, n, b);
        MG_CUDA(cudaMemcpyAsync(h_lam.data(), S.lam, sizeof(double) * b, cudaMemcpyDeviceToHost, c.stream));
        MG_CUDA(cudaMemcpyAsync(h_res.data(), S.res, sizeof(double) * b, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        check_device_error(c);
        double worst = 0;
        for (int i = 0; i < k; ++i) worst = std::max(worst, h_res[i] / std::fabs(h_lam[i]));
        if (c.opt.verbose)
            fprintf(stderr, "[mgmlmc] deflation level %d it %d worst rel residual %.3e\n", l + 1, it, worst);
        conv = worst <= tol;
        if (conv || it + 1 >= max_iters) {
            std::swap(S.X, S.T);   // the Ritz vectors and their values
        } else {
            std::swap(S.X, S.T2);
            orthonormalize(c, S.X, S.Y, n, b, fast);
        }
    }
    return conv;
}

// Iterations of the eigensolver on a coarser level that only shapes the start block.
constexpr int kCoarseStartIters = 8;

// Orthonormal start block of the subspace iteration on level l.  The coarser level's
// Q_{l+1} = P^H Q_l P is Q_l's Galerkin (Rayleigh-Ritz) projection on range(P), which
// holds the near-kernel the test vectors captured; so, where a coarser level has room
// for the block, its approximate smallest-|lambda| Ritz vectors (a few iterations, the
// same construction one level down) are prolongated; else seeded Z2 noise.
static void subspace_start(Ctx& c, int l, int k, int b, double solve_tol, Subspace& S) {
    const Level& L = c.lev[l];
    if (l + 1 < c.L && c.lev[l + 1].n >= 2LL * b) {
        Subspace Sc = subspace_buffers(c, l + 1, b);
        subspace_start(c, l + 1, k, b, solve_tol, Sc);
        std::vector<double> hl;
        subspace_iteration(c, l + 1, k, b, 1e-2, kCoarseStartIters, std::max(solve_tol, 1e-8), Sc, hl);
        apply_prolong<double2>(c, l, S.X, Sc.X, b, false);
    } else {
        launch_noise<double2>(S.X, L.n, b, 0x2211153830ull, 77 + (uint64_t)l, 0, c.stream);
    }
    orthonormalize(c, S.X, S.Y, L.n, b, fast_block_products(L.n, b, 1.0));
}

void compute_deflation(Ctx& c, int l, int k, double tol, int max_iters, bool inexact, double eig_solve_tol) {
    // The iteration's solves need a few digits beyond its Ritz tolerance, not the
    // estimator's: any vectors leave the estimator unbiased (the deflated trace is taken
    // from the stored factors), their accuracy only sets how much variance is removed,
    // and convergence is judged on residuals of Q itself.
    if (eig_solve_tol <= 0) eig_solve_tol = std::max(c.opt.solve_tol, std::min(1e-6, 1e-3 * tol));
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "compute_deflation: no hierarchy");
    MG_REQUIRE(l >= 0 && l < c.L, MGMLMC_EINVAL, "compute_deflation: bad level");
    free_one_deflation(c, c.defl);
    if (k == 0) return;
    const Level& L = c.lev[l];
    const long long n = L.n;
    MG_REQUIRE(k >= 1 && k <= n && k <= 1024, MGMLMC_EINVAL, "compute_deflation: 0 <= k <= min(n_L, 1024)");
    MG_REQUIRE(tol > 0 && max_iters >= 1, MGMLMC_EINVAL, "compute_deflation: tol > 0 and max_iters >= 1");
    const int b = (int)std::min<long long>(n, std::max(2 * k, k + 16));
    // the eigensolver's blocks are not needed once the triplets are stored
    struct FreeBlocks {
        Ctx& c;
        ~FreeBlocks() {
            try {
                c.free_scratch({"df_", "jacobi_work", "chol_work", "sv_chunk_"});
            } catch (...) {
            }
        }
    } free_blocks{c};
    Subspace S = subspace_buffers(c, l, b);
    subspace_start(c, l, k, b, eig_solve_tol, S);
    std::vector<double> h_lam;
    const bool conv = subspace_iteration(c, l, k, b, tol, max_iters, eig_solve_tol, S, h_lam);
    double2* X = S.X;
    double2* T = S.T;
    double* lam = S.lam;
    if (inexact) {
        // orthogonal projector on U = Gamma5 X (Sect. 2's Pi = U U^H) with the deflated
        // part recomputed from the approximate vectors by k extra solves
        double2* R = c.scratch<double2>("df_Rin", (size_t)n * k);
        launch_gamma5<double2>(T, X, L.nsites, L.d, b, c.stream);
        MG_CUDA(cudaMemcpy2DAsync(R, sizeof(double2) * k, T, sizeof(double2) * b, sizeof(double2) * k, n,
                                  cudaMemcpyDeviceToDevice, c.stream));
        set_deflation_vectors(c, l, -1, R, k);
        c.defl.lambda.assign(h_lam.begin(), h_lam.begin() + k);
        c.defl.inexact = true;
        if (!conv) throw Error(MGMLMC_ENOTCONVERGED, "compute_deflation: eigensolver did not reach tol (results kept)");
        return;
    }
    // store V = X_k, U = Gamma5 X_k sign(lambda), a = 1/|lambda|
    c.defl.k = k;
    c.defl.fine = l;
    c.defl.Lv = c.alloc_n<double2>((size_t)n * k);
    c.defl.Rv = c.alloc_n<double2>((size_t)n * k);
    c.defl.a = c.alloc_n<double>(k);
    MG_CUDA(cudaMemcpy2DAsync(c.defl.Lv, sizeof(double2) * k, X, sizeof(double2) * b, sizeof(double2) * k, n,
                              cudaMemcpyDeviceToDevice, c.stream));
    launch_gamma5<double2>(T, X, L.nsites, L.d, b, c.stream);
    k_sign_cols<<<(unsigned)((n * b + 255) / 256), 256, 0, c.stream>>>(T, lam, n, b);
    small_launch_check();
    MG_CUDA(cudaMemcpy2DAsync(c.defl.Rv, sizeof(double2) * k, T, sizeof(double2) * b, sizeof(double2) * k, n,
                              cudaMemcpyDeviceToDevice, c.stream));
    k_inv_abs<<<(k + 127) / 128, 128, 0, c.stream>>>(c.defl.a, lam, k);
    small_launch_check();
    // tau = sum_i a_i u_i^H v_i  (Eq. small_trace_term), FP64 from the stored factors
    double2* t = c.scratch<double2>("df_t", k);
    double2* tau = c.scratch<double2>("df_tau", 1);
    double2* dpart = c.scratch<double2>("df_dpart", (size_t)reduce_groups(n, k) * k);
    launch_dot<double2, double2>(t, c.defl.Rv, c.defl.Lv, n, k, dpart, c.stream);
    k_weighted_sum<<<1, 1, 0, c.stream>>>(tau, t, c.defl.a, k);
    small_launch_check();
    double2 htau;
    MG_CUDA(cudaMemcpyAsync(&htau, tau, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    c.defl.tau_re = htau.x;
    c.defl.tau_im = htau.y;
    c.defl.lambda.assign(h_lam.begin(), h_lam.begin() + k);
    prepare_tc_deflation(c, c.defl);
    if (!conv) throw Error(MGMLMC_ENOTCONVERGED, "compute_deflation: eigensolver did not reach tol (results kept)");
}

}  // namespace mg

namespace mg {

// Y = J X = D_a^{-1} Gamma5^a X - P D_b^{-1} Gamma5^b P^H X  (FP64-accurate solves)
static void apply_J(Ctx& c, int a, int b, const double2* X, double2* Y, int nb, double tol) {
    const Level& La = c.lev[a];
    double2* T = c.scratch<double2>("dd_T", (size_t)La.n * nb);
    int ok = 0;
    launch_gamma5<double2>(T, X, La.nsites, La.d, nb, c.stream);
    solve(c, a, T, Y, nb, tol, &ok);
    MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED, "difference deflation: solve on the fine level did not converge");
    const double2* cur = X;
    for (int l = a; l < b; ++l) {
        double2* nx = c.scratch<double2>("dd_R" + std::to_string(l + 1), (size_t)c.lev[l + 1].n * nb);
        apply_restrict<double2>(c, l, nx, cur, nb);
        cur = nx;
    }
    const Level& Lb = c.lev[b];
    double2* Tb = c.scratch<double2>("dd_Tb", (size_t)Lb.n * nb);
    double2* Zb = c.scratch<double2>("dd_Zb", (size_t)Lb.n * nb);
    launch_gamma5<double2>(Tb, cur, Lb.nsites, Lb.d, nb, c.stream);
    solve(c, b, Tb, Zb, nb, tol, &ok);
    MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED, "difference deflation: solve on the coarse level did not converge");
    // prolongate back to level a and subtract
    const double2* up = Zb;
    for (int l = b - 1; l >= a; --l) {
        double2* px = c.scratch<double2>("dd_P" + std::to_string(l), (size_t)c.lev[l].n * nb);
        apply_prolong<double2>(c, l, px, up, nb, false);
        up = px;
    }
    launch_axpy_rhs<double2, double2>(Y, nullptr, nullptr, -1.0, up, La.n, nb, c.stream);
}

void compute_difference_deflation(Ctx& c, int a, int b, int k, double tol, int max_iters, bool inexact,
                                  double eig_solve_tol) {
    if (eig_solve_tol <= 0) eig_solve_tol = c.opt.solve_tol;
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "difference deflation: no hierarchy");
    MG_REQUIRE(a >= 0 && b > a && b < c.L, MGMLMC_EINVAL, "difference deflation: bad term");
    Deflation& D = c.ddefl[a];
    free_one_deflation(c, D);
    if (k == 0) return;
    const Level& La = c.lev[a];
    const long long n = La.n;
    MG_REQUIRE(k >= 1 && k <= n && k <= 512, MGMLMC_EINVAL, "difference deflation: 0 <= k <= min(n_a, 512)");
    MG_REQUIRE(tol > 0 && max_iters >= 1, MGMLMC_EINVAL, "difference deflation: tol > 0 and max_iters >= 1");
    const int nb = (int)std::min<long long>(n, std::max(2 * k, k + 16));
    double2* X = c.scratch<double2>("dd_X", (size_t)n * nb);
    double2* Y = c.scratch<double2>("dd_Y", (size_t)n * nb);
    double2* Xr = c.scratch<double2>("dd_Xr", (size_t)n * nb);
    double2* Yr = c.scratch<double2>("dd_Yr", (size_t)n * nb);
    double2* H = c.scratch<double2>("dd_H", (size_t)nb * nb);
    double2* W = c.scratch<double2>("dd_W", (size_t)nb * nb);
    double* lam = c.scratch<double>("dd_lam", nb);
    double* res = c.scratch<double>("dd_res", nb);
    const bool fast = fast_block_products(n, nb, tol);
    launch_noise<double2>(X, n, nb, 0x2211153831ull, 78 + a, 0, c.stream);
    orthonormalize(c, X, Y, n, nb, fast);
    std::vector<double> h_lam(nb), h_res(nb);
    bool conv = false;
    for (int it = 0; it < max_iters && !conv; ++it) {
        apply_J(c, a, b, X, Y, nb, eig_solve_tol);
        if ((it + 1) % kRayleighRitzEvery != 0 && it + 1 < max_iters) {
            std::swap(X, Y);               // X <- J X, orthonormalised
            orthonormalize(c, X, Y, n, nb, fast);
            continue;
        }
        // Rayleigh-Ritz on span(X): H = X^H J X, largest |lambda| first
        block_hn(c, fast, H, X, Y, n, nb, nb, "dd_part");
        k_hermitize<<<(nb * nb + 127) / 128, 128, 0, c.stream>>>(H, nb);
        small_launch_check();
        {
            ProfScope ps(c, "setup.jacobi", 0, 0);
            launch_jacobi_eig(H, W, lam, nb, 40, c.scratch_bytes("jacobi_work", jacobi_work_bytes(nb)),
                              device_error_flag(c), c.stream, true);
        }
        block_nn(c, fast, Xr, X, W, n, nb, nb);
        block_nn(c, fast, Yr, Y, W, n, nb, nb);
        k_resid_cols<<<(unsigned)((n * nb + 255) / 256), 256, 0, c.stream>>>(Y, Yr, Xr, lam, n, nb);
        small_launch_check();
        column_norms(c, res, Y, n, nb);
        MG_CUDA(cudaMemcpyAsync(h_lam.data(), lam, sizeof(double) * nb, cudaMemcpyDeviceToHost, c.stream));
        MG_CUDA(cudaMemcpyAsync(h_res.data(), res, sizeof(double) * nb, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        check_device_error(c);
        double worst = 0;
        for (int i = 0; i < k; ++i) worst = std::max(worst, h_res[i] / std::fabs(h_lam[i]));
        if (c.opt.verbose) fprintf(stderr, "[mgmlmc] difference deflation level %d it %d worst rel residual %.3e\n",
                                   a + 1, it, worst);
        conv = worst <= tol;
        if (conv) {
            std::swap(X, Xr);          // X = Ritz vectors
            break;
        }
        // next iterate: J applied to the Ritz vectors, orthonormalised
        std::swap(X, Yr);
        orthonormalize(c, X, Y, n, nb, fast);
    }
    if (!conv) {
        // the last Ritz vectors are the best available
        std::swap(X, Xr);
    }
    if (inexact) {
        // orthogonal projector on V = Gamma5^a X, deflated part recomputed from the
        // approximate vectors by k extra applications of M
        double2* R = c.scratch<double2>("dd_Rin", (size_t)n * k);
        double2* T0 = c.scratch<double2>("dd_T2", (size_t)n * nb);
        launch_gamma5<double2>(T0, X, La.nsites, La.d, nb, c.stream);
        MG_CUDA(cudaMemcpy2DAsync(R, sizeof(double2) * k, T0, sizeof(double2) * nb, sizeof(double2) * k, n,
                                  cudaMemcpyDeviceToDevice, c.stream));
        set_deflation_vectors(c, a, b, R, k);
        c.ddefl[a].lambda.assign(h_lam.begin(), h_lam.begin() + k);
        c.ddefl[a].inexact = true;
        if (!conv) throw Error(MGMLMC_ENOTCONVERGED, "difference deflation: eigensolver did not reach tol (results kept)");
        return;
    }
    // U = X sign(lambda) (left, L), V = Gamma5^a X (right, R), a = |lambda|
    D.k = k;
    D.fine = a;
    D.coarse = b;
    D.Lv = c.alloc_n<double2>((size_t)n * k);
    D.Rv = c.alloc_n<double2>((size_t)n * k);
    D.a = c.alloc_n<double>(k);
    double2* T = c.scratch<double2>("dd_T2", (size_t)n * nb);
    MG_CUDA(cudaMemcpyAsync(T, X, sizeof(double2) * n * nb, cudaMemcpyDeviceToDevice, c.stream));
    k_sign_cols<<<(unsigned)((n * nb + 255) / 256), 256, 0, c.stream>>>(T, lam, n, nb);
    small_launch_check();
    MG_CUDA(cudaMemcpy2DAsync(D.Lv, sizeof(double2) * k, T, sizeof(double2) * nb, sizeof(double2) * k, n,
                              cudaMemcpyDeviceToDevice, c.stream));
    launch_gamma5<double2>(T, X, La.nsites, La.d, nb, c.stream);
    MG_CUDA(cudaMemcpy2DAsync(D.Rv, sizeof(double2) * k, T, sizeof(double2) * nb, sizeof(double2) * k, n,
                              cudaMemcpyDeviceToDevice, c.stream));
    k_abs<<<(k + 127) / 128, 128, 0, c.stream>>>(D.a, lam, k);
    small_launch_check();
    double2* t = c.scratch<double2>("dd_t", k);
    double2* tau = c.scratch<double2>("dd_tau", 1);
    double2* dpart = c.scratch<double2>("dd_dpart", (size_t)reduce_groups(n, k) * k);
    launch_dot<double2, double2>(t, D.Rv, D.Lv, n, k, dpart, c.stream);
    k_weighted_sum<<<1, 1, 0, c.stream>>>(tau, t, D.a, k);
    small_launch_check();
    double2 htau;
    MG_CUDA(cudaMemcpyAsync(&htau, tau, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    D.tau_re = htau.x;
    D.tau_im = htau.y;
    D.lambda.assign(h_lam.begin(), h_lam.begin() + k);
    prepare_tc_deflation(c, D);
    if (!conv) throw Error(MGMLMC_ENOTCONVERGED, "difference deflation: eigensolver did not reach tol (results kept)");
}

}  // namespace mg

namespace mg {

// Y = A X for the traced operator of term (a, b): D_a^{-1} X - P D_b^{-1} P^H X,
// or D_a^{-1} X for the last term (b < 0).  FP64-accurate solves.
static void apply_traced(Ctx& c, int a, int b, const double2* X, double2* Y, int nb) {
    int ok = 0;
    solve(c, a, X, Y, nb, c.opt.solve_tol, &ok);
    MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED, "deflation: solve on the fine level did not converge");
    if (b < 0) return;
    const double2* cur = X;
    for (int l = a; l < b; ++l) {
        double2* nx = c.scratch<double2>("at_R" + std::to_string(l + 1), (size_t)c.lev[l + 1].n * nb);
        apply_restrict<double2>(c, l, nx, cur, nb);
        cur = nx;
    }
    double2* Zb = c.scratch<double2>("at_Zb", (size_t)c.lev[b].n * nb);
    solve(c, b, cur, Zb, nb, c.opt.solve_tol, &ok);
    MG_REQUIRE(ok, MGMLMC_ENOTCONVERGED, "deflation: solve on the coarse level did not converge");
    const double2* up = Zb;
    for (int l = b - 1; l >= a; --l) {
        double2* px = c.scratch<double2>("at_P" + std::to_string(l), (size_t)c.lev[l].n * nb);
        apply_prolong<double2>(c, l, px, up, nb, false);
        up = px;
    }
    launch_axpy_rhs<double2, double2>(Y, nullptr, nullptr, -1.0, up, c.lev[a].n, nb, c.stream);
}

__global__ void k_fill(double* a, double v, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) a[i] = v;
}

void set_deflation_vectors(Ctx& c, int a, int b, const double2* R, int k) {
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "deflation: no hierarchy");
    MG_REQUIRE(a >= 0 && a < c.L && (b < 0 || (b > a && b < c.L)), MGMLMC_EINVAL, "deflation: bad term");
    const long long n = c.lev[a].n;
    MG_REQUIRE(k >= 1 && k <= n && k <= 4096, MGMLMC_EINVAL, "deflation: 1 <= k <= min(n_a, 4096)");
    Deflation& D = (b < 0) ? c.defl : c.ddefl[a];
    // R may live in scratch that apply_traced reuses: keep a private copy first
    double2* Rv = c.alloc_n<double2>((size_t)n * k);
    MG_CUDA(cudaMemcpyAsync(Rv, R, sizeof(double2) * n * k, cudaMemcpyDeviceToDevice, c.stream));
    double2* Lv = c.alloc_n<double2>((size_t)n * k);
    apply_traced(c, a, b, Rv, Lv, k);
    free_one_deflation(c, D);
    D.k = k;
    D.fine = a;
    D.coarse = b;
    D.Lv = Lv;
    D.Rv = Rv;
    D.a = c.alloc_n<double>(k);
    k_fill<<<(k + 127) / 128, 128, 0, c.stream>>>(D.a, 1.0, k);
    small_launch_check();
    // tau = sum_i r_i^H l_i = tr(R^H A R)
    double2* t = c.scratch<double2>("sv_t", k);
    double2* tau = c.scratch<double2>("sv_tau", 1);
    double2* dpart = c.scratch<double2>("sv_dpart", (size_t)reduce_groups(n, k) * k);
    launch_dot<double2, double2>(t, D.Rv, D.Lv, n, k, dpart, c.stream);
    k_weighted_sum<<<1, 1, 0, c.stream>>>(tau, t, D.a, k);
    small_launch_check();
    double2 htau;
    MG_CUDA(cudaMemcpyAsync(&htau, tau, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    D.tau_re = htau.x;
    D.tau_im = htau.y;
    D.inexact = true;
    D.lambda.assign(k, 0.0);
    prepare_tc_deflation(c, D);
}

}  // namespace mg
