// C ABI entry points (declared and documented in include/mgmlmc.h).  Every
// entry catches all exceptions and turns them into a status code.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "context.h"
#include "footprint.h"

using mg::Ctx;
using mg::Error;

#define API_BEGIN(ctxp)                          \
    if (!(ctxp)) return MGMLMC_EINVAL;           \
    Ctx& c = (ctxp)->c;                          \
    c.err.clear();                               \
    try {
#define API_END                                                  \
    }                                                            \
    catch (const Error& e) {                                     \
        c.err = e.what();                                        \
        return e.code;                                           \
    }                                                            \
    catch (const std::bad_alloc&) {                              \
        c.err = "host allocation failed";                        \
        return MGMLMC_ENOMEM;                                    \
    }                                                            \
    catch (const std::exception& e) {                            \
        c.err = e.what();                                        \
        return MGMLMC_ECUDA;                                     \
    }                                                            \
    return MGMLMC_OK;

namespace mg {

void check_options(const mgmlmc_options& o) {
    MG_REQUIRE(o.mg_precision == 64 || o.mg_precision == 32 || o.mg_precision == 16, MGMLMC_EINVAL,
               "options: mg_precision must be 64, 32 or 16");
    MG_REQUIRE(o.solve_tol > 0 && o.solve_tol < 1, MGMLMC_EINVAL, "options: 0 < solve_tol < 1");
    MG_REQUIRE(o.fgmres_restart >= 1 && o.fgmres_restart <= 63, MGMLMC_EINVAL, "options: 1 <= fgmres_restart <= 63");
    MG_REQUIRE(o.max_iters >= 1, MGMLMC_EINVAL, "options: max_iters >= 1");
    MG_REQUIRE(o.nu_pre >= 0 && o.nu_post >= 0 && o.nu_pre + o.nu_post <= 64, MGMLMC_EINVAL,
               "options: smoothing steps");
    MG_REQUIRE(o.max_block_rhs >= 1 && o.max_block_rhs <= 4096, MGMLMC_EINVAL, "options: 1 <= max_block_rhs <= 4096");
    MG_REQUIRE(o.kcycle_iters >= 0 && o.kcycle_iters <= 16, MGMLMC_EINVAL, "options: 0 <= kcycle_iters <= 16");
}

}  // namespace mg

using mg::check_options;

namespace {

void require_level(const Ctx& c, int level) {
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "no hierarchy: call mgmlmc_set_hierarchy first");
    MG_REQUIRE(level >= 1 && level <= c.L, MGMLMC_EINVAL, "level out of range");
}

struct TermLevels {
    int a, b;          // 0-based fine / coarse level; b = -1 for the last term
    const mg::Deflation* defl;   // exact deflation of this term, if computed
};

TermLevels term_levels(const Ctx& c, int t) {
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "no hierarchy: call mgmlmc_set_hierarchy first");
    MG_REQUIRE(t >= 0 && t < c.nterms, MGMLMC_EINVAL, "term out of range");
    TermLevels tl;
    tl.a = c.term_level[t];
    tl.b = (t + 1 < c.nterms) ? c.term_level[t + 1] : -1;
    tl.defl = mg::term_deflation(c, tl.a, tl.b);
    return tl;
}

// Samples of one block: smp[j] = x_j^H D_a^{-1} x_j - (P^H x_j)^H D_b^{-1} (P^H x_j) [- deflated part].
bool run_term_block(Ctx& c, const TermLevels& tl, const double2* X, int Nb, double2* smp, long long* iters) {
    const mg::Level& La = c.lev[tl.a];
    const double tol = c.opt.solve_tol;
    struct Fp32Residuals {
        Ctx& c;
        bool keep;
        ~Fp32Residuals() { c.fp32_residual_updates = keep; }
    } fp32_residuals{c, c.fp32_residual_updates};
    c.fp32_residual_updates = true;
    bool all_ok = true;
    int ok = 0;
    double2* Z = c.scratch<double2>("est_Z", (size_t)La.n * Nb);
    *iters += mg::solve(c, tl.a, X, Z, Nb, tol, &ok);
    all_ok &= ok != 0;
    double2* part = c.scratch<double2>("est_part", (size_t)mg::reduce_groups(La.n, Nb) * Nb);
    mg::launch_dot<double2, double2>(smp, X, Z, La.n, Nb, part, c.stream);
    if (tl.b >= 0) {
        const double2* Ycur = X;
        for (int l = tl.a; l < tl.b; ++l) {
            double2* Yn = c.scratch<double2>("est_Y" + std::to_string(l + 1), (size_t)c.lev[l + 1].n * Nb);
            mg::apply_restrict<double2>(c, l, Yn, Ycur, Nb);
            Ycur = Yn;
        }
        const mg::Level& Lb = c.lev[tl.b];
        double2* W = c.scratch<double2>("est_W", (size_t)Lb.n * Nb);
        *iters += mg::solve(c, tl.b, Ycur, W, Nb, tol, &ok);
        all_ok &= ok != 0;
        double2* s2 = c.scratch<double2>("est_s2", Nb);
        double2* part2 = c.scratch<double2>("est_part2", (size_t)mg::reduce_groups(Lb.n, Nb) * Nb);
        mg::launch_dot<double2, double2>(s2, Ycur, W, Lb.n, Nb, part2, c.stream);
        mg::launch_axpy_rhs<double2, double2>(smp, nullptr, nullptr, -1.0, s2, 1, Nb, c.stream);
    }
    if (tl.defl && tl.defl->W16) {
        // tensor cores: BF16 factors, FP32 accumulation; algorithmic traffic = the BF16
        // factors once + the probe block (FP64) once, flops 8 n k N
        const mg::Deflation& D = *tl.defl;
        void* scr = c.scratch_bytes("est_tcd", mg::deflation_bf16_scratch(La.n, D.k, Nb));
        mg::ProfScope ps(c, "defl.bf16", (double)mg::tc_deflation_rows(D.k) * La.n * 2 + (double)La.n * Nb * 16,
                         8.0 * La.n * D.k * Nb);
        mg::launch_deflation_correction_bf16(smp, X, D.W16, D.a, La.n, D.k, Nb, scr, mg::device_error_flag(c),
                                             c.stream);
    } else if (tl.defl) {
        const mg::Deflation& D = *tl.defl;
        const int k = D.k;
        double2* A = c.scratch<double2>("est_A", (size_t)k * Nb);
        double2* B = c.scratch<double2>("est_B", (size_t)k * Nb);
        const int groups = mg::gemm_hn_groups(La.n, k, Nb);
        double2* part3 = c.scratch<double2>("est_part3", (size_t)groups * k * Nb);
        mg::ProfScope ps(c, "defl.f64", 2.0 * La.n * k * 16 + (double)La.n * Nb * 16, 2.0 * 8.0 * La.n * k * Nb);
        mg::launch_gemm_hn<double2>(A, D.Rv, X, La.n, k, Nb, part3, groups, c.stream);
        mg::launch_gemm_hn<double2>(B, D.Lv, X, La.n, k, Nb, part3, groups, c.stream);
        mg::launch_deflation_correction(smp, A, B, D.a, k, Nb, c.stream);
    }
    return all_ok;
}

// Runs nsamples samples of term t with X produced by make_x(off, Nb, X).
template <typename MakeX>
int estimate_term(Ctx& c, int t, int nsamples, double* samples_out, mgmlmc_level_stats* out, MakeX make_x) {
    const TermLevels tl = term_levels(c, t);
    MG_REQUIRE(nsamples >= 0, MGMLMC_EINVAL, "nsamples must be >= 0");
    const mg::Level& La = c.lev[tl.a];
    const int blk = c.opt.max_block_rhs;
    double2* X = c.scratch<double2>("est_X", (size_t)La.n * std::min(blk, std::max(nsamples, 1)));
    double2* smp = c.scratch<double2>("est_smp", (size_t)std::max(nsamples, 1));
    double* acc = c.scratch<double>("est_acc", 4);
    MG_CUDA(cudaMemsetAsync(acc, 0, 4 * sizeof(double), c.stream));
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    MG_CUDA(cudaEventRecord(e0, c.stream));
    long long iters = 0;
    bool ok = true;
    for (int off = 0; off < nsamples; off += blk) {
        const int Nb = std::min(blk, nsamples - off);
        make_x(off, Nb, X);
        ok &= run_term_block(c, tl, X, Nb, smp + off, &iters);
    }
    if (nsamples > 0) mg::launch_sample_stats(acc, smp, nsamples, c.stream);
    MG_CUDA(cudaEventRecord(e1, c.stream));
    double hacc[4] = {0, 0, 0, 0};
    MG_CUDA(cudaMemcpyAsync(hacc, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (samples_out && nsamples > 0)
        MG_CUDA(cudaMemcpyAsync(samples_out, smp, sizeof(double2) * nsamples, cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    float ms = 0;
    MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mg::TermStats& S = c.stats[t];
    S.n += nsamples;
    S.sum_re += hacc[0];
    S.sum_im += hacc[1];
    S.sum_abs2 += hacc[2];
    S.seconds += ms * 1e-3;
    S.iters += iters;
    if (out) {
        out->nsamples = nsamples;
        out->sum_re = hacc[0];
        out->sum_im = hacc[1];
        out->sum_abs2 = hacc[2];
        out->mean_re = nsamples ? hacc[0] / nsamples : 0;
        out->mean_im = nsamples ? hacc[1] / nsamples : 0;
        out->variance = nsamples > 1 ? (hacc[2] - nsamples * (out->mean_re * out->mean_re + out->mean_im * out->mean_im)) /
                                           (nsamples - 1)
                                     : 0;
        out->seconds = ms * 1e-3;
        out->iters = iters;
    }
    if (!ok) throw Error(MGMLMC_ENOTCONVERGED, "a sample solve reached max_iters (samples kept)");
    return MGMLMC_OK;
}

void fill_stats(const mg::TermStats& S, mgmlmc_level_stats* o) {
    o->nsamples = S.n;
    o->sum_re = S.sum_re;
    o->sum_im = S.sum_im;
    o->sum_abs2 = S.sum_abs2;
    o->mean_re = S.n ? S.sum_re / S.n : 0;
    o->mean_im = S.n ? S.sum_im / S.n : 0;
    o->variance = S.n > 1 ? (S.sum_abs2 - S.n * (o->mean_re * o->mean_re + o->mean_im * o->mean_im)) / (S.n - 1) : 0;
    o->seconds = S.seconds;
    o->iters = S.iters;
}

// [nv][n] host complex -> [n][nv] device
double2* upload_block(Ctx& c, const double* host, long long n, int nv, const char* name) {
    double2* tmp = c.scratch<double2>(std::string(name) + "_t", (size_t)n * nv);
    double2* out = c.scratch<double2>(name, (size_t)n * nv);
    MG_CUDA(cudaMemcpyAsync(tmp, host, sizeof(double2) * n * nv, cudaMemcpyHostToDevice, c.stream));
    mg::launch_transpose(out, tmp, nv, (int)n, c.stream);
    return out;
}
void download_block(Ctx& c, double* host, const double2* dev, long long n, int nv, const char* name) {
    double2* tmp = c.scratch<double2>(name, (size_t)n * nv);
    mg::launch_transpose(tmp, dev, n, nv, c.stream);
    MG_CUDA(cudaMemcpyAsync(host, tmp, sizeof(double2) * n * nv, cudaMemcpyDeviceToHost, c.stream));
    c.sync();
}

}  // namespace

extern "C" {

void mgmlmc_default_options(mgmlmc_options* o) {
    if (!o) return;
    o->mg_precision = 64;
    o->solve_tol = 1e-12;
    o->fgmres_restart = 24;
    o->max_iters = 2000;
    o->nu_pre = 0;
    o->nu_post = 4;
    o->max_block_rhs = 256;
    o->verbose = 0;
    o->kcycle_iters = 0;
}

int mgmlmc_create(mgmlmc_ctx** out, const mgmlmc_options* opt, void* cuda_stream, mgmlmc_alloc_fn alloc,
                  mgmlmc_free_fn free_fn, void* alloc_user) {
    if (!out) return MGMLMC_EINVAL;
    *out = nullptr;
    mgmlmc_ctx* h = new (std::nothrow) mgmlmc_ctx();
    if (!h) return MGMLMC_ENOMEM;
    Ctx& c = h->c;
    try {
        mgmlmc_default_options(&c.opt);
        if (opt) c.opt = *opt;
        check_options(c.opt);
        MG_REQUIRE((alloc == nullptr) == (free_fn == nullptr), MGMLMC_EINVAL, "alloc and free must both be given");
        c.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
        c.alloc = alloc;
        c.free_fn = free_fn;
        c.alloc_user = alloc_user;
        int dev = 0;
        MG_CUDA(cudaGetDevice(&dev));
        c.hbuf_bytes = 4096;
        MG_CUDA(cudaMallocHost(reinterpret_cast<void**>(&c.hbuf), c.hbuf_bytes));
    } catch (const Error& e) {
        const int code = e.code;
        if (c.hbuf) cudaFreeHost(c.hbuf);
        delete h;
        return code;
    }
    *out = h;
    return MGMLMC_OK;
}

int mgmlmc_create_copy(mgmlmc_ctx** out, mgmlmc_ctx* src, void* cuda_stream, mgmlmc_alloc_fn alloc,
                       mgmlmc_free_fn free_fn, void* alloc_user) {
    if (!out || !src) return MGMLMC_EINVAL;
    *out = nullptr;
    mgmlmc_ctx* h = nullptr;
    const int rc = mgmlmc_create(&h, &src->c.opt, cuda_stream, alloc, free_fn, alloc_user);
    if (rc != MGMLMC_OK) return rc;
    Ctx& c = h->c;
    try {
        mg::copy_state(c, src->c);
    } catch (const Error& e) {
        const int code = e.code;
        src->c.err = std::string("create_copy: ") + e.what();
        mgmlmc_destroy(h);
        return code;
    }
    *out = h;
    return MGMLMC_OK;
}

void mgmlmc_destroy(mgmlmc_ctx* h) {
    if (!h) return;
    h->c.release_all();
    if (h->c.hbuf) cudaFreeHost(h->c.hbuf);
    delete h;
}

const char* mgmlmc_last_error(const mgmlmc_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

int mgmlmc_set_options(mgmlmc_ctx* h, const mgmlmc_options* opt) {
    API_BEGIN(h)
    MG_REQUIRE(opt, MGMLMC_EINVAL, "set_options: opt is NULL");
    check_options(*opt);
    MG_REQUIRE(opt->mg_precision == c.opt.mg_precision, MGMLMC_EINVAL,
               "set_options: mg_precision is fixed for the life of a context");
    c.opt = *opt;
    API_END
}

int mgmlmc_set_gauge(mgmlmc_ctx* h, int Lx, int Lt, const double* theta) {
    API_BEGIN(h)
    MG_REQUIRE(theta, MGMLMC_EINVAL, "set_gauge: theta is NULL");
    MG_REQUIRE(Lx >= 2 && Lt >= 2 && Lx % 2 == 0 && Lt % 2 == 0 && (long long)Lx * Lt <= (1LL << 26), MGMLMC_EINVAL,
               "set_gauge: Lx, Lt even, >= 2, Lx*Lt <= 2^26");
    c.free_hierarchy();
    c.have_gauge = false;
    c.Lx = Lx;
    c.Lt = Lt;
    mg::upload_links(c, theta);
    c.have_gauge = true;
    API_END
}

int mgmlmc_set_mass(mgmlmc_ctx* h, double m0) {
    API_BEGIN(h)
    MG_REQUIRE(std::isfinite(m0), MGMLMC_ENAN, "set_mass: non-finite m0");
    c.free_hierarchy();
    c.m0 = m0;
    c.have_mass = true;
    API_END
}

int mgmlmc_set_hierarchy(mgmlmc_ctx* h, int nlevels, const int* agg_x, const int* agg_t, const int* nvec,
                         int setup_iters, double setup_tol, const double* const* start_vectors) {
    API_BEGIN(h)
    MG_REQUIRE(setup_tol > 0 && setup_tol < 1, MGMLMC_EINVAL, "set_hierarchy: 0 < setup_tol < 1");
    mg::build_hierarchy(c, nlevels, agg_x, agg_t, nvec, setup_iters, setup_tol, start_vectors);
    API_END
}

int mgmlmc_set_terms(mgmlmc_ctx* h, int nskip, const int* skip) {
    API_BEGIN(h)
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "set_terms: no hierarchy");
    MG_REQUIRE(nskip >= 0 && (nskip == 0 || skip), MGMLMC_EINVAL, "set_terms: bad skip list");
    std::vector<int> sk(skip, skip + nskip);
    for (int s : sk)
        MG_REQUIRE(s >= 2 && s <= c.L, MGMLMC_EINVAL, "set_terms: only levels 2..L can be skipped");
    c.nterms = 0;
    for (int l = 0; l < c.L; ++l)
        if (std::find(sk.begin(), sk.end(), l + 1) == sk.end()) c.term_level[c.nterms++] = l;
    c.skip = sk;
    for (auto& s : c.stats) s = mg::TermStats();
    API_END
}

int mgmlmc_num_terms(const mgmlmc_ctx* h, int* nterms, int* term_level) {
    if (!h || !nterms) return MGMLMC_EINVAL;
    const Ctx& c = h->c;
    if (!c.have_hier) return MGMLMC_ESTATE;
    *nterms = c.nterms;
    if (term_level)
        for (int t = 0; t < c.nterms; ++t) term_level[t] = c.term_level[t] + 1;
    return MGMLMC_OK;
}

int mgmlmc_compute_deflation(mgmlmc_ctx* h, int k, double tol, int max_iters) {
    API_BEGIN(h)
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "compute_deflation: no hierarchy");
    mg::compute_deflation(c, c.term_level[c.nterms - 1], k, tol, max_iters);
    API_END
}

int mgmlmc_compute_term_deflation(mgmlmc_ctx* h, int term, int k, double tol, int max_iters) {
    API_BEGIN(h)
    const TermLevels tl = term_levels(c, term);
    if (tl.b < 0) mg::compute_deflation(c, tl.a, k, tol, max_iters);
    else mg::compute_difference_deflation(c, tl.a, tl.b, k, tol, max_iters);
    API_END
}

int mgmlmc_compute_term_deflation_inexact(mgmlmc_ctx* h, int term, int k, double eig_tol, double inner_tol,
                                          int max_iters) {
    API_BEGIN(h)
    MG_REQUIRE(inner_tol > 0 && inner_tol < 1, MGMLMC_EINVAL, "inexact deflation: 0 < inner_tol < 1");
    const TermLevels tl = term_levels(c, term);
    // eigensolver solves at inner_tol; the k extra solves of the deflated part at solve_tol
    if (tl.b < 0) mg::compute_deflation(c, tl.a, k, eig_tol, max_iters, true, inner_tol);
    else mg::compute_difference_deflation(c, tl.a, tl.b, k, eig_tol, max_iters, true, inner_tol);
    API_END
}

int mgmlmc_set_term_deflation_vectors(mgmlmc_ctx* h, int term, int k, const double* V) {
    API_BEGIN(h)
    MG_REQUIRE(V, MGMLMC_EINVAL, "set_term_deflation_vectors: V is NULL");
    const TermLevels tl = term_levels(c, term);
    const long long n = c.lev[tl.a].n;
    MG_REQUIRE(k >= 1 && k <= n, MGMLMC_EINVAL, "set_term_deflation_vectors: 1 <= k <= n_a");
    double2* R = upload_block(c, V, n, k, "stdv_R");
    mg::set_deflation_vectors(c, tl.a, tl.b, R, k);
    API_END
}

int mgmlmc_get_term_deflation(mgmlmc_ctx* h, int term, int* k, double* lambda, double* L, double* R, double* tau) {
    API_BEGIN(h)
    const TermLevels tl = term_levels(c, term);
    MG_REQUIRE(tl.defl, MGMLMC_ESTATE, "get_term_deflation: this term has no deflation");
    const mg::Deflation& D = *tl.defl;
    const long long n = c.lev[tl.a].n;
    if (k) *k = D.k;
    if (lambda)
        for (int i = 0; i < D.k; ++i) lambda[i] = i < (int)D.lambda.size() ? D.lambda[i] : 0.0;
    if (L) download_block(c, L, D.Lv, n, D.k, "gd_tmp");
    if (R) download_block(c, R, D.Rv, n, D.k, "gd_tmp");
    if (tau) {
        tau[0] = D.tau_re;
        tau[1] = D.tau_im;
    }
    API_END
}

int mgmlmc_term_deflated_part(mgmlmc_ctx* h, int term, double* tau) {
    API_BEGIN(h)
    MG_REQUIRE(tau, MGMLMC_EINVAL, "term_deflated_part: tau is NULL");
    const TermLevels tl = term_levels(c, term);
    tau[0] = tl.defl ? tl.defl->tau_used_re() : 0.0;
    tau[1] = tl.defl ? tl.defl->tau_used_im() : 0.0;
    API_END
}

int mgmlmc_get_deflation(mgmlmc_ctx* h, double* lambda, double* sigma, double* U, double* V, double* tau) {
    API_BEGIN(h)
    const int k = c.defl.k;
    MG_REQUIRE(k > 0, MGMLMC_ESTATE, "get_deflation: no deflation computed");
    const long long n = c.lev[c.defl.fine].n;   // the level of the last term (the coarsest unless skipped)
    for (int i = 0; i < k; ++i) {
        const double li = i < (int)c.defl.lambda.size() ? c.defl.lambda[i] : 0.0;
        if (lambda) lambda[i] = li;
        if (sigma) sigma[i] = std::fabs(li);
    }
    if (U) download_block(c, U, c.defl.Rv, n, k, "gd_tmp");
    if (V) download_block(c, V, c.defl.Lv, n, k, "gd_tmp");
    if (tau) {
        tau[0] = c.defl.tau_re;
        tau[1] = c.defl.tau_im;
    }
    API_END
}

int mgmlmc_estimate_level(mgmlmc_ctx* h, int term, int64_t first_sample, int nsamples, uint64_t seed,
                          double* samples_out, mgmlmc_level_stats* stats) {
    API_BEGIN(h)
    MG_REQUIRE(first_sample >= 0, MGMLMC_EINVAL, "first_sample must be >= 0");
    const TermLevels tl = term_levels(c, term);
    const long long n = c.lev[tl.a].n;
    estimate_term(c, term, nsamples, samples_out, stats, [&](int off, int Nb, double2* X) {
        mg::launch_noise<double2>(X, n, Nb, seed, (uint64_t)(tl.a + 1), first_sample + off, c.stream);
    });
    API_END
}

int mgmlmc_estimate_level_probes(mgmlmc_ctx* h, int term, int nsamples, const int8_t* probes, double* samples_out,
                                 mgmlmc_level_stats* stats) {
    API_BEGIN(h)
    MG_REQUIRE(probes || nsamples == 0, MGMLMC_EINVAL, "probes is NULL");
    const TermLevels tl = term_levels(c, term);
    const long long n = c.lev[tl.a].n;
    const int blk = c.opt.max_block_rhs;
    int8_t* dp = c.scratch<int8_t>("probes", (size_t)n * std::min(blk, std::max(nsamples, 1)));
    estimate_term(c, term, nsamples, samples_out, stats, [&](int off, int Nb, double2* X) {
        MG_CUDA(cudaMemcpyAsync(dp, probes + (size_t)off * n, (size_t)Nb * n, cudaMemcpyHostToDevice, c.stream));
        mg::launch_probes<double2>(X, dp, n, Nb, c.stream);
    });
    API_END
}

int mgmlmc_estimate_concurrent(mgmlmc_ctx* const* contexts, int n, const int* terms, int64_t first_sample,
                               int nsamples, uint64_t seed, const int8_t* const* probes, double* const* samples_out,
                               mgmlmc_level_stats* stats) {
    if (!contexts || !terms || n < 1 || n > 64) return MGMLMC_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!contexts[i]) return MGMLMC_EINVAL;
        for (int k = 0; k < i; ++k)
            if (contexts[k] == contexts[i]) return MGMLMC_EINVAL;   // one host thread per context
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MGMLMC_ECUDA;
    std::vector<int> rc(n, MGMLMC_OK);
    auto run = [&](int i) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            rc[i] = MGMLMC_ECUDA;
            return;
        }
        double* out = samples_out ? samples_out[i] : nullptr;
        mgmlmc_level_stats* st = stats ? stats + i : nullptr;
        rc[i] = (probes && probes[i])
                    ? mgmlmc_estimate_level_probes(contexts[i], terms[i], nsamples, probes[i], out, st)
                    : mgmlmc_estimate_level(contexts[i], terms[i], first_sample, nsamples, seed, out, st);
    };
    std::vector<std::thread> pool;
    try {
        for (int i = 1; i < n; ++i) pool.emplace_back(run, i);
    } catch (...) {
        for (auto& t : pool) t.join();
        return MGMLMC_ENOMEM;
    }
    run(0);
    for (auto& t : pool) t.join();
    for (int i = 0; i < n; ++i)
        if (rc[i] != MGMLMC_OK) return rc[i];
    return MGMLMC_OK;
}

int mgmlmc_get_stats(mgmlmc_ctx* h, int term, mgmlmc_level_stats* stats) {
    API_BEGIN(h)
    MG_REQUIRE(stats && term >= 0 && term < MGMLMC_MAX_LEVELS, MGMLMC_EINVAL, "get_stats: bad argument");
    fill_stats(c.stats[term], stats);
    API_END
}

int mgmlmc_reset_stats(mgmlmc_ctx* h) {
    API_BEGIN(h)
    for (auto& s : c.stats) s = mg::TermStats();
    API_END
}

}  // extern "C"

namespace mg {

// The MLMC loop (Sect. 3.2 with the cited allocation rule): term t draws its samples
// on ctx_of[t]; with `concurrent` the draws of one round run on one host thread per
// term (the contexts are then distinct, each on its own stream).
void mlmc_loop(const std::vector<Ctx*>& ctx_of, bool concurrent, double rel_tol, int64_t max_samples, uint64_t seed,
               const double* costs, mgmlmc_trace_result* out, const std::atomic<bool>* cancel) {
    auto check_cancel = [&] {
        if (cancel && cancel->load()) throw Error(MGMLMC_ECANCELLED, "estimate_trace: cancelled");
    };
    MG_REQUIRE(out && rel_tol > 0 && max_samples > 0, MGMLMC_EINVAL, "estimate_trace: bad argument");
    const int T = ctx_of[0]->nterms;
    for (Ctx* ct : ctx_of) {
        MG_REQUIRE(ct->have_hier, MGMLMC_ESTATE, "estimate_trace: no hierarchy");
        MG_REQUIRE(ct->nterms == T, MGMLMC_EINVAL, "estimate_trace: contexts with different term lists");
        for (auto& st : ct->stats) st = mg::TermStats();
    }
    const int pilot = 16;
    auto draw = [&](int t, long long first, long long count) {
        Ctx& ct = *ctx_of[t];
        while (count > 0) {
            const int cnt = (int)std::min<long long>(count, 1 << 20);
            const TermLevels tl = term_levels(ct, t);
            const long long n = ct.lev[tl.a].n;
            estimate_term(ct, t, cnt, nullptr, nullptr, [&](int off, int Nb, double2* X) {
                mg::launch_noise<double2>(X, n, Nb, seed, (uint64_t)(tl.a + 1), first + off, ct.stream);
            });
            first += cnt;
            count -= cnt;
        }
    };
    // one round of draws: [first, first + count) of term t for every t with count > 0
    auto round = [&](const std::vector<long long>& first, const std::vector<long long>& count) {
        if (!concurrent) {
            for (int t = 0; t < T; ++t)
                if (count[t] > 0) draw(t, first[t], count[t]);
            return;
        }
        int dev = 0;
        MG_CUDA(cudaGetDevice(&dev));
        std::vector<int> code(T, MGMLMC_OK);
        std::vector<std::string> msg(T);
        auto run = [&](int t) {
            try {
                MG_CUDA(cudaSetDevice(dev));
                draw(t, first[t], count[t]);
            } catch (const Error& e) {
                code[t] = e.code;
                msg[t] = e.what();
            } catch (const std::exception& e) {
                code[t] = MGMLMC_ECUDA;
                msg[t] = e.what();
            }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < T; ++t)
            if (count[t] > 0) pool.emplace_back(run, t);
        if (count[0] > 0) run(0);
        for (auto& th : pool) th.join();
        for (int t = 0; t < T; ++t)
            if (code[t] != MGMLMC_OK) throw Error(code[t], "term " + std::to_string(t) + ": " + msg[t]);
    };
    round(std::vector<long long>(T, 0), std::vector<long long>(T, pilot));
    int rounds = 0;
    double est_re = 0, est_im = 0, rel = 0, tau_re = 0, tau_im = 0;
    for (int t = 0; t < T; ++t) {
        const TermLevels tl = term_levels(*ctx_of[t], t);
        if (tl.defl) {
            tau_re += tl.defl->tau_used_re();
            tau_im += tl.defl->tau_used_im();
        }
    }
    bool converged = false;
    for (;;) {
        check_cancel();
        std::vector<double> N(T), V(T), C(T);
        est_re = tau_re;
        est_im = tau_im;
        double err2 = 0;
        long long total = 0;
        for (int t = 0; t < T; ++t) {
            const mg::TermStats& S = ctx_of[t]->stats[t];
            N[t] = (double)S.n;
            const double mr = S.sum_re / S.n, mi = S.sum_im / S.n;
            V[t] = std::max(0.0, (S.sum_abs2 - S.n * (mr * mr + mi * mi)) / (S.n - 1));
            C[t] = costs ? costs[t] : std::max(S.seconds / S.n, 1e-12);
            est_re += mr;
            est_im += mi;
            err2 += V[t] / N[t];
            total += S.n;
        }
        const double mag = std::hypot(est_re, est_im);
        rel = mag > 0 ? std::sqrt(err2) / mag : INFINITY;
        if (rel <= rel_tol) {
            converged = true;
            break;
        }
        if (total >= max_samples) break;
        // Giles-style allocation, growth capped at x2 per round
        const double eps = rel_tol * mag;
        double sum_vc = 0;
        for (int t = 0; t < T; ++t) sum_vc += std::sqrt(V[t] * C[t]);
        std::vector<long long> target(T);
        bool grow = false;
        for (int t = 0; t < T; ++t) {
            const double want = std::ceil(std::sqrt(V[t] / C[t]) * sum_vc / (eps * eps));
            long long nn = (long long)std::min(std::max(want, N[t]), 2 * N[t]);
            target[t] = nn;
            grow |= nn > (long long)N[t];
        }
        if (!grow) {
            int worst = 0;
            for (int t = 1; t < T; ++t)
                if (V[t] / N[t] > V[worst] / N[worst]) worst = t;
            target[worst] = 2 * (long long)N[worst];
        }
        std::vector<long long> first(T), count(T);
        for (int t = 0; t < T; ++t) {
            first[t] = (long long)N[t];
            count[t] = std::max(0LL, target[t] - (long long)N[t]);
        }
        round(first, count);
        ++rounds;
    }
    out->trace_re = est_re;
    out->trace_im = est_im;
    out->rel_err = rel;
    out->deflated_part = tau_re;
    out->nterms = T;
    out->converged = converged ? 1 : 0;
    out->rounds = rounds;
    for (int t = 0; t < MGMLMC_MAX_LEVELS; ++t) {
        std::memset(&out->term[t], 0, sizeof(mgmlmc_level_stats));
        if (t < T) fill_stats(ctx_of[t]->stats[t], &out->term[t]);
    }
}

}  // namespace mg

using mg::mlmc_loop;

extern "C" {

int mgmlmc_estimate_trace(mgmlmc_ctx* h, double rel_tol, int64_t max_samples, uint64_t seed, const double* costs,
                          mgmlmc_trace_result* out) {
    API_BEGIN(h)
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "estimate_trace: no hierarchy");
    mlmc_loop(std::vector<Ctx*>(c.nterms, &c), false, rel_tol, max_samples, seed, costs, out);
    API_END
}

int mgmlmc_estimate_trace_concurrent(mgmlmc_ctx* const* contexts, int n, double rel_tol, int64_t max_samples,
                                     uint64_t seed, const double* costs, mgmlmc_trace_result* out) {
    if (!contexts || n < 1) return MGMLMC_EINVAL;
    mgmlmc_ctx* h = contexts[0];
    API_BEGIN(h)
    MG_REQUIRE(c.have_hier && n == c.nterms, MGMLMC_EINVAL, "estimate_trace_concurrent: one context per term");
    std::vector<Ctx*> ctx_of(n);
    for (int t = 0; t < n; ++t) {
        MG_REQUIRE(contexts[t], MGMLMC_EINVAL, "estimate_trace_concurrent: null context");
        for (int k = 0; k < t; ++k)
            MG_REQUIRE(contexts[k] != contexts[t], MGMLMC_EINVAL, "estimate_trace_concurrent: contexts must differ");
        ctx_of[t] = &contexts[t]->c;
    }
    mlmc_loop(ctx_of, true, rel_tol, max_samples, seed, costs, out);
    API_END
}

int mgmlmc_apply(mgmlmc_ctx* h, int op, int level, int nrhs, const double* x, double* y) {
    API_BEGIN(h)
    require_level(c, level);
    MG_REQUIRE(x && y && nrhs >= 1, MGMLMC_EINVAL, "apply: bad argument");
    const int l = level - 1;
    long long nin = c.lev[l].n, nout = c.lev[l].n;
    if (op == MGMLMC_OP_PH || op == MGMLMC_OP_P) {
        MG_REQUIRE(level < c.L, MGMLMC_EINVAL, "apply: P/P^H need level < L");
        if (op == MGMLMC_OP_PH) nout = c.lev[l + 1].n;
        else nin = c.lev[l + 1].n;
    }
    if (op == MGMLMC_OP_DINV_C) MG_REQUIRE(level == c.L, MGMLMC_EINVAL, "apply: DINV_C needs level == L");
    if (op == MGMLMC_OP_SMOOTH)
        MG_REQUIRE(level >= 2 && level < c.L, MGMLMC_EINVAL, "apply: SMOOTH needs 2 <= level < L");
    MG_REQUIRE(op >= 0 && op <= 6, MGMLMC_EINVAL, "apply: unknown op");
    double2* xt = upload_block(c, x, nin, nrhs, "ap_x");
    double2* yt = c.scratch<double2>("ap_y", (size_t)nout * nrhs);
    switch (op) {
        case MGMLMC_OP_D: mg::apply_D<double2>(c, l, yt, xt, nullptr, nrhs, 0, nullptr); break;
        case MGMLMC_OP_PH: mg::apply_restrict<double2>(c, l, yt, xt, nrhs); break;
        case MGMLMC_OP_P: mg::apply_prolong<double2>(c, l, yt, xt, nrhs, false); break;
        case MGMLMC_OP_G5: mg::launch_gamma5<double2>(yt, xt, c.lev[l].nsites, c.lev[l].d, nrhs, c.stream); break;
        case MGMLMC_OP_SMOOTH:
            if (c.opt.mg_precision == 64) {
                mg::apply_smoother_operator<double2>(c, l, yt, xt, nrhs, nullptr);
            } else {
                float2* x32 = c.scratch<float2>("ap_x32", (size_t)nin * nrhs);
                float2* y32 = c.scratch<float2>("ap_y32", (size_t)nout * nrhs);
                mg::launch_convert<float2, double2>(x32, xt, nin * nrhs, c.stream);
                mg::apply_smoother_operator<float2>(c, l, y32, x32, nrhs, nullptr);
                mg::launch_convert<double2, float2>(yt, y32, nout * nrhs, c.stream);
            }
            break;
        default:
            if (c.opt.mg_precision == 64) {
                mg::mg_cycle<double2>(c, l, yt, xt, nrhs);
            } else {
                float2* x32 = c.scratch<float2>("ap_x32", (size_t)nin * nrhs);
                float2* y32 = c.scratch<float2>("ap_y32", (size_t)nout * nrhs);
                mg::launch_convert<float2, double2>(x32, xt, nin * nrhs, c.stream);
                mg::mg_cycle<float2>(c, l, y32, x32, nrhs);
                mg::launch_convert<double2, float2>(yt, y32, nout * nrhs, c.stream);
            }
    }
    mg::check_device_error(c);
    download_block(c, y, yt, nout, nrhs, "ap_out");
    API_END
}

int mgmlmc_solve(mgmlmc_ctx* h, int level, int nrhs, const double* b, double* x, int* iters) {
    API_BEGIN(h)
    require_level(c, level);
    MG_REQUIRE(b && x && nrhs >= 1, MGMLMC_EINVAL, "solve: bad argument");
    const int l = level - 1;
    const long long n = c.lev[l].n;
    double2* bt = upload_block(c, b, n, nrhs, "sv_b");
    double2* xt = c.scratch<double2>("sv_x", (size_t)n * nrhs);
    int ok = 0;
    const long long it = mg::solve(c, l, bt, xt, nrhs, c.opt.solve_tol, &ok);
    download_block(c, x, xt, n, nrhs, "sv_out");
    if (iters) *iters = (int)it;
    if (!ok) throw Error(MGMLMC_ENOTCONVERGED, "solve: max_iters reached");
    API_END
}

int mgmlmc_noise(mgmlmc_ctx* h, int level, int64_t first_sample, int nsamples, uint64_t seed, double* x) {
    API_BEGIN(h)
    require_level(c, level);
    MG_REQUIRE(x && nsamples >= 1 && first_sample >= 0, MGMLMC_EINVAL, "noise: bad argument");
    const long long n = c.lev[level - 1].n;
    double2* X = c.scratch<double2>("nz_X", (size_t)n * nsamples);
    mg::launch_noise<double2>(X, n, nsamples, seed, (uint64_t)level, first_sample, c.stream);
    std::vector<double> tmp((size_t)2 * n * nsamples);
    download_block(c, tmp.data(), X, n, nsamples, "nz_out");
    for (size_t i = 0; i < (size_t)n * nsamples; ++i) x[i] = tmp[2 * i];
    API_END
}

int mgmlmc_get_test_vectors(mgmlmc_ctx* h, int level, double* v) {
    API_BEGIN(h)
    require_level(c, level);
    MG_REQUIRE(level < c.L && v, MGMLMC_EINVAL, "get_test_vectors: level < L and v != NULL");
    const mg::Level& L = c.lev[level - 1];
    MG_CUDA(cudaMemcpyAsync(v, L.tv, sizeof(double2) * L.n * L.nvec, cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    API_END
}

int mgmlmc_profile(mgmlmc_ctx* h, int enable, int reset) {
    API_BEGIN(h)
    c.sync();
    c.prof.on = enable != 0;
    if (reset) c.prof.clear();
    API_END
}

int mgmlmc_profile_report(mgmlmc_ctx* h, char* buf, size_t cap, size_t* needed) {
    API_BEGIN(h)
    c.sync();
    std::string js = "{";
    bool first = true;
    char tmp[256];
    for (const auto& kv : c.prof.stats) {
        snprintf(tmp, sizeof(tmp),
                 "%s\"%s\": {\"count\": %lld, \"ms\": %.6f, \"bytes\": %.6e, \"flops\": %.6e, \"impl_bytes\": %.6e}",
                 first ? "" : ", ", kv.first.c_str(), kv.second.count, kv.second.ms, kv.second.bytes, kv.second.flops,
                 kv.second.impl_bytes);
        js += tmp;
        first = false;
    }
    snprintf(tmp, sizeof(tmp), "%s\"__launches__\": {\"count\": %lld, \"ms\": 0, \"bytes\": 0, \"flops\": 0}",
             first ? "" : ", ", mg::launch_counter() - c.prof.launch_base);
    js += tmp;
    js += "}";
    if (needed) *needed = js.size();
    if (buf && cap > 0) {
        const size_t m = std::min(cap - 1, js.size());
        memcpy(buf, js.data(), m);
        buf[m] = 0;
    }
    API_END
}

int mgmlmc_memory(const mgmlmc_ctx* h, size_t* live, size_t* peak) {
    if (!h) return MGMLMC_EINVAL;
    if (live) *live = h->c.live_bytes;
    if (peak) *peak = h->c.peak_bytes;
    return MGMLMC_OK;
}

int mgmlmc_level_info(const mgmlmc_ctx* h, int level, int* lx, int* lt, int* d, int64_t* n) {
    if (!h) return MGMLMC_EINVAL;
    const Ctx& c = h->c;
    if (!c.have_hier) return MGMLMC_ESTATE;
    if (level < 1 || level > c.L) return MGMLMC_EINVAL;
    const mg::Level& L = c.lev[level - 1];
    if (lx) *lx = L.lx;
    if (lt) *lt = L.lt;
    if (d) *d = L.d;
    if (n) *n = L.n;
    return MGMLMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------
// Autotuner (no counterpart in the paper; it picks how the estimator's blocks are
// cut and solved on this GPU).  A candidate is (block width N, FGMRES restart m,
// post-smoothing steps nu, K-cycle steps); the device-memory model of the
// context's shape (footprint.h) discards those that exceed the HBM budget, and the
// rest are timed on one block of N samples of every term (the same Z2 noise each
// time, CUDA events on the context's stream).  Coordinate search: the widest
// blocks first, then the restart length, the smoother steps and the coarse-grid
// correction.  The fastest setting by samples per second becomes the context's.
namespace {

mg::Shape context_shape(const Ctx& c) {
    mg::Shape s;
    s.L = c.L;
    s.nterm_levels = c.term_level[c.nterms - 1] + 1;
    for (int l = 0; l < c.L; ++l) {
        s.sites[l] = c.lev[l].nsites;
        s.n[l] = c.lev[l].n;
        s.d[l] = c.lev[l].d;
        s.nvec[l] = c.lev[l].nvec;
    }
    s.k = c.defl.k;
    s.precision = c.opt.mg_precision;
    return s;
}

void release_scratch(Ctx& c) {
    c.sync();
    for (auto& kv : c.ws) c.dev_free(kv.second.p);
    c.ws.clear();
    c.dev_err = nullptr;
}

}  // namespace

extern "C" int mgmlmc_autotune(mgmlmc_ctx* h, size_t hbm_budget, int max_trials, mgmlmc_tune_result* out) {
    API_BEGIN(h)
    MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "autotune: no hierarchy");
    MG_REQUIRE(out && max_trials >= 1, MGMLMC_EINVAL, "autotune: bad argument");
    std::memset(out, 0, sizeof(*out));
    size_t free_b = 0, total_b = 0;
    MG_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)(free_b + c.live_bytes));
    mg::Shape base = context_shape(c);
    const mgmlmc_options start = c.opt;
    struct Cand {
        int N, m, nu, kc;
    };
    auto fits = [&](const Cand& q, size_t* bytes) {
        mg::Shape s = base;
        s.N = q.N;
        s.m = q.m;
        s.kcycle = q.kc;
        const size_t b = mg::footprint_bytes(s);
        if (bytes) *bytes = b;
        return b <= budget;
    };
    const uint64_t kSeed = 0x2211153839ull;
    int trials = 0, last_N = -1, warm_m = 0, warm_kc = -1;
    double best_rate = -1;
    Cand best{start.max_block_rhs, start.fgmres_restart, start.nu_post, start.kcycle_iters};
    std::vector<Cand> tried;
    auto was_tried = [&](const Cand& q) {
        for (const Cand& t : tried)
            if (t.N == q.N && t.m == q.m && t.nu == q.nu && t.kc == q.kc) return true;
        return false;
    };
    auto time_one = [&](const Cand& q) -> double {
        tried.push_back(q);
        c.opt.max_block_rhs = q.N;
        c.opt.fgmres_restart = q.m;
        c.opt.nu_post = q.nu;
        c.opt.kcycle_iters = q.kc;
        auto run_all = [&]() {
            long long iters = 0;
            for (int t = 0; t < c.nterms; ++t) {
                const TermLevels tl = term_levels(c, t);
                const long long n = c.lev[tl.a].n;
                double2* X = c.scratch<double2>("tune_X", (size_t)n * q.N);
                double2* smp = c.scratch<double2>("tune_smp", (size_t)q.N);
                mg::launch_noise<double2>(X, n, q.N, kSeed, (uint64_t)(tl.a + 1), 0, c.stream);
                MG_REQUIRE(run_term_block(c, tl, X, q.N, smp, &iters), MGMLMC_ENOTCONVERGED,
                           "autotune: a trial solve did not converge");
            }
        };
        // work space of this width, a longer restart or another coarse-grid correction:
        // allocated in an untimed run
        if (q.N != last_N || q.m > warm_m || q.kc != warm_kc) {
            if (q.N != last_N) release_scratch(c);
            run_all();
            if (q.N != last_N) warm_m = 0;
            last_N = q.N;
            warm_m = std::max(warm_m, q.m);
            warm_kc = q.kc;
        }
        cudaEvent_t e0, e1;
        MG_CUDA(cudaEventCreate(&e0));
        MG_CUDA(cudaEventCreate(&e1));
        MG_CUDA(cudaEventRecord(e0, c.stream));
        run_all();
        MG_CUDA(cudaEventRecord(e1, c.stream));
        c.sync();
        float ms = 0;
        MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double rate = (double)c.nterms * q.N / (ms * 1e-3);
        if (trials < MGMLMC_TUNE_LOG) {
            mgmlmc_tune_trial& tr = out->log[trials];
            tr.block_rhs = q.N;
            tr.fgmres_restart = q.m;
            tr.nu_post = q.nu;
            tr.kcycle_iters = q.kc;
            tr.samples_per_s = rate;
        }
        ++trials;
        if (rate > best_rate) {
            best_rate = rate;
            best = q;
        }
        return rate;
    };
    try {
        // 1. block width: the three widest that fit with a restart of at most 16 (the
        //    restart is chosen next, for the width found here)
        const int m1 = std::min(start.fgmres_restart, 16);
        std::vector<int> widths;
        for (int N : {1024, 512, 256, 128, 64, 32}) {
            Cand q{N, m1, start.nu_post, start.kcycle_iters};
            if (fits(q, nullptr)) widths.push_back(N);
        }
        MG_REQUIRE(!widths.empty(), MGMLMC_ENOMEM, "autotune: no block width fits the budget");
        for (size_t i = 0; i < widths.size() && i < 3 && trials < max_trials; ++i)
            time_one(Cand{widths[i], m1, start.nu_post, start.kcycle_iters});
        // 2. restart length: 8, then 4 where 8 won; 12; 24 where 16 still leads
        for (int m : {8, 4, 12, 24}) {
            if ((m == 4 && best.m != 8) || (m == 24 && best.m != 16)) continue;
            Cand q{best.N, m, best.nu, best.kc};
            if (trials < max_trials && !was_tried(q) && fits(q, nullptr)) time_one(q);
        }
        // 3. smoother steps, 4. coarse-grid correction
        for (int nu : {2, 6}) {
            Cand q{best.N, best.m, nu, best.kc};
            if (trials < max_trials && !was_tried(q)) time_one(q);
        }
        if (c.L >= 4) {
            Cand q{best.N, best.m, best.nu, best.kc > 0 ? 0 : 2};
            if (trials < max_trials && !was_tried(q) && fits(q, nullptr)) time_one(q);
        }
    } catch (...) {
        c.opt = start;
        release_scratch(c);
        throw;
    }
    c.opt.max_block_rhs = best.N;
    c.opt.fgmres_restart = best.m;
    c.opt.nu_post = best.nu;
    c.opt.kcycle_iters = best.kc;
    release_scratch(c);
    out->block_rhs = best.N;
    out->fgmres_restart = best.m;
    out->nu_post = best.nu;
    out->kcycle_iters = best.kc;
    out->samples_per_s = best_rate;
    size_t fb = 0;
    fits(best, &fb);
    out->footprint = fb;
    out->budget = budget;
    out->trials = trials;
    API_END
}

