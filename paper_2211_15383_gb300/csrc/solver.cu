// Solver layer: operator application per level, the multigrid cycle used as a
// preconditioner (Sect. 3.1, Eq. two_level_mg_method applied recursively), the
// multi-RHS flexible GMRES, and the FP64 outer solve (plain FP64 FGMRES, or
// FP64 iterative refinement around an FP32 FGMRES for the mixed mode).
//
// The smoother S^(nu) is nu steps of minimal residual (GMRES(1)) per rhs: one
// of the Krylov smoothers Sect. 3.1 lists; FGMRES tolerates its
// non-linearity.  The coarsest level is solved by its stored dense inverse.
#include <cmath>
#include <cstdio>

#include "context.h"

namespace mg {

template <typename C> static const C* links(Ctx& c);
template <> const double2* links<double2>(Ctx& c) { return c.U64; }
template <> const float2* links<float2>(Ctx& c) { return c.U32; }
template <typename C> static const C* blocks(const Level& L);
template <> const double2* blocks<double2>(const Level& L) { return L.A64; }
template <> const float2* blocks<float2>(const Level& L) { return L.A32; }
template <typename C> static const C* hat_blocks(const Level& L);
template <> const double2* hat_blocks<double2>(const Level& L) { return L.Ahat64; }
template <> const float2* hat_blocks<float2>(const Level& L) { return L.Ahat32; }
template <typename C> static const C* minv(const Level& L);
template <> const double2* minv<double2>(const Level& L) { return L.Minv64; }
template <> const float2* minv<float2>(const Level& L) { return L.Minv32; }
template <typename C> static const C* prol(const Level& L);
template <> const double2* prol<double2>(const Level& L) { return L.P64; }
template <> const float2* prol<float2>(const Level& L) { return L.P32; }

static std::string nm(const char* base, int l, size_t sz) {
    return std::string(base) + "_" + std::to_string(l) + "_" + std::to_string(sz);
}

static const char* prec_tag(size_t sz) { return sz == sizeof(double2) ? "f64" : "f32"; }

// On the first coarse level D_2 = P_1^H D_1 P_1 (the Galerkin product); in FP64,
// where the pipe issues 2 FMA per SM and clock, restrict(Wilson(prolong(x))) can be
// cheaper than the 5-point stencil with dense d x d blocks.
static bool galerkin_form_cheaper(const Ctx& c, int l) {
    if (l != 1) return false;
    const Level& F = c.lev[0];
    const Level& Cl = c.lev[1];
    const double galerkin = 16.0 * F.nvec * F.n + 60.0 * F.nsites;   // prolong + restrict + Wilson
    const double direct = 40.0 * Cl.d * Cl.d * Cl.nsites;            // 5 blocks of d x d per site
    return galerkin < direct;
}

template <typename C> static bool galerkin_apply(Ctx&, C*, const C*, const C*, int, int) { return false; }
template <> bool galerkin_apply<double2>(Ctx& c, double2* y, const double2* x, const double2* b, int N, int mode) {
    if (mode == 2 || !galerkin_form_cheaper(c, 1)) return false;
    const Level& F = c.lev[0];
    const Level& Cl = c.lev[1];
    double2* t = c.scratch<double2>("gal64_t", (size_t)F.n * N);
    double2* u = c.scratch<double2>("gal64_u", (size_t)F.n * N);
    apply_prolong<double2>(c, 0, t, x, N, false);
    apply_D<double2>(c, 0, u, t, nullptr, N, 0, nullptr);
    if (mode == 0) {
        apply_restrict<double2>(c, 0, y, u, N);
        return true;
    }
    double2* v = c.scratch<double2>("gal64_v", (size_t)Cl.n * N);
    apply_restrict<double2>(c, 0, v, u, N);
    MG_CUDA(cudaMemcpyAsync(y, b, sizeof(double2) * Cl.n * N, cudaMemcpyDeviceToDevice, c.stream));
    launch_axpy_rhs<double2, double2>(y, nullptr, nullptr, -1.0, v, Cl.n, N, c.stream);
    return true;
}

template <typename C>
void apply_D(Ctx& c, int l, C* y, const C* x, const C* b, int N, int mode, double2* dots) {
    if (l == 1 && galerkin_apply<C>(c, y, x, b, N, mode)) return;
    const Level& L = c.lev[l];
    const int groups = (l == 0) ? stencil_groups(L.nsites, N) : block_stencil_groups(L.nsites, L.d, N);
    // algorithmic traffic: read x once, write y once (+ b for the residual form),
    // operator data once; flops: 60 per fine site and rhs, 8 d^2 * 5 per coarse site and rhs
    const double s = sizeof(C);
    const double vec = (double)L.n * N * s;
    const double bytes = vec * (mode == 1 ? 3 : 2) +
                         (l == 0 ? 2.0 * L.nsites * s : 5.0 * L.nsites * L.d * L.d * s);
    const double flops = (l == 0) ? 60.0 * L.nsites * N : 40.0 * L.d * L.d * (double)L.nsites * N;
    double2* part = nullptr;
    if (mode == 2) part = c.scratch<double2>("part_st", (size_t)groups * 2 * N);
    {
        ProfScope ps(c, "D" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)), bytes, flops);
        if (l == 0)
            launch_wilson<C>(y, x, b, links<C>(c), c.m0, L.lx, L.lt, N, mode, part, groups, c.stream);
        else
            launch_block_stencil<C>(y, x, b, blocks<C>(L), L.lx, L.lt, L.d, N, mode, part, groups, c.stream);
    }
    if (mode == 2) {
        ProfScope ps(c, "reduce", (double)groups * 2 * N * 16, (double)groups * 2 * N * 2);
        launch_finalize_rows(dots, part, groups, 2 * N, c.stream);
    }
}

int* device_error_flag(Ctx& c) {
    if (!c.dev_err) {
        c.dev_err = c.scratch<int>("dev_err", 1);
        MG_CUDA(cudaMemsetAsync(c.dev_err, 0, sizeof(int), c.stream));
    }
    return c.dev_err;
}

// The block stencil of D M^{-1} runs on the tensor cores (BF16 operands, FP32
// accumulation) when mg_precision is 16 and d = 16: the smoother only
// preconditions the FP32 FGMRES, whose own matrix-vector products stay FP32.
template <typename C> static bool tc_smoother(const Level&, int) { return false; }
template <> bool tc_smoother<float2>(const Level& L, int N) { return L.Ahat16 && tc_stencil_supported(L.d, N); }

static __nv_bfloat16* tc_tiles(Ctx& c, int l, int N) {
    return reinterpret_cast<__nv_bfloat16*>(c.scratch_bytes(nm("mr_rt", l, 2), tc_tiles_bytes(c.lev[l].nsites, N)));
}

// y = (D_l M_l^{-1}) x on the tensor cores, x given as its BF16 tiles xt, y as FP32 rows
// (y) or BF16 tiles (yt); dots as apply_Dhat (against the BF16 x).
static void apply_Dhat_tc(Ctx& c, int l, float2* y, __nv_bfloat16* yt, const __nv_bfloat16* xt, int N,
                          double2* dots) {
    const Level& L = c.lev[l];
    const int groups = block_stencil_tc_groups(L.nsites, N);
    double2* part = c.scratch<double2>("part_st", (size_t)groups * 2 * N);
    {
        // algorithmic traffic: BF16 x (4 B per complex) and y (FP32 8 B or BF16 4 B) once,
        // the BF16 operands once
        ProfScope ps(c, "D" + std::to_string(l + 1) + ".bf16",
                     (double)L.n * N * (4 + (yt ? 4 : 8)) + 5.0 * L.nsites * 8.0 * L.d * L.d,
                     40.0 * L.d * L.d * (double)L.nsites * N);
        launch_block_stencil_tc(y, yt, nullptr, xt, L.Ahat16, L.lx, L.lt, N, part, groups, device_error_flag(c),
                                c.stream);
    }
    ProfScope ps(c, "reduce", (double)groups * 2 * N * 16, (double)groups * 2 * N * 2);
    launch_finalize_rows(dots, part, groups, 2 * N, c.stream);
}

static void pack_tiles(Ctx& c, int l, __nv_bfloat16* xt, const float2* x, int N) {
    const Level& L = c.lev[l];
    ProfScope ps(c, "pack" + std::to_string(l + 1) + ".bf16", (double)L.n * N * (8 + 4), 0.0);
    launch_pack_tiles_bf16(xt, x, L.nsites, N, c.stream);
}

// y = (D_l M_l^{-1}) x with the precomputed block stencil (block-Jacobi smoother).
template <typename C>
static void apply_Dhat(Ctx& c, int l, C* y, const C* x, int N, double2* dots) {
    const Level& L = c.lev[l];
    const int groups = block_stencil_groups(L.nsites, L.d, N);
    const double s = sizeof(C);
    double2* part = c.scratch<double2>("part_st", (size_t)groups * 2 * N);
    {
        ProfScope ps(c, "D" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)),
                     (double)L.n * N * s * 2 + 5.0 * L.nsites * L.d * L.d * s,
                     40.0 * L.d * L.d * (double)L.nsites * N);
        launch_block_stencil<C>(y, x, nullptr, hat_blocks<C>(L), L.lx, L.lt, L.d, N, 2, part, groups, c.stream);
    }
    ProfScope ps(c, "reduce", (double)groups * 2 * N * 16, (double)groups * 2 * N * 2);
    launch_finalize_rows(dots, part, groups, 2 * N, c.stream);
}

template <typename C> static bool apply_smoother_tc(Ctx&, int, C*, const C*, int, double2*) { return false; }
template <> bool apply_smoother_tc<float2>(Ctx& c, int l, float2* y, const float2* x, int N, double2* dots) {
    if (!tc_smoother<float2>(c.lev[l], N)) return false;
    __nv_bfloat16* xt = tc_tiles(c, l, N);
    pack_tiles(c, l, xt, x, N);
    apply_Dhat_tc(c, l, y, nullptr, xt, N, dots);
    return true;
}

template <typename C>
void apply_smoother_operator(Ctx& c, int l, C* y, const C* x, int N, double2* dots) {
    MG_REQUIRE(l >= 1 && l < c.L - 1 && hat_blocks<C>(c.lev[l]), MGMLMC_EINVAL,
               "smoother operator: only coarse levels above the coarsest");
    if (!dots) dots = c.scratch<double2>("smop_dots", 2 * (size_t)N);
    if (!apply_smoother_tc<C>(c, l, y, x, N, dots)) apply_Dhat<C>(c, l, y, x, N, dots);
}

template <typename C>
void apply_restrict(Ctx& c, int l, C* xc, const C* x, int N) {
    const Level& L = c.lev[l];
    const double s = sizeof(C);
    ProfScope ps(c, "PH" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)),
                 (double)L.n * N * s + (double)c.lev[l + 1].n * N * s + (double)L.n * L.nvec * s,
                 8.0 * L.nvec * (double)L.n * N);
    launch_restrict<C>(xc, x, prol<C>(L), L.lx, L.lt, L.d, L.ax, L.at, L.nvec, N, c.stream);
}

template <typename C>
void apply_prolong(Ctx& c, int l, C* x, const C* xc, int N, bool accumulate) {
    const Level& L = c.lev[l];
    const double s = sizeof(C);
    ProfScope ps(c, "P" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)),
                 (double)L.n * N * s * (accumulate ? 2 : 1) + (double)c.lev[l + 1].n * N * s + (double)L.n * L.nvec * s,
                 8.0 * L.nvec * (double)L.n * N);
    launch_prolong<C>(x, xc, prol<C>(L), L.lx, L.lt, L.d, L.ax, L.at, L.nvec, N, accumulate, c.stream);
}

template <typename C> static void coarsest_apply(Ctx& c, C* e, const C* r, int N);
static double dinv_bytes(const Level& L, int N, double s) { return (double)L.n * L.n * s + 2.0 * L.n * N * s; }
static double dinv_flops(const Level& L, int N) { return 8.0 * (double)L.n * L.n * N; }
template <> void coarsest_apply<double2>(Ctx& c, double2* e, const double2* r, int N) {
    const Level& L = c.lev[c.L - 1];
    ProfScope ps(c, "Dinv.f64", dinv_bytes(L, N, 16), dinv_flops(L, N));
    launch_gemm_nn<double2>(e, L.Dinv64, r, (int)L.n, (int)L.n, N, false, c.stream);
}
template <> void coarsest_apply<float2>(Ctx& c, float2* e, const float2* r, int N) {
    const Level& L = c.lev[c.L - 1];
    if (L.Dinv16) {
        // BF16 inverse on the tensor cores; algorithmic bytes: the BF16 matrix once + FP32 in/out
        ProfScope ps(c, "Dinv.bf16", (double)L.n * 2 * L.n * 2 + 2.0 * L.n * N * 8, dinv_flops(L, N));
        void* scr = c.scratch_bytes("tc_scratch", coarse_inverse_bf16_scratch((int)L.n, N));
        launch_coarse_inverse_bf16(e, r, L.Dinv16, (int)L.n, N, scr, device_error_flag(c), c.stream);
        return;
    }
    ProfScope ps(c, "Dinv.f32", dinv_bytes(L, N, 8), dinv_flops(L, N));
    launch_gemm_nn<float2>(e, L.Dinv32, r, (int)L.n, (int)L.n, N, false, c.stream);
}

// nu block-Jacobi MR steps from the residual's BF16 tiles rt (overwritten), r and p
// only as BF16 tiles; yh receives the preconditioned correction.
static void smooth_tc_tiles(Ctx& c, int l, float2* yh, __nv_bfloat16* rt, int N, int nu, double2* dots) {
    const Level& L = c.lev[l];
    __nv_bfloat16* pt =
        reinterpret_cast<__nv_bfloat16*>(c.scratch_bytes(nm("mr_pt", l, 2), tc_tiles_bytes(L.nsites, N)));
    for (int s = 0; s < nu; ++s) {
        apply_Dhat_tc(c, l, nullptr, pt, rt, N, dots);
        // traffic: r and p tiles read, r tiles written (4 B per complex), yh read and written
        ProfScope ps(c, "mr" + std::to_string(l + 1) + ".bf16", (double)L.n * N * (3 * 4 + (s ? 16 : 8)),
                     16.0 * L.n * N);
        launch_mr_update_bf16(yh, rt, pt, dots, L.nsites, N, s == 0, c.stream);
    }
}

// Post-smoothing of the V-cycle on the tensor cores: the residual r - D_l e is formed
// from BF16 tiles of e straight into the smoother's BF16 residual tiles (it only
// feeds the smoother, which needs a few digits), then the BF16 smoother; e += M^{-1} yh.
template <typename C> static bool residual_smooth_tc(Ctx&, int, C*, const C*, int) { return false; }

// Block-Jacobi MR on the tensor cores.  The residual's BF16 tiles are packed once;
// when the caller does not need the final residual (post-smoothing), r and p live
// only as BF16 tiles from there on (the smoother needs a few digits, and FGMRES
// is flexible), else r stays FP32 and each update writes the next tiles.
template <typename C> static bool mr_smooth_tc(Ctx&, int, C*, C*, int, int, bool, bool) { return false; }
template <>
bool mr_smooth_tc<float2>(Ctx& c, int l, float2* e, float2* r, int N, int nu, bool e_zero, bool need_r) {
    const Level& L = c.lev[l];
    if (nu <= 0 || !tc_smoother<float2>(L, N)) return false;
    float2* yh = c.scratch<float2>(nm("mr_y", l, sizeof(float2)), (size_t)L.n * N);
    double2* dots = c.scratch<double2>(nm("mr_dots", l, sizeof(float2)), 2 * (size_t)N);
    __nv_bfloat16* rt = tc_tiles(c, l, N);
    pack_tiles(c, l, rt, r, N);
    if (need_r) {
        float2* p = c.scratch<float2>(nm("mr_p", l, sizeof(float2)), (size_t)L.n * N);
        for (int s = 0; s < nu; ++s) {
            apply_Dhat_tc(c, l, p, nullptr, rt, N, dots);
            const bool more = s + 1 < nu;
            ProfScope ps(c, "mr" + std::to_string(l + 1) + ".f32", (double)L.n * N * (5 * 8 + (more ? 4 : 0)),
                         16.0 * L.n * N);
            launch_mr_update_tc(yh, r, p, dots, L.nsites, N, s == 0, more ? rt : nullptr, c.stream);
        }
    } else {
        smooth_tc_tiles(c, l, yh, rt, N, nu, dots);
    }
    ProfScope ps(c, "bjac" + std::to_string(l + 1) + ".f32", 3.0 * L.n * N * sizeof(float2),
                 8.0 * L.d * (double)L.n * N);
    launch_block_diag_apply<float2>(e, yh, L.Minv32, L.nsites, L.d, N, !e_zero, c.stream);
    return true;
}

// Plain MR on the fine level with r and p in BF16 (mg_precision 16, post-smoothing):
// the same few digits as the coarse smoother, half the traffic of the FP32 vectors;
// the correction e stays FP32.
template <typename C> static bool mr_smooth_fine_bf16(Ctx&, int, C*, C*, int, int, bool, bool) { return false; }
template <>
bool mr_smooth_fine_bf16<float2>(Ctx& c, int l, float2* e, float2* r, int N, int nu, bool e_zero, bool need_r) {
    if (l != 0 || need_r || nu <= 0 || c.opt.mg_precision != 16 || N % 4) return false;
    const Level& L = c.lev[0];
    const size_t nN = (size_t)L.n * N;
    uint32_t* rb = c.scratch<uint32_t>("mrf_rb", nN);
    uint32_t* pb = c.scratch<uint32_t>("mrf_pb", nN);
    double2* dots = c.scratch<double2>(nm("mr_dots", 0, sizeof(float2)), 2 * (size_t)N);
    const int groups = stencil_groups_bf16(L.nsites, N);
    double2* part = c.scratch<double2>("part_st", (size_t)groups * 2 * N);
    {
        ProfScope ps(c, "pack1.bf16", (double)nN * (8 + 4), 0.0);
        launch_pack_bf16(rb, r, (long long)nN, c.stream);
    }
    for (int s = 0; s < nu; ++s) {
        {
            // algorithmic traffic: BF16 x read and y written once (4 B per complex), links once
            ProfScope ps(c, "D1.bf16", (double)nN * 8 + 2.0 * L.nsites * 8, 60.0 * L.nsites * N);
            launch_wilson_bf16(pb, rb, c.U32, c.m0, L.lx, L.lt, N, part, groups, c.stream);
        }
        {
            ProfScope ps(c, "reduce", (double)groups * 2 * N * 16, (double)groups * 2 * N * 2);
            launch_finalize_rows(dots, part, groups, 2 * N, c.stream);
        }
        // traffic: r and p read, r written (4 B each), e read (after the first step) and written
        ProfScope ps(c, "mr1.bf16", (double)nN * (12 + (e_zero && s == 0 ? 8 : 16)), 16.0 * nN);
        launch_mr_update_fine_bf16(e, rb, pb, dots, L.n, N, e_zero && s == 0, c.stream);
    }
    return true;
}

// nu MR steps on D_l e = r0 starting from e (or 0); r holds the current residual on
// entry and is overwritten (with the final residual when need_r).
template <>
bool residual_smooth_tc<float2>(Ctx& c, int l, float2* e, const float2* r, int N) {
    const Level& L = c.lev[l];
    const int nu = c.opt.nu_post;
    if (nu <= 0 || !L.A16 || !tc_smoother<float2>(L, N)) return false;
    float2* yh = c.scratch<float2>(nm("mr_y", l, sizeof(float2)), (size_t)L.n * N);
    double2* dots = c.scratch<double2>(nm("mr_dots", l, sizeof(float2)), 2 * (size_t)N);
    __nv_bfloat16* et =
        reinterpret_cast<__nv_bfloat16*>(c.scratch_bytes(nm("cyc_et", l, 2), tc_tiles_bytes(L.nsites, N)));
    __nv_bfloat16* rt = tc_tiles(c, l, N);
    pack_tiles(c, l, et, e, N);
    {
        const int groups = block_stencil_tc_groups(L.nsites, N);
        double2* part = c.scratch<double2>("part_st", (size_t)groups * 2 * N);
        // algorithmic traffic: e tiles (4 B per complex) and r (8 B) read, residual tiles written (4 B)
        ProfScope ps(c, "D" + std::to_string(l + 1) + "res.bf16",
                     (double)L.n * N * (4 + 8 + 4) + 5.0 * L.nsites * 8.0 * L.d * L.d,
                     40.0 * L.d * L.d * (double)L.nsites * N);
        launch_block_stencil_tc(nullptr, rt, r, et, L.A16, L.lx, L.lt, N, part, groups, device_error_flag(c),
                                c.stream);
    }
    smooth_tc_tiles(c, l, yh, rt, N, nu, dots);
    ProfScope ps(c, "bjac" + std::to_string(l + 1) + ".f32", 3.0 * L.n * N * sizeof(float2),
                 8.0 * L.d * (double)L.n * N);
    launch_block_diag_apply<float2>(e, yh, L.Minv32, L.nsites, L.d, N, true, c.stream);
    return true;
}

template <typename C>
static void mr_smooth(Ctx& c, int l, C* e, C* r, int N, int nu, bool e_zero, bool need_r) {
    if (mr_smooth_tc<C>(c, l, e, r, N, nu, e_zero, need_r)) return;
    const Level& L = c.lev[l];
    C* p = c.scratch<C>(nm("mr_p", l, sizeof(C)), (size_t)L.n * N);
    double2* dots = c.scratch<double2>(nm("mr_dots", l, sizeof(C)), 2 * (size_t)N);
    if (hat_blocks<C>(L)) {
        // block-Jacobi MR: minimal residual steps on D M^{-1} (y accumulates the
        // preconditioned correction), then e += M^{-1} y
        C* yh = c.scratch<C>(nm("mr_y", l, sizeof(C)), (size_t)L.n * N);
        for (int s = 0; s < nu; ++s) {
            apply_Dhat<C>(c, l, p, r, N, dots);
            ProfScope ps(c, "mr" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)), 5.0 * L.n * N * sizeof(C),
                         16.0 * L.n * N);
            launch_mr_update<C>(yh, r, p, dots, L.n, N, s == 0, c.stream);
        }
        if (nu > 0) {
            ProfScope ps(c, "bjac" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)),
                         3.0 * L.n * N * sizeof(C), 8.0 * L.d * (double)L.n * N);
            launch_block_diag_apply<C>(e, yh, minv<C>(L), L.nsites, L.d, N, !e_zero, c.stream);
        }
        return;
    }
    if (mr_smooth_fine_bf16<C>(c, l, e, r, N, nu, e_zero, need_r)) return;
    for (int s = 0; s < nu; ++s) {
        apply_D<C>(c, l, p, r, nullptr, N, 2, dots);
        ProfScope ps(c, "mr" + std::to_string(l + 1) + "." + prec_tag(sizeof(C)), 5.0 * L.n * N * sizeof(C),
                     16.0 * L.n * N);
        launch_mr_update<C>(e, r, p, dots, L.n, N, e_zero && s == 0, c.stream);
    }
}

__global__ void k_sqrt_inplace(double* v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = sqrt(v[i]);
}
__global__ void k_add2(double2* a, const double2* b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = make_double2(a[i].x + b[i].x, a[i].y + b[i].y);
}

// Unnormalised basis vectors are kept while eta = |w| lies in [2^-32, 2^32]: their FP32
// entries, dot products and squared sums then stay far inside the normal range.
constexpr double kEtaLow = 0x1p-32, kEtaHigh = 0x1p32;
__device__ __forceinline__ void keep_eta(double* eta, double* rsc, double en) {
    const bool out = en > 0.0 && (en < kEtaLow || en > kEtaHigh);
    *rsc = out ? 1.0 / en : 0.0;   // the vector is rescaled to unit norm where rsc != 0
    *eta = out ? 1.0 : en;
}

// Arnoldi column j of FGMRES with an unnormalised basis w_i = eta_i v_i (per rhs r):
// on entry h[i] = <w_i, u> summed over the Gram-Schmidt passes and hn2 = |u' / eta_j|^2
// for the orthogonalised u' (u = D M(w_j)); on exit h[i] = H_ij = h[i] / (eta_i eta_j),
// hn2 = H_{j+1,j} = |u'| / eta_j, and w_{j+1} = u' has eta_{j+1} = |u'| (or is marked in
// rsc for rescaling, eta_{j+1} = 1).  A zero eta_j (a zero vector, as a zero rhs or an
// exhausted Krylov space gives) leaves a zero column.
__global__ void k_lazy_column(double2* __restrict__ h, double* __restrict__ hn2, double* __restrict__ eta,
                              double* __restrict__ rsc, int j, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double ej = eta[(long long)j * N + r];
    const double hs = sqrt(hn2[r]);
    for (int i = 0; i <= j; ++i) {
        const double d = eta[(long long)i * N + r] * ej;
        const double f = (d != 0.0) ? 1.0 / d : 0.0;
        const double2 v = h[(long long)i * N + r];
        h[(long long)i * N + r] = make_double2(v.x * f, v.y * f);
    }
    hn2[r] = (ej != 0.0) ? hs : 0.0;
    keep_eta(eta + (long long)(j + 1) * N + r, rsc + r, hs * ej);
}

// The same range check for the first basis vector of a cycle (eta_0 = |r|).
__global__ void k_eta_range(double* __restrict__ eta, double* __restrict__ rsc, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) keep_eta(eta + r, rsc + r, eta[r]);
}

// out = max_j a_j b_j / c_j (terms with c_j = 0 skipped; NaN kept visible).
__global__ void k_max_scaled_ratio(double* out, const double* a, const double* b, const double* cden, int N) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double v = (cden[j] > 0.0) ? a[j] * b[j] / cden[j] : 0.0;
        if (v != v) v = __longlong_as_double(0x7ff8000000000000ll);
        if (!(v <= m)) m = v;
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st && !(sh[threadIdx.x + st] <= sh[threadIdx.x])) sh[threadIdx.x] = sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

static void sqrt_inplace(Ctx& c, double* v, int n) {
    k_sqrt_inplace<<<(n + 127) / 128, 128, 0, c.stream>>>(v, n);
    MG_LAUNCHED();
}

template <typename C>
static void norms(Ctx& c, double* out, const C* x, long long n, int N) {
    double* part = c.scratch<double>("part_nrm", (size_t)reduce_groups(n, N) * N);
    launch_norm2<C>(out, x, n, N, part, c.stream);
    sqrt_inplace(c, out, N);
}

// K-cycle coarse-grid correction: e ~ D_l^{-1} r by k steps of flexible GMRES from
// e = 0, preconditioned by the multigrid cycle of level l.  A fixed number of steps
// with no convergence test, so nothing is read back to the host; the Arnoldi
// bookkeeping (Givens rotations, least-squares solve) runs per rhs on the device.
template <typename C>
static void kcycle(Ctx& c, int l, C* e, const C* r, int N, int k) {
    const Level& L = c.lev[l];
    const long long n = L.n;
    const size_t nN = (size_t)n * N;
    const size_t sz = sizeof(C);
    C* V = c.scratch<C>(nm("kc_V", l, sz), (size_t)(k + 1) * nN);
    C* Z = c.scratch<C>(nm("kc_Z", l, sz), (size_t)k * nN);
    double* beta = c.scratch<double>(nm("kc_beta", l, sz), N);
    double* hnorm = c.scratch<double>(nm("kc_hn", l, sz), N);
    double* resid = c.scratch<double>(nm("kc_res", l, sz), N);
    double2* h = c.scratch<double2>(nm("kc_h", l, sz), (size_t)(k + 1) * N);
    double2* y = c.scratch<double2>(nm("kc_y", l, sz), (size_t)(k + 1) * N);
    double2* H = c.scratch<double2>(nm("kc_H", l, sz), (size_t)N * (k + 1) * k);
    double* cs = c.scratch<double>(nm("kc_cs", l, sz), (size_t)N * k);
    double2* sn = c.scratch<double2>(nm("kc_sn", l, sz), (size_t)N * k);
    double2* g = c.scratch<double2>(nm("kc_g", l, sz), (size_t)N * (k + 1));
    // own partials: the caller's FGMRES holds the pointer of its "part_md" across this call
    double2* part = c.scratch<double2>(nm("kc_part", l, sz), (size_t)reduce_groups(n, N) * (k + 1) * N);
    double* npart = c.scratch<double>(nm("kc_npart", l, sz), (size_t)axpy_groups(n, N) * N);
    norms<C>(c, beta, r, n, N);
    launch_scale_rhs<C, C>(V, r, beta, true, n, N, c.stream);
    launch_init_g(g, beta, k, N, c.stream);
    for (int j = 0; j < k; ++j) {
        C* Vj = V + (size_t)j * nN;
        C* Vn = V + (size_t)(j + 1) * nN;
        C* Zj = Z + (size_t)j * nN;
        mg_cycle<C>(c, l, Zj, Vj, N);
        apply_D<C>(c, l, Vn, Zj, nullptr, N, 0, nullptr);
        {
            ProfScope ps(c, "orth." + std::string(prec_tag(sz)), (j + 1) * (double)nN * sz,
                         2.0 * 8.0 * (j + 1) * (double)nN, (2 * j + 5) * (double)nN * sz);
            launch_multidot<C>(h, V, j + 1, Vn, n, N, part, c.stream);
            launch_multiaxpy_norm2<C>(Vn, h, j + 1, V, -1.0, n, N, hnorm, npart, c.stream);
        }
        sqrt_inplace(c, hnorm, N);
        if (j + 1 < k) launch_scale_rhs<C, C>(Vn, Vn, hnorm, true, n, N, c.stream);
        launch_arnoldi_column(H, cs, sn, g, resid, h, hnorm, j, k, N, c.stream);
    }
    launch_back_substitute(y, H, g, k - 1, k, N, c.stream);
    launch_multiaxpy<C>(e, y, k, Z, 1.0, n, N, c.stream, nullptr, 0, false);   // e = Z y
}

template <typename C>
void mg_cycle(Ctx& c, int l, C* e, const C* r, int N) {
    if (l == c.L - 1) {
        coarsest_apply<C>(c, e, r, N);
        return;
    }
    const Level& L = c.lev[l];
    const Level& Lc = c.lev[l + 1];
    C* res = c.scratch<C>(nm("cyc_res", l, sizeof(C)), (size_t)L.n * N);
    C* rc = c.scratch<C>(nm("cyc_rc", l + 1, sizeof(C)), (size_t)Lc.n * N);
    C* ec = c.scratch<C>(nm("cyc_ec", l + 1, sizeof(C)), (size_t)Lc.n * N);
    bool e_zero = true;
    if (c.opt.nu_pre > 0) {
        MG_CUDA(cudaMemcpyAsync(res, r, sizeof(C) * L.n * N, cudaMemcpyDeviceToDevice, c.stream));
        mr_smooth<C>(c, l, e, res, N, c.opt.nu_pre, true, true);   // leaves res = r - D e
        e_zero = false;
        apply_restrict<C>(c, l, rc, res, N);
    } else {
        apply_restrict<C>(c, l, rc, r, N);
    }
    if (c.opt.kcycle_iters > 0 && l + 2 < c.L)
        kcycle<C>(c, l + 1, ec, rc, N, c.opt.kcycle_iters);
    else
        mg_cycle<C>(c, l + 1, ec, rc, N);
    apply_prolong<C>(c, l, e, ec, N, !e_zero);
    if (c.opt.nu_post > 0 && !residual_smooth_tc<C>(c, l, e, r, N)) {
        apply_D<C>(c, l, res, e, r, N, 1, nullptr);
        mr_smooth<C>(c, l, e, res, N, c.opt.nu_post, false, false);
    }
}

static double read_scalar(Ctx& c, const double* dev) {
    MG_CUDA(cudaMemcpyAsync(c.hbuf, dev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    return c.hbuf[0];
}

template <typename C>
long long fgmres(Ctx& c, int l, const C* b, C* x, int N, double tol, long long maxit, bool x_zero, int* ok,
                 int max_cycles) {
    const Level& L = c.lev[l];
    const long long n = L.n;
    const int m = c.opt.fgmres_restart;
    const size_t nN = (size_t)n * N;
    const size_t sz = sizeof(C);
    C* V = c.scratch<C>(nm("fg_V", 0, sz), (size_t)(m + 1) * nN);
    C* Z = c.scratch<C>(nm("fg_Z", 0, sz), (size_t)m * nN);
    double* bnorm = c.scratch<double>(nm("fg_bn", 0, sz), N);
    double* beta = c.scratch<double>(nm("fg_beta", 0, sz), N);
    double* hnorm = c.scratch<double>(nm("fg_hn", 0, sz), N);
    double* resid = c.scratch<double>(nm("fg_res", 0, sz), N);
    double* maxr = c.scratch<double>(nm("fg_maxr", 0, sz), 1);
    double2* h = c.scratch<double2>(nm("fg_h", 0, sz), (size_t)(m + 1) * N);
    double2* h2 = c.scratch<double2>(nm("fg_h2", 0, sz), (size_t)(m + 1) * N);
    double2* y = c.scratch<double2>(nm("fg_y", 0, sz), (size_t)(m + 1) * N);
    double2* H = c.scratch<double2>(nm("fg_H", 0, sz), (size_t)N * (m + 1) * m);
    double* cs = c.scratch<double>(nm("fg_cs", 0, sz), (size_t)N * m);
    double2* sn = c.scratch<double2>(nm("fg_sn", 0, sz), (size_t)N * m);
    double2* g = c.scratch<double2>(nm("fg_g", 0, sz), (size_t)N * (m + 1));
    double2* part = c.scratch<double2>("part_md", (size_t)reduce_groups(n, N) * (m + 1) * N);

    // The Arnoldi basis is kept unnormalised, w_i = eta_i v_i with eta_i = |w_i| per rhs
    // (eta: (m + 1) x N): the Gram-Schmidt coefficients are divided by eta_i^2, the
    // Hessenberg column by eta_i eta_j, and the correction takes y_j / eta_j of z_j =
    // M(w_j).  This is FGMRES on the normalised basis exactly (the preconditioner of
    // each step is whatever maps v_j to z_j / eta_j: no property of M is assumed) and
    // saves the pass that would scale each new vector.  A vector whose eta leaves
    // [2^-32, 2^32] (an iteration run on past convergence shrinks it by the FP32
    // rounding level each step) is rescaled to unit norm, only for that rhs.
    double* eta = c.scratch<double>(nm("fg_eta", 0, sz), (size_t)(m + 1) * N);
    double* rsc = c.scratch<double>(nm("fg_rsc", 0, sz), N);
    MG_REQUIRE(b != V || (x_zero && max_cycles == 1), MGMLMC_EINVAL,
               "fgmres: a right-hand side in the basis needs x = 0 and one cycle");
    norms<C>(c, bnorm, b, n, N);
    // x = 0 is not written: the first correction overwrites x (or x is zeroed on exit)
    bool x_unset = x_zero;
    long long it = 0;
    int cycles = 0;
    *ok = 0;
    for (;;) {
        if (x_unset) {
            if (b != V) MG_CUDA(cudaMemcpyAsync(V, b, sz * nN, cudaMemcpyDeviceToDevice, c.stream));
            MG_CUDA(cudaMemcpyAsync(eta, bnorm, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream));
        } else {
            apply_D<C>(c, l, V, x, b, N, 1, nullptr);
            norms<C>(c, eta, V, n, N);
        }
        launch_max_ratio(maxr, eta, bnorm, N, c.stream);
        const double ratio = read_scalar(c, maxr);
        if (ratio != ratio) throw Error(MGMLMC_ENAN, "FGMRES: NaN residual");
        if (c.opt.verbose)
            fprintf(stderr, "[mgmlmc] fgmres level %d prec %zu it %lld true rel res %.3e\n", l + 1, sz * 4, it,
                    ratio);
        if (ratio <= tol) {
            *ok = 1;
            break;
        }
        if (it >= maxit) break;
        launch_init_g(g, eta, m, N, c.stream);
        k_eta_range<<<(N + 127) / 128, 128, 0, c.stream>>>(eta, rsc, N);
        MG_LAUNCHED();
        launch_scale_cols_if<C>(V, rsc, n, N, c.stream);
        int j_end = -1;
        // Inner cycles of the refinement loop converge in a repeatable number of steps
        // per level and tolerance: the host reads the residual estimate (a round trip
        // that leaves the GPU idle) only from two steps before the last such count on.
        int* hint = nullptr;
        if (max_cycles == 1) {
            const int dec = std::min(15, std::max(0, (int)std::floor(-std::log10(tol))));
            hint = &c.cycle_hint[((long long)l * 16 + dec) * (1LL << 32) + N];
        }
        const int check_from = hint ? std::max(1, *hint - 2) : 1;
        for (int j = 0; j < m; ++j) {
            C* Vj = V + (size_t)j * nN;
            C* Vn = V + (size_t)(j + 1) * nN;
            C* Zj = Z + (size_t)j * nN;
            mg_cycle<C>(c, l, Zj, Vj, N);
            apply_D<C>(c, l, Vn, Zj, nullptr, N, 0, nullptr);
            // classical Gram-Schmidt: twice in FP64; once in the FP32 inner solve of the
            // refinement loop, whose FP64 residual absorbs the loss of orthogonality
            {
                // algorithmic bytes: the j+1 basis vectors read once per Gram-Schmidt pass;
                // the implementation reads them twice (dot products, then the update) and
                // reads w twice and writes it once per pass: (2j + 5) vectors
                const int passes = (sz == sizeof(double2)) ? 2 : 1;
                ProfScope ps(c, "orth." + std::string(prec_tag(sz)), passes * (j + 1) * (double)nN * sz,
                             passes * 2.0 * 8.0 * (j + 1) * (double)nN, passes * (2 * j + 5) * (double)nN * sz);
                // the last axpy also returns |Vn|^2 (its partials), saving a pass over Vn
                double* npart = c.scratch<double>("part_nrm_ax", (size_t)axpy_groups(n, N) * N);
                launch_multidot<C>(h, V, j + 1, Vn, n, N, part, c.stream);
                if (passes == 2) {
                    launch_multiaxpy<C>(Vn, h, j + 1, V, -1.0, n, N, c.stream, eta, 2);
                    launch_multidot<C>(h2, V, j + 1, Vn, n, N, part, c.stream);
                    launch_multiaxpy_norm2<C>(Vn, h2, j + 1, V, -1.0, n, N, hnorm, npart, c.stream, eta, 2,
                                              eta + (size_t)j * N);
                    k_add2<<<((j + 1) * N + 127) / 128, 128, 0, c.stream>>>(h, h2, (j + 1) * N);
                    MG_LAUNCHED();
                } else {
                    launch_multiaxpy_norm2<C>(Vn, h, j + 1, V, -1.0, n, N, hnorm, npart, c.stream, eta, 2,
                                              eta + (size_t)j * N);
                }
            }
            k_lazy_column<<<(N + 127) / 128, 128, 0, c.stream>>>(h, hnorm, eta, rsc, j, N);
            MG_LAUNCHED();
            launch_scale_cols_if<C>(Vn, rsc, n, N, c.stream);
            launch_arnoldi_column(H, cs, sn, g, resid, h, hnorm, j, m, N, c.stream);
            ++it;
            j_end = j;
            if (j + 1 < check_from && j + 1 < m && it < maxit) continue;
            launch_max_ratio(maxr, resid, bnorm, N, c.stream);
            const double est = read_scalar(c, maxr);
            if (est != est) throw Error(MGMLMC_ENAN, "FGMRES: NaN in Arnoldi");
            if (est <= tol || it >= maxit) break;
        }
        if (hint) *hint = j_end + 1;
        launch_back_substitute(y, H, g, j_end, m, N, c.stream);
        launch_multiaxpy<C>(x, y, j_end + 1, Z, 1.0, n, N, c.stream, eta, 1, !x_unset);
        x_unset = false;
        if (++cycles >= max_cycles) {
            // the caller checks the residual itself (inner solve of the refinement loop)
            *ok = 1;
            break;
        }
    }
    if (x_unset) launch_zero<C>(x, (long long)nN, c.stream);
    return it;
}

// The Krylov basis block of fgmres<C> for N right-hand sides on level l: a caller that
// builds its rhs there (x = 0, one cycle) saves the copy into the basis.
template <typename C>
static C* fgmres_basis(Ctx& c, int l, int N) {
    return c.scratch<C>(nm("fg_V", 0, sizeof(C)), (size_t)(c.opt.fgmres_restart + 1) * c.lev[l].n * N);
}

static long long solve_block(Ctx& c, int l, const double2* b, double2* x, int N, double tol, int* ok);

// Blocks wider than opt.max_block_rhs (the eigensolvers' subspaces) are solved in
// column chunks of at most that width, so the Krylov work space stays bounded.
long long solve(Ctx& c, int l, const double2* b, double2* x, int N, double tol, int* ok) {
    const int blk = c.opt.max_block_rhs;
    if (N <= blk) return solve_block(c, l, b, x, N, tol, ok);
    const long long n = c.lev[l].n;
    double2* bb = c.scratch<double2>("sv_chunk_b", (size_t)n * blk);
    double2* xb = c.scratch<double2>("sv_chunk_x", (size_t)n * blk);
    const size_t w = sizeof(double2);
    long long it = 0;
    int all = 1;
    for (int j0 = 0; j0 < N; j0 += blk) {
        const int nb = std::min(blk, N - j0);
        MG_CUDA(cudaMemcpy2DAsync(bb, nb * w, b + j0, (size_t)N * w, nb * w, (size_t)n, cudaMemcpyDeviceToDevice,
                                  c.stream));
        int okb = 0;
        it += solve_block(c, l, bb, xb, nb, tol, &okb);
        all &= okb;
        MG_CUDA(cudaMemcpy2DAsync(x + j0, (size_t)N * w, xb, nb * w, nb * w, (size_t)n, cudaMemcpyDeviceToDevice,
                                  c.stream));
    }
    *ok = all;
    c.last_iters = it;
    return it;
}

static long long solve_block(Ctx& c, int l, const double2* b, double2* x, int N, double tol, int* ok) {
    const long long maxit = c.opt.max_iters;
    if (c.opt.mg_precision == 64) {
        const long long it = fgmres<double2>(c, l, b, x, N, tol, maxit, true, ok, 1 << 30);
        c.last_iters = it;
        return it;
    }
    // Mixed: FP64 iterative refinement, FP32 FGMRES + FP32 multigrid inside.
    const Level& L = c.lev[l];
    const long long n = L.n;
    const size_t nN = (size_t)n * N;
    double2* r = c.scratch<double2>("ir_r", nN);
    // the FP32 rhs of each inner cycle is built in the inner FGMRES's first basis vector
    float2* r32 = fgmres_basis<float2>(c, l, N);
    float2* e32 = c.scratch<float2>("ir_e32", nN);
    double* bnorm = c.scratch<double>("ir_bn", N);
    double* rnorm = c.scratch<double>("ir_rn", N);
    double* maxr = c.scratch<double>("ir_maxr", 1);
    // inner tolerance: the reduction still needed this cycle (with margin), but no
    // tighter than FP32 arithmetic can deliver
    const double inner_floor = 2e-7;
    // In the estimator's solves (c.fp32_residual_updates) the next residual comes from an
    // FP32 product, r <- r - |r| D e, between FP64 ones.  Its error against
    // the FP64 residual b - D x is below kFp32Product ||D|| |e| |r| (rounding of the FP32
    // operator and of the product's sums), with ||D_l|| <= ||D_1|| <= |m0 + 2| + 4 (each
    // hopping term has norm 1, the prolongators have orthonormal columns).  On the 256^2
    // workload the errors measured at the FP64 recomputations were 11 to 14 times below
    // this bound on all levels (verbose mode prints both).  |e| carries the
    // cancellation: a correction much longer than its residual (a rhs near the
    // near-kernel, as in the setup's inverse iteration) makes the FP32 product inexact.
    // drift bounds the error accumulated since the last FP64 residual (relative to |b|,
    // max over the rhs); the FP64 residual is recomputed once drift exceeds 1 % of the
    // residual, and for the convergence decision unless drift is below tol / 20.  Cycles
    // that reduce the residual a little then share one FP64 residual, which on a coarse
    // level costs as much as tens of FP32 products (d = 16: 1/64 of the FP32 FMA rate).
    // Every other solve (the setup's inverse iteration and the eigensolvers, whose
    // right-hand sides lie near the near-kernel) takes the FP64 residual after every
    // cycle but the last: below 500 tol the FP32 product's error (under 1e-4 |r|) stays
    // below tol / 20 of |b|.
    constexpr double kFp32Product = 4.0 * 0x1p-24;
    constexpr double kRecursiveResidual = 500.0;
    const bool fp32_updates = c.fp32_residual_updates;
    const double dnorm = std::fabs(c.m0 + 2.0) + 4.0;
    double* enorm = c.scratch<double>("ir_en", N);
    double drift = 0.0;
    norms<double2>(c, bnorm, b, n, N);
    launch_zero<double2>(x, (long long)nN, c.stream);
    MG_CUDA(cudaMemcpyAsync(r, b, sizeof(double2) * nN, cudaMemcpyDeviceToDevice, c.stream));
    long long it = 0;
    *ok = 0;
    // cycles until the FP64 residual meets tol or the iteration budget is spent
    for (int cycle = 0;; ++cycle) {
        norms<double2>(c, rnorm, r, n, N);
        launch_max_ratio(maxr, rnorm, bnorm, N, c.stream);
        const double ratio = read_scalar(c, maxr);
        if (ratio != ratio) throw Error(MGMLMC_ENAN, "refinement: NaN residual");
        if (drift > 0.0 && (drift > 1e-2 * ratio || (ratio <= tol && drift > tol / 20))) {
            double2* rrec = nullptr;
            if (c.opt.verbose) {
                rrec = c.scratch<double2>("ir_rrec", nN);
                MG_CUDA(cudaMemcpyAsync(rrec, r, sizeof(double2) * nN, cudaMemcpyDeviceToDevice, c.stream));
            }
            apply_D<double2>(c, l, r, x, b, N, 1, nullptr);
            if (rrec) {
                // the error the FP32 updates actually made, against the bound
                launch_axpy_rhs<double2, double2>(rrec, nullptr, nullptr, -1.0, r, n, N, c.stream);
                norms<double2>(c, rnorm, rrec, n, N);
                launch_max_ratio(maxr, rnorm, bnorm, N, c.stream);
                fprintf(stderr, "[mgmlmc] refine level %d FP64 residual: FP32 drift %.3e (bound %.3e)\n", l + 1,
                        read_scalar(c, maxr), drift);
            }
            drift = 0.0;
            continue;
        }
        if (c.opt.verbose)
            fprintf(stderr, "[mgmlmc] refine level %d cycle %d it %lld rel res %.3e\n", l + 1, cycle, it, ratio);
        if (ratio <= tol) {
            *ok = 1;
            break;
        }
        if (it >= maxit) break;
        launch_scale_rhs<float2, double2>(r32, r, rnorm, true, n, N, c.stream);
        const double inner_tol = std::max(inner_floor, 0.3 * tol / ratio);
        int iok = 0;
        // one FGMRES cycle in FP32: its own FP32 residual cannot certify more than
        // ~1e-6 relative, so the FP64 residual of this loop decides on restarts
        it += fgmres<float2>(c, l, r32, e32, N, inner_tol, maxit - it, true, &iok, 1);
        launch_axpy_rhs<double2, float2>(x, nullptr, rnorm, 1.0, e32, n, N, c.stream);
        if (!fp32_updates && ratio > kRecursiveResidual * tol) {
            apply_D<double2>(c, l, r, x, b, N, 1, nullptr);
            continue;
        }
        float2* de = c.scratch<float2>("ir_de32", nN);
        apply_D<float2>(c, l, de, e32, nullptr, N, 0, nullptr);
        launch_axpy_rhs<double2, float2>(r, nullptr, rnorm, -1.0, de, n, N, c.stream);
        if (!fp32_updates) continue;   // the last cycle: accepted on this residual
        // the bound of this update: max_j |e_j| |r_j| / |b_j|
        norms<float2>(c, enorm, e32, n, N);
        k_max_scaled_ratio<<<1, 256, 0, c.stream>>>(maxr, enorm, rnorm, bnorm, N);
        MG_LAUNCHED();
        drift += kFp32Product * dnorm * read_scalar(c, maxr);
    }
    c.last_iters = it;
    check_device_error(c);
    return it;
}

void check_device_error(Ctx& c) {
    if (!c.dev_err) return;
    int h = 0;
    MG_CUDA(cudaMemcpyAsync(&h, c.dev_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    if (h) {
        MG_CUDA(cudaMemsetAsync(c.dev_err, 0, sizeof(int), c.stream));
        throw Error(MGMLMC_ETIMEOUT, "a tensor-core kernel gave up waiting on an mbarrier (bounded wait)");
    }
}

#define INST(C)                                                                                           \
    template void apply_D<C>(Ctx&, int, C*, const C*, const C*, int, int, double2*);                        \
    template void apply_restrict<C>(Ctx&, int, C*, const C*, int);                                          \
    template void apply_prolong<C>(Ctx&, int, C*, const C*, int, bool);                                     \
    template void mg_cycle<C>(Ctx&, int, C*, const C*, int);                                                \
    template void apply_smoother_operator<C>(Ctx&, int, C*, const C*, int, double2*);                       \
    template long long fgmres<C>(Ctx&, int, const C*, C*, int, double, long long, bool, int*, int);
INST(double2)
INST(float2)

}  // namespace mg

namespace mg {
void column_norms(Ctx& c, double* out, const double2* x, long long n, int N) { norms<double2>(c, out, x, n, N); }

void approx_inverse(Ctx& c, int l, const double2* b, double2* x, int N) {
    int ok = 0;
    if (c.opt.mg_precision == 64) {
        fgmres<double2>(c, l, b, x, N, 1e-14, c.opt.fgmres_restart, true, &ok, 1);
        return;
    }
    const size_t nN = (size_t)c.lev[l].n * N;
    float2* b32 = c.scratch<float2>("ai_b32", nN);
    float2* x32 = c.scratch<float2>("ai_x32", nN);
    launch_convert<float2, double2>(b32, b, (long long)nN, c.stream);
    fgmres<float2>(c, l, b32, x32, N, 1e-6, c.opt.fgmres_restart, true, &ok, 1);
    launch_convert<double2, float2>(x, x32, (long long)nN, c.stream);
}
}  // namespace mg
