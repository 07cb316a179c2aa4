// Host-side launchers of every kernel of the library.  Vectors are blocks of N
// right-hand sides stored [row][rhs] (rhs fastest, row = site * d + dof), so a
// warp reads 32 consecutive right-hand sides of one row: fully coalesced.
// Per-rhs reductions are deterministic two-pass: each block writes partial
// sums to a scratch array [group][...][N], a second kernel adds them in a fixed
// order.
#pragma once

#include "common.cuh"

namespace mg {

// Neighbour of a coarse site in direction dir of the 5-point block stencil:
// 0 self, 1 +x, 2 -x, 3 +t, 4 -t (periodic wrap; sites are x-fastest).
__device__ __forceinline__ int nbr_site(int site, int dir, int lx, int lt) {
    const int xx = site % lx, t = site / lx;
    switch (dir) {
        case 1: return (xx + 1 == lx ? 0 : xx + 1) + lx * t;
        case 2: return (xx == 0 ? lx - 1 : xx - 1) + lx * t;
        case 3: return xx + lx * (t + 1 == lt ? 0 : t + 1);
        case 4: return xx + lx * (t == 0 ? lt - 1 : t - 1);
        default: return site;
    }
}

// ---------------------------------------------------------------- vectors
// Z2 noise block: x[i][j] = +-1 (imag 0) for sample first+j, entry i (Sect. 1).
template <typename C>
void launch_noise(C* x, long long n, int N, uint64_t seed, uint64_t term, int64_t first, cudaStream_t s);
// x[i][j] = probes[j][i] (host-supplied probe vectors already on the device).
template <typename C>
void launch_probes(C* x, const int8_t* probes, long long n, int N, cudaStream_t s);
template <typename Cout, typename Cin>
void launch_convert(Cout* y, const Cin* x, long long count, cudaStream_t s);
// y[i][j] = scale[j] * x[i][j] (scale real, per rhs); scale may be inverted (1/scale, 0 if scale == 0)
template <typename Cy, typename Cx_>
void launch_scale_rhs(Cy* y, const Cx_* x, const double* scale, bool invert, long long n, int N, cudaStream_t s);
// w[:, j] *= s[j] where s[j] != 0 (other columns untouched).
template <typename C>
void launch_scale_cols_if(C* w, const double* s, long long n, int N, cudaStream_t st);
// y[i][j] += sign * alpha[j] * x[i][j]  (alpha complex per rhs, optionally times real beta[j])
template <typename Cy, typename Cx_>
void launch_axpy_rhs(Cy* y, const double2* alpha, const double* beta, double sign, const Cx_* x,
                     long long n, int N, cudaStream_t s);
template <typename C>
void launch_zero(C* x, long long count, cudaStream_t s);
// out[c][r] = in[r][c] (rows x cols complex, row-major)
void launch_transpose(double2* out, const double2* in, long long rows, int cols, cudaStream_t s);

// ------------------------------------------------------------- reductions
// Number of row groups (partials) used by the reduction kernels for (n, N).
int reduce_groups(long long n, int N);
// Row groups of launch_multiaxpy(_norm2): size of the norm partials is axpy_groups * N.
int axpy_groups(long long n, int N);
// out[j] = sum_i conj(x[i][j]) * y[i][j]  (double2), via scratch part[groups][N]
template <typename Cx_, typename Cy>
void launch_dot(double2* out, const Cx_* x, const Cy* y, long long n, int N, double2* part, cudaStream_t s);
// out[j] = sum_i |x[i][j]|^2
template <typename C>
void launch_norm2(double* out, const C* x, long long n, int N, double* part, cudaStream_t s);
// out[k][j] = <V_k, w>_j for k < m; V_k = V + k * n * N.  part: [groups][m][N].
template <typename C>
void launch_multidot(double2* out, const C* V, int m, const C* w, long long n, int N, double2* part,
                     cudaStream_t s);
// w[i][j] = (accumulate ? w[i][j] : 0) + sign * sum_k c[k][j] V_k[i][j], with
// c[k][j] = coef[k][j], or coef[k][j] / eta[k][j]^eta_pow (eta_pow 1 or 2; 0 where eta is 0)
// when eta is given: the coefficients of unnormalised basis vectors V_k = eta_k v_k.
template <typename C>
void launch_multiaxpy(C* w, const double2* coef, int m, const C* V, double sign, long long n, int N,
                      cudaStream_t s, const double* eta = nullptr, int eta_pow = 0, bool accumulate = true);
// As launch_multiaxpy (accumulating), and norm2[j] = |w_j / norm_div[j]|^2 of the updated
// w (norm_div NULL or 0: 1; part: axpy_groups(n, N) * N scratch).
template <typename C>
void launch_multiaxpy_norm2(C* w, const double2* coef, int m, const C* V, double sign, long long n, int N,
                            double* norm2, double* part, cudaStream_t s, const double* eta = nullptr,
                            int eta_pow = 0, const double* norm_div = nullptr);
// Sum of partials: out[j] = sum_g part[g][j] (count = values per group).
void launch_finalize(double2* out, const double2* part, int groups, int count, cudaStream_t s);
void launch_finalize(double* out, const double* part, int groups, int count, cudaStream_t s);
// Row-major partials (the stencils' minimal-residual dots): out[i] = sum_g part[i * groups + g].
void launch_finalize_rows(double2* out, const double2* part, int groups, int count, cudaStream_t s);

// --------------------------------------------------------------- stencils
// Fine Wilson-Schwinger operator (2 spins, U(1) links U[site][mu]).
//  mode 0: y = D x;  mode 1: y = b - D x;
//  mode 2: y = D x and part[0][j][g] = <y, x>_j, part[1][j][g] = <y, y>_j (MR smoother;
//          row-major in the group index g = blockIdx.y, see launch_finalize_rows)
template <typename C>
void launch_wilson(C* y, const C* x, const C* b, const C* U, double m0, int lx, int lt, int N,
                   int mode, double2* part, int groups, cudaStream_t s);
// Fine-level smoother in BF16 (one bf16x2 word per complex value, [row][rhs]):
// y = D x with per-rhs dots conj(y).x, |y|^2 (partials as launch_wilson mode 2; N % 4 == 0),
// the FP32 -> BF16 conversion, and e (=|+=) alpha r, r -= alpha p (r in place).
void launch_wilson_bf16(uint32_t* y, const uint32_t* x, const float2* U, double m0, int lx, int lt, int N,
                        double2* part, int groups, cudaStream_t s);
void launch_pack_bf16(uint32_t* y, const float2* x, long long count, cudaStream_t s);
void launch_mr_update_fine_bf16(float2* e, uint32_t* r, const uint32_t* p, const double2* dots, long long n, int N,
                                bool e_is_zero, cudaStream_t s);
// Coarse 5-point block stencil y_s = sum_dir A[s][dir] x_nbr(s,dir), d x d complex blocks,
// dir = 0 self, 1 +x, 2 -x, 3 +t, 4 -t (periodic; boundary signs live in the blocks).
template <typename C>
void launch_block_stencil(C* y, const C* x, const C* b, const C* A, int lx, int lt, int d, int N,
                          int mode, double2* part, int groups, cudaStream_t s);
int stencil_groups(int nsites, int N);
// Row groups (partials) of launch_wilson_bf16.
int stencil_groups_bf16(int nsites, int N);
// Row groups (grid.y) the block-stencil launcher expects for (nsites, d, N); the MR
// partials array holds groups * 2 * N values.
int block_stencil_groups(int nsites, int d, int N);
// Restriction xc = P^H x and prolongation x (+)= P xc for aggregates ax x at,
// P stored [fine site][d][nvec]; coarse dof (S, spin block, j).
template <typename C>
void launch_restrict(C* xc, const C* x, const C* P, int lx, int lt, int d, int ax, int at, int nvec,
                     int N, cudaStream_t s);
template <typename C>
void launch_prolong(C* x, const C* xc, const C* P, int lx, int lt, int d, int ax, int at, int nvec,
                    int N, bool accumulate, cudaStream_t s);
// MR update: alpha_j = <p,r>/<p,p> from dots[2][N]; e += alpha r; r -= alpha p.
template <typename C>
void launch_mr_update(C* e, C* r, const C* p, const double2* dots, long long n, int N, bool e_is_zero,
                      cudaStream_t s);
// Gamma5 on a level with d dof per site: +1 on the first d/2 dof, -1 on the rest.
template <typename C>
void launch_gamma5(C* y, const C* x, long long nsites, int d, int N, cudaStream_t s);

// ----------------------------------------------------------------- dense
// C[M][Nc] = A[M][K] * B[K][Nc] (+ C if accumulate), complex, row-major.
template <typename C>
void launch_gemm_nn(C* Cm, const C* A, const C* B, int M, int K, int Nc, bool accumulate, cudaStream_t s);
// C[ka][kb] = A^H B for A [n][ka], B [n][kb] (reduction over n, deterministic two-pass).
template <typename C>
void launch_gemm_hn(double2* Cm, const C* A, const C* B, long long n, int ka, int kb, double2* part,
                    int groups, cudaStream_t s);
int gemm_hn_groups(long long n, int ka, int kb);
// The same two products with FP64 storage and FP32 arithmetic (the eigensolvers'
// block operations on large levels; the partial sums of at most 16384 rows are
// FP32, their sum FP64).  part: gemm_hn_fp32_groups(...) * ka * kb values.
void launch_gemm_nn_fp32(double2* Cm, const double2* A, const double2* B, int M, int K, int Nc, cudaStream_t s);
void launch_gemm_hn_fp32(double2* Cm, const double2* A, const double2* B, long long n, int ka, int kb,
                         double2* part, int groups, cudaStream_t s);
int gemm_hn_fp32_groups(long long n, int ka, int kb);
// In-place Gauss-Jordan inverse of a dense complex n x n matrix (partial pivoting).
// work: n doubles + n ints + a few scalars.  Returns via *status_dev 0 ok, 1 singular.
template <typename C>
void launch_gauss_jordan(C* A, int n, void* work, cudaStream_t s);
size_t gauss_jordan_work_bytes(int n);
// Hermitian eigenproblem of a b x b matrix (b <= 2048; cyclic Jacobi in one
// cooperative kernel over all SMs, round-robin pairs, one bounded grid barrier per
// round): H is read, W receives the eigenvectors (columns) and lam the eigenvalues,
// sorted by increasing |lambda| (decreasing with descending).  work: at least
// jacobi_work_bytes(b), 256-byte aligned.  err (may be null) is set to 1 if a grid
// barrier gave up waiting.
void launch_jacobi_eig(double2* H, double2* W, double* lam, int b, int sweeps, void* work, int* err, cudaStream_t s,
                       bool descending = false);
size_t jacobi_work_bytes(int b);
size_t jacobi_smem_bytes(int b);
// G (b x b, Hermitian positive definite) = R^H R; Rinv = R^{-1} (upper triangular),
// one cooperative kernel over all SMs (G is overwritten).  status[0] = 1 if G was
// not positive definite; err (may be null) = 1 if a grid barrier gave up waiting.
// work: cholesky_work_bytes(b).
size_t cholesky_work_bytes(int b);
void launch_cholesky_inv(double2* G, double2* Rinv, int b, void* work, int* status, int* err, cudaStream_t s);
// BF16 real embedding [Re A | Im A] (n x 2n) of a complex FP32 n x n matrix for the
// tensor-core coarsest solve.
void launch_embed_bf16(__nv_bfloat16* E, const float2* A, int n, cudaStream_t s);
bool tc_coarse_supported(int n);
// Y[n][N] = A * X with the BF16 embedding E of A (tcgen05 tensor cores, FP32 accumulation);
// X, Y FP32 complex [n][N].  *err set to 1 if a bounded wait gave up.
void launch_coarse_inverse_bf16(float2* Y, const float2* X, const __nv_bfloat16* E, int n, int N,
                                void* scratch, int* err, cudaStream_t s);
size_t coarse_inverse_bf16_scratch(int n, int N);
// Deflation projections on the tensor cores: W (tc_deflation_rows(k) x n BF16,
// pre-tiled) holds [Re R | -Im R | Re L | -Im L]^T of the deflation's factors
// R, L [n][k]; launch_deflation_correction_bf16 forms A = R^H X and B = L^H X for
// a real block X [n][N] (FP32 accumulation) and does s[j] -= sum_m a_m conj(B) A.
// t[m] = R~_m^H L~_m over the BF16-rounded factors (FP64 sums).
bool tc_deflation_supported(long long n, int k);
int tc_deflation_rows(int k);
void launch_embed_deflation_bf16(__nv_bfloat16* W, const double2* R, const double2* L, long long n, int k,
                                 cudaStream_t s);
void launch_deflation_tau_bf16(double2* t, const double2* R, const double2* L, long long n, int k, cudaStream_t s);
size_t deflation_bf16_scratch(long long n, int k, int N);
void launch_deflation_correction_bf16(double2* smp, const double2* X, const __nv_bfloat16* W, const double* a,
                                      long long n, int k, int N, void* scratch, int* err, cudaStream_t s);
// Coarse block stencil (d = 16) on the tensor cores for the block-Jacobi
// smoother: E holds the blocks of every site and direction as BF16 real 32 x 32
// operands (launch_embed_stencil_bf16); the input x is given as BF16 tiles
// (per site and 128-rhs tile, 8 KB in the MMA's K-major layout, written by
// launch_pack_tiles_bf16 or launch_mr_update_tc).  y = A x in FP32 plus per-rhs
// dots conj(y).x, |y|^2 (partials as launch_block_stencil).  err: device flag set
// when a bounded wait gave up.
bool tc_stencil_supported(int d, int N);
void launch_embed_stencil_bf16(__nv_bfloat16* E, const float2* A, int nsites, cudaStream_t s);
size_t tc_tiles_bytes(int nsites, int N);
void launch_pack_tiles_bf16(__nv_bfloat16* rt, const float2* x, int nsites, int N, cudaStream_t s);
// yh (= or +=) alpha r, r -= alpha p with alpha = dots[j] / dots[N + j]; rt (may be
// null) receives the BF16 tiles of the new r.  d = 16.
void launch_mr_update_tc(float2* yh, float2* r, const float2* p, const double2* dots, int nsites, int N, bool first,
                         __nv_bfloat16* rt, cudaStream_t s);
// yh (= or +=) alpha r, r -= alpha p with r and p as BF16 tiles (r updated in place).
void launch_mr_update_bf16(float2* yh, __nv_bfloat16* rt, const __nv_bfloat16* pt, const double2* dots, int nsites,
                           int N, bool first, cudaStream_t s);
int block_stencil_tc_groups(int nsites, int N);
// Output: y (FP32 rows) or yt (BF16 tiles), exactly one non-null; with b (FP32 rows,
// yt only) the tiles receive the residual b - A x and no dots are formed.
void launch_block_stencil_tc(float2* y, __nv_bfloat16* yt, const float2* b, const __nv_bfloat16* xt,
                             const __nv_bfloat16* E, int lx, int lt, int N, double2* part, int groups, int* err,
                             cudaStream_t s);

// ----------------------------------------------------------------- setup
// Block-stencil form of the fine Wilson operator: A[site][5][2][2].
void launch_materialize_wilson(double2* A, const double2* U, double m0, int lx, int lt, cudaStream_t s);
// Galerkin coarse blocks Ac[S][5][dc][dc] = P^H D P, D given as block stencil Af (d x d);
// T: scratch of galerkin_scratch_count(...) complex values.
void launch_galerkin(double2* Ac, const double2* Af, const double2* P, int lx, int lt, int d, int ax,
                     int at, int nvec, double2* T, cudaStream_t s);
size_t galerkin_scratch_count(int lx, int lt, int d, int nvec);
// P[site][d][nvec] from test vectors tv[nvec][n]: MGS per (aggregate, spin block).
// status[0] set to 1 if a block is rank deficient.
void launch_build_prolongator(double2* P, const double2* tv, int lx, int lt, int d, int ax, int at,
                              int nvec, int* status, cudaStream_t s);
// Small per-rhs FGMRES bookkeeping (one thread per rhs).
void launch_arnoldi_column(double2* H, double* cs, double2* sn, double2* g, double* resid,
                           const double2* h, const double* hnorm, int j, int m, int N, cudaStream_t s);
void launch_back_substitute(double2* y, const double2* H, const double2* g, int j, int m, int N,
                            cudaStream_t s);
void launch_init_g(double2* g, const double* beta, int m, int N, cudaStream_t s);
// max over rhs of resid[j] / bnorm[j] -> out (device scalar)
void launch_max_ratio(double* out, const double* resid, const double* bnorm, int N, cudaStream_t s);
// samples: s[j] = sign * <x, z>_j + s[j] (accumulate) helpers live in the estimator.
void launch_deflation_correction(double2* s, const double2* A, const double2* B, const double* a, int k,
                                 int N, cudaStream_t s_);
void launch_sample_stats(double* acc, const double2* samples, int N, cudaStream_t s);
// Block-Jacobi smoother data: Minv[s] = A[s][0]^{-1} (work: nsites d^2 scratch) and the
// block stencil Ahat of D M^{-1} (Ahat[s][dir] = A[s][dir] Minv[nbr(s,dir)]).
void launch_block_diag_inverse(double2* Minv, double2* work, const double2* A, int nsites, int d, int* status,
                               cudaStream_t s);
void launch_precondition_blocks(double2* Ahat, const double2* A, const double2* Minv, int lx, int lt, int d,
                                cudaStream_t s);
// y[s] (+)= Minv[s] x[s] for every site (d x d complex blocks), N rhs.
template <typename C>
void launch_block_diag_apply(C* y, const C* x, const C* Minv, int nsites, int d, int N, bool accumulate,
                             cudaStream_t s);
// Dense [n][n] matrix of a 5-point block stencil (entries of coinciding neighbours add up).
void launch_dense_from_blocks(double2* Dd, const double2* A, int lx, int lt, int d, cudaStream_t s);

}  // namespace mg
