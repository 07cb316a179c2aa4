// Dense complex kernels: GEMM (C = A B), tall-skinny inner products (C = A^H B),
// in-place Gauss-Jordan inversion of the coarsest operator, and a one-CTA
// cyclic Jacobi eigensolver for the small Hermitian Rayleigh-Ritz problems of
// the deflation setup.  FP64 instances run on the FP64 pipe, FP32 on the FP32
// pipe; the BF16 tensor-core coarsest solve lives in kernels_tc.cu.
#include "kernels.cuh"

namespace mg {

// ------------------------------------------------------------------ GEMM nn
// Tile 64 x 32 (rows x cols), K step 16; thread (tx, ty) owns column tx and rows
// ty*8 .. ty*8+7.  All threads of a warp share ty, so A reads are broadcasts.
constexpr int GM = 64, GN = 32, GK = 16;

template <typename C>
__global__ void __launch_bounds__(256) k_gemm_nn(C* __restrict__ Cm, const C* __restrict__ A,
                                                 const C* __restrict__ B, int M, int K, int Nc, bool accumulate) {
    __shared__ C As[GM][GK + 1];
    __shared__ C Bs[GK][GN];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int row0 = blockIdx.y * GM, col0 = blockIdx.x * GN;
    C acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = czero<C>();
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = tid; e < GM * GK; e += 256) {
            const int r = e / GK, k = e % GK;
            const int gr = row0 + r, gk = k0 + k;
            As[r][k] = (gr < M && gk < K) ? A[(long long)gr * K + gk] : czero<C>();
        }
        for (int e = tid; e < GK * GN; e += 256) {
            const int k = e / GN, c = e % GN;
            const int gk = k0 + k, gc = col0 + c;
            Bs[k][c] = (gk < K && gc < Nc) ? B[(long long)gk * Nc + gc] : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            const C bv = Bs[k][tx];
#pragma unroll
            for (int r = 0; r < 8; ++r) cfma(acc[r], As[ty * 8 + r][k], bv);
        }
        __syncthreads();
    }
    const int gc = col0 + tx;
    if (gc >= Nc) return;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int gr = row0 + ty * 8 + r;
        if (gr < M) {
            const long long idx = (long long)gr * Nc + gc;
            Cm[idx] = accumulate ? cadd(Cm[idx], acc[r]) : acc[r];
        }
    }
}

// Narrow variant for few columns (the setup solves run 8 right-hand sides):
// tile 16 x 8 so that a 4096-row product still spreads over 256 CTAs; thread
// (tx < 8 column, ty < 16 row) owns one output.
template <typename C>
__global__ void __launch_bounds__(128) k_gemm_nn8(C* __restrict__ Cm, const C* __restrict__ A,
                                                  const C* __restrict__ B, int M, int K, int Nc, bool accumulate) {
    constexpr int ROWS = 16, KT = 64;
    __shared__ C As[ROWS][KT + 1];
    __shared__ C Bs[KT][8];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 8 + tx;
    const int row0 = blockIdx.y * ROWS, col0 = blockIdx.x * 8;
    C acc = czero<C>();
    for (int k0 = 0; k0 < K; k0 += KT) {
        for (int e = tid; e < ROWS * KT; e += 128) {
            const int r = e / KT, k = e % KT;
            const int gr = row0 + r, gk = k0 + k;
            As[r][k] = (gr < M && gk < K) ? A[(long long)gr * K + gk] : czero<C>();
        }
        for (int e = tid; e < KT * 8; e += 128) {
            const int k = e / 8, c = e % 8;
            const int gk = k0 + k, gc = col0 + c;
            Bs[k][c] = (gk < K && gc < Nc) ? B[(long long)gk * Nc + gc] : czero<C>();
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KT; ++k) cfma(acc, As[ty][k], Bs[k][tx]);
        __syncthreads();
    }
    const int gc = col0 + tx, gr = row0 + ty;
    if (gc < Nc && gr < M) {
        const long long idx = (long long)gr * Nc + gc;
        Cm[idx] = accumulate ? cadd(Cm[idx], acc) : acc;
    }
}

template <typename C>
void launch_gemm_nn(C* Cm, const C* A, const C* B, int M, int K, int Nc, bool accumulate, cudaStream_t s) {
    if (Nc <= 8) {
        dim3 g(1, (M + 15) / 16);
        k_gemm_nn8<C><<<g, dim3(8, 16), 0, s>>>(Cm, A, B, M, K, Nc, accumulate);
        MG_LAUNCHED();
        return;
    }
    dim3 g((Nc + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm_nn<C><<<g, dim3(32, 8), 0, s>>>(Cm, A, B, M, K, Nc, accumulate);
    MG_LAUNCHED();
}

// ------------------------------------------------------------------ GEMM hn
// part[g][a][b] = sum_{i in slice g} conj(A[i][a]) B[i][b]; tile 32 x 32, thread
// (tx = b, ty) owns a = ty*4 .. ty*4+3.
template <typename C>
__global__ void __launch_bounds__(256) k_gemm_hn(double2* __restrict__ part, const C* __restrict__ A,
                                                 const C* __restrict__ B, long long n, int ka, int kb,
                                                 long long slice) {
    __shared__ C As[16][33];
    __shared__ C Bs[16][33];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    const long long i_begin = (long long)blockIdx.z * slice;
    long long i_end = i_begin + slice;
    if (i_end > n) i_end = n;
    C acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = czero<C>();
    for (long long i0 = i_begin; i0 < i_end; i0 += 16) {
        for (int e = tid; e < 16 * 32; e += 256) {
            const int ii = e / 32, c = e % 32;
            const long long gi = i0 + ii;
            As[ii][c] = (gi < i_end && a0 + c < ka) ? A[gi * ka + a0 + c] : czero<C>();
            Bs[ii][c] = (gi < i_end && b0 + c < kb) ? B[gi * kb + b0 + c] : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < 16; ++ii) {
            const C bv = Bs[ii][tx];
#pragma unroll
            for (int r = 0; r < 4; ++r) cfmac(acc[r], As[ii][ty * 4 + r], bv);
        }
        __syncthreads();
    }
    const int b = b0 + tx;
    if (b >= kb) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int a = a0 + ty * 4 + r;
        if (a < ka) part[((long long)blockIdx.z * ka + a) * kb + b] = to_d(acc[r]);
    }
}

int gemm_hn_groups(long long n, int ka, int kb) {
    const long long tiles = (long long)((ka + 31) / 32) * ((kb + 31) / 32);
    long long g = (4LL * kNumSM) / tiles;
    if (g < 1) g = 1;
    const long long maxg = (n + 63) / 64;
    if (g > maxg) g = maxg;
    return (int)g;
}

template <typename C>
void launch_gemm_hn(double2* Cm, const C* A, const C* B, long long n, int ka, int kb, double2* part, int groups,
                    cudaStream_t s) {
    long long slice = (n + groups - 1) / groups;
    slice = ((slice + 15) / 16) * 16;
    dim3 g((kb + 31) / 32, (ka + 31) / 32, groups);
    k_gemm_hn<C><<<g, dim3(32, 8), 0, s>>>(part, A, B, n, ka, kb, slice);
    MG_LAUNCHED();
    launch_finalize(Cm, part, groups, ka * kb, s);
}

// ---------------------------------------------------------------- Gauss-Jordan
// In-place inversion with partial pivoting (Gauss-Jordan elimination in its
// textbook in-place form: for each k pick the largest |A[i][k]|, i >= k, swap it to
// row k, scale row k by 1/pivot with A[k][k] = 1 first, eliminate column k from every
// other row with A[i][k] = 0 first; at the end undo the row swaps as column swaps in
// reverse order), blocked by panels of GJPanel<C>::B columns S = [k0, k0 + kb).
// The steps of a panel touch only its own columns; their product T is the identity
// outside the columns S, and its columns S are what the panel columns hold after
// those steps.  The other columns then take the panel's row swaps and
// A[:, c] <- T A[:, c] = A[:, c] (rows S zeroed) + A[:, S] A[S, c], one complex GEMM
// of depth kb, so the whole matrix is streamed once per panel instead of once per
// column.
struct GJWork {
    int* perm;       // n
    double2* fcol;   // n   column k before elimination
    int* status;     // 1 = zero pivot met
    void* rows;      // B x n copy of the panel's pivot rows (type C)
};

template <typename C> struct GJPanel;
template <> struct GJPanel<float2> { static constexpr int B = 32; };
template <> struct GJPanel<double2> { static constexpr int B = 16; };

// Step k of the panel [k0, k0 + kb): pivot search in column k (rows >= k), swap rows
// k and p within the panel columns, scale the panel part of row k, save column k.
template <typename C>
__global__ void __launch_bounds__(1024) k_gj_pivot(C* A, int n, int k, int k0, int kb, GJWork w) {
    __shared__ double best[1024];
    __shared__ int bidx[1024];
    double bv = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const C v = A[(long long)i * n + k];
        const double m = (double)v.x * v.x + (double)v.y * v.y;
        if (m > bv) { bv = m; bi = i; }
    }
    best[threadIdx.x] = bv;
    bidx[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double o = best[threadIdx.x + st];
            const int oi = bidx[threadIdx.x + st];
            if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
                best[threadIdx.x] = o;
                bidx[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int p = bidx[0];
    if (threadIdx.x == 0) {
        w.perm[k] = p;
        if (!(best[0] > 0.0)) *w.status = 1;
    }
    if (p != k)
        for (int c = k0 + threadIdx.x; c < k0 + kb; c += blockDim.x) {
            const C t = A[(long long)k * n + c];
            A[(long long)k * n + c] = A[(long long)p * n + c];
            A[(long long)p * n + c] = t;
        }
    __syncthreads();
    C piv = A[(long long)k * n + k];
    if (!(best[0] > 0.0)) piv = mk((decltype(piv.x))1, (decltype(piv.x))0);
    const double2 pd = to_d(piv);
    const double den = pd.x * pd.x + pd.y * pd.y;
    const C inv = cvt<C>(make_double2(pd.x / den, -pd.y / den));
    __syncthreads();
    for (int c = k0 + threadIdx.x; c < k0 + kb; c += blockDim.x) {
        C v = (c == k) ? mk((decltype(piv.x))1, (decltype(piv.x))0) : A[(long long)k * n + c];
        A[(long long)k * n + c] = cmul(v, inv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) w.fcol[i] = to_d(A[(long long)i * n + k]);
}

// Elimination of column k from every other row, within the panel columns: one warp
// per row, lanes over the columns.
template <typename C>
__global__ void __launch_bounds__(256) k_gj_eliminate(C* A, int n, int k, int k0, int kb, GJWork w) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n || i == k) return;
    const C f = cvt<C>(w.fcol[i]);
    for (int c = k0 + lane; c < k0 + kb; c += 32) {
        const C pk = A[(long long)k * n + c];
        const long long idx = (long long)i * n + c;
        const C v = (c == k) ? czero<C>() : A[idx];
        A[idx] = csub(v, cmul(f, pk));
    }
}

// The panel's row swaps on the other columns (in the order they were taken), then a
// copy of the pivot rows R[s][c] = A[k0 + s][c]: one thread per column.
template <typename C>
__global__ void __launch_bounds__(256) k_gj_swap_rows(C* A, int n, int k0, int kb, GJWork w) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    C* R = reinterpret_cast<C*>(w.rows);
    const bool in_panel = c >= k0 && c < k0 + kb;
    for (int j = k0; j < k0 + kb; ++j) {
        const int p = w.perm[j];
        if (!in_panel && p != j) {
            const C t = A[(long long)j * n + c];
            A[(long long)j * n + c] = A[(long long)p * n + c];
            A[(long long)p * n + c] = t;
        }
        R[(long long)(j - k0) * n + c] = A[(long long)j * n + c];
    }
}

// A[i][c] = [i outside S] A[i][c] + sum_s A[i][k0 + s] R[s][c] for every column c
// outside the panel.  Tile 64 x 64, thread (tx, ty) owns rows ty + 16a and columns
// tx + 16b (a, b < 4); the panel columns are read, never written.
template <typename C, int B>
__global__ void __launch_bounds__(256) k_gj_update(C* A, int n, int k0, int kb, GJWork w) {
    __shared__ C Ts[64][B + 1];
    __shared__ C Rs[B][64];
    const C* R = reinterpret_cast<const C*>(w.rows);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * B; e += 256) {
        const int r = e / B, s = e % B, gr = row0 + r;
        Ts[r][s] = (gr < n && s < kb) ? A[(long long)gr * n + k0 + s] : czero<C>();
    }
    for (int e = threadIdx.x; e < B * 64; e += 256) {
        const int s = e / 64, cc = e % 64, gc = col0 + cc;
        Rs[s][cc] = (s < kb && gc < n) ? R[(long long)s * n + gc] : czero<C>();
    }
    __syncthreads();
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = czero<C>();
#pragma unroll 4
    for (int s = 0; s < B; ++s) {
        C t[4], r[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = Ts[ty + 16 * a][s];
#pragma unroll
        for (int b = 0; b < 4; ++b) r[b] = Rs[s][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cfma(acc[a][b], t[a], r[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = row0 + ty + 16 * a, c = col0 + tx + 16 * b;
            if (i >= n || c >= n || (c >= k0 && c < k0 + kb)) continue;
            const long long idx = (long long)i * n + c;
            const C old = (i >= k0 && i < k0 + kb) ? czero<C>() : A[idx];
            A[idx] = cadd(old, acc[a][b]);
        }
}

template <typename C>
__global__ void k_gj_unpermute(C* A, int n, GJWork w) {
    // column swaps in reverse order of the row swaps; one thread per row
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = n - 1; k >= 0; --k) {
        const int p = w.perm[k];
        if (p != k) {
            const C t = A[(long long)i * n + k];
            A[(long long)i * n + k] = A[(long long)i * n + p];
            A[(long long)i * n + p] = t;
        }
    }
}

// fcol (n double2) | perm (n int) | status | pad to 256 B | pivot rows (B x n, 256 n bytes
// for both instances: 32 x 8 B and 16 x 16 B per column)
static size_t gj_rows_offset(int n) { return (((size_t)n * sizeof(double2) + (size_t)n * sizeof(int) + 64) + 255) / 256 * 256; }
size_t gauss_jordan_work_bytes(int n) { return gj_rows_offset(n) + (size_t)n * 256 + 256; }

template <typename C>
void launch_gauss_jordan(C* A, int n, void* work, cudaStream_t s) {
    constexpr int B = GJPanel<C>::B;
    static_assert(B * sizeof(C) == 256, "pivot-row buffer is 256 bytes per column");
    GJWork w;
    w.fcol = reinterpret_cast<double2*>(work);
    w.perm = reinterpret_cast<int*>(w.fcol + n);
    w.status = w.perm + n;
    w.rows = reinterpret_cast<char*>(work) + gj_rows_offset(n);
    MG_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s));
    long long launches = 0;
    const dim3 tiles((n + 63) / 64, (n + 63) / 64);
    for (int k0 = 0; k0 < n; k0 += B) {
        const int kb = n - k0 < B ? n - k0 : B;
        for (int k = k0; k < k0 + kb; ++k) {
            k_gj_pivot<C><<<1, 1024, 0, s>>>(A, n, k, k0, kb, w);
            k_gj_eliminate<C><<<(n + 7) / 8, 256, 0, s>>>(A, n, k, k0, kb, w);
        }
        k_gj_swap_rows<C><<<(n + 255) / 256, 256, 0, s>>>(A, n, k0, kb, w);
        k_gj_update<C, B><<<tiles, 256, 0, s>>>(A, n, k0, kb, w);
        launches += 2LL * kb + 2;
    }
    launch_counter().fetch_add(launches - 1);
    MG_LAUNCHED();
    k_gj_unpermute<C><<<(n + 127) / 128, 128, 0, s>>>(A, n, w);
    MG_LAUNCHED();
}

// ------------------------------------------------------------- Jacobi eigen
// Cyclic Jacobi for a Hermitian b x b matrix H (row-major, global memory), one
// CTA.  Rounds of b/2 disjoint (p, q) pairs in round-robin order; each pair's
// rotation G = diag(1, e^{-i phi}) [[c, s], [-s, c]] removes H[p][q] = |h| e^{i phi}
// with (c, s) from the symmetric 2x2 Schur decomposition (tau = (h_qq - h_pp)/(2|h|),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c).
// Eigenvalues are returned sorted by increasing |lambda| (decreasing with
// descending = 1), eigenvectors in the matching columns of W.
__global__ void __launch_bounds__(1024) k_jacobi(double2* H, double2* W, double* lam, int b, int sweeps,
                                                int descending) {
    extern __shared__ double sm_jac[];
    const int bp = b + (b & 1);                  // padded to even
    int* order = reinterpret_cast<int*>(sm_jac);               // bp
    double* cs = sm_jac + (bp + 1) / 2 + 1;                      // bp/2
    double* sn = cs + bp / 2;                                    // bp/2
    double* ph_re = sn + bp / 2;                                 // bp/2
    double* ph_im = ph_re + bp / 2;                              // bp/2
    __shared__ double offn, totn;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < b * b; e += nt) W[e] = make_double2((e / b) == (e % b) ? 1.0 : 0.0, 0.0);
    for (int i = tid; i < bp; i += nt) order[i] = i;
    __syncthreads();
    for (int sw = 0; sw < sweeps; ++sw) {
        // convergence test: off-diagonal Frobenius norm vs total
        if (tid == 0) { offn = 0; totn = 0; }
        __syncthreads();
        double lo = 0, lt_ = 0;
        for (int e = tid; e < b * b; e += nt) {
            const double2 v = H[e];
            const double m = v.x * v.x + v.y * v.y;
            lt_ += m;
            if ((e / b) != (e % b)) lo += m;
        }
        atomicAdd(&offn, lo);
        atomicAdd(&totn, lt_);
        __syncthreads();
        if (offn <= 1e-30 * totn) break;
        for (int round = 0; round < bp - 1; ++round) {
            // pair k: (order[k], order[bp-1-k])
            for (int k = tid; k < bp / 2; k += nt) {
                int p = order[k], q = order[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, pr = 1.0, pi = 0.0;
                if (q < b) {
                    const double2 hpq = H[p * b + q];
                    const double a = sqrt(hpq.x * hpq.x + hpq.y * hpq.y);
                    if (a > 0.0) {
                        const double hpp = H[p * b + p].x, hqq = H[q * b + q].x;
                        const double tau = (hqq - hpp) / (2.0 * a);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        pr = hpq.x / a;     // e^{i phi}
                        pi = hpq.y / a;
                    }
                }
                cs[k] = c; sn[k] = s; ph_re[k] = pr; ph_im[k] = pi;
            }
            __syncthreads();
            // rows: [H_pj; H_qj] <- G^H [H_pj; H_qj],  G^H = [[c, -s e^{i phi}], [s, c e^{i phi}]]
            for (int e = tid; e < (bp / 2) * b; e += nt) {
                const int k = e / b, jcol = e % b;
                int p = order[k], q = order[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= b) continue;
                const double c = cs[k], s = sn[k];
                const double2 ph = make_double2(ph_re[k], ph_im[k]);
                const double2 hp = H[p * b + jcol], hq = H[q * b + jcol];
                const double2 phq = cmul(ph, hq);
                H[p * b + jcol] = make_double2(c * hp.x - s * phq.x, c * hp.y - s * phq.y);
                H[q * b + jcol] = make_double2(s * hp.x + c * phq.x, s * hp.y + c * phq.y);
            }
            __syncthreads();
            // columns: [H_ip, H_iq] <- [H_ip, H_iq] G, G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]; same for W
            for (int e = tid; e < (bp / 2) * b * 2; e += nt) {
                const int which = e / ((bp / 2) * b);
                const int e2 = e % ((bp / 2) * b);
                const int k = e2 / b, i = e2 % b;
                int p = order[k], q = order[bp - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= b) continue;
                double2* M = which ? W : H;
                const double c = cs[k], s = sn[k];
                const double2 phc = make_double2(ph_re[k], -ph_im[k]);
                const double2 mp = M[i * b + p], mq = M[i * b + q];
                const double2 mqp = cmul(mq, phc);
                M[i * b + p] = make_double2(c * mp.x - s * mqp.x, c * mp.y - s * mqp.y);
                M[i * b + q] = make_double2(s * mp.x + c * mqp.x, s * mp.y + c * mqp.y);
            }
            __syncthreads();
            // round-robin: keep order[0], rotate the rest
            if (tid == 0) {
                const int last = order[bp - 1];
                for (int i = bp - 1; i > 1; --i) order[i] = order[i - 1];
                order[1] = last;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // sort by |lambda| (rank sort), eigenvectors move with their eigenvalue; H is scratch
    for (int i = tid; i < b; i += nt) lam[i] = H[i * b + i].x;
    __syncthreads();
    for (int e = tid; e < b * b; e += nt) H[e] = W[e];
    __syncthreads();
    for (int i = tid; i < b; i += nt) {
        const double li = descending ? -fabs(lam[i]) : fabs(lam[i]);
        int rank = 0;
        for (int j2 = 0; j2 < b; ++j2) {
            const double lj = descending ? -fabs(lam[j2]) : fabs(lam[j2]);
            if (lj < li || (lj == li && j2 < i)) ++rank;
        }
        order[i] = rank;
    }
    __syncthreads();
    double* lcopy = cs;   // reuse (needs b doubles: cs..ph_im hold 2*bp)
    for (int i = tid; i < b; i += nt) lcopy[order[i]] = lam[i];
    for (int e = tid; e < b * b; e += nt) {
        const int row = e / b, col = e % b;
        W[row * b + order[col]] = H[row * b + col];
    }
    __syncthreads();
    for (int i = tid; i < b; i += nt) lam[i] = lcopy[i];
}

// Cholesky factor of a Hermitian positive definite b x b matrix G = R^H R (R upper,
// right-looking outer-product form, in place in G), then Rinv = R^{-1} by
// back-substitution, one column per thread.  One CTA; status[0] = 1 if a pivot is
// not positive.
__global__ void __launch_bounds__(1024) k_cholesky_inv(double2* G, double2* Rinv, int b, int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            double d = G[j * b + j].x;
            if (!(d > 0.0)) {
                *status = 1;
                d = 1e-300;
            }
            G[j * b + j] = make_double2(sqrt(d), 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / G[j * b + j].x;
        for (int i = j + 1 + tid; i < b; i += nt) G[j * b + i] = make_double2(G[j * b + i].x * inv, G[j * b + i].y * inv);
        __syncthreads();
        const int m = b - j - 1;
        for (int e = tid; e < m * m; e += nt) {
            const int p = j + 1 + e / m, q = j + 1 + e % m;
            if (q < p) continue;
            const double2 rp = G[j * b + p], rq = G[j * b + q];
            // G[p][q] -= conj(R[j][p]) R[j][q]
            G[p * b + q] = make_double2(G[p * b + q].x - (rp.x * rq.x + rp.y * rq.y),
                                        G[p * b + q].y - (rp.x * rq.y - rp.y * rq.x));
        }
        __syncthreads();
    }
    // Rinv: solve R z = e_c for each column c (upper triangular back substitution)
    for (int c = tid; c < b; c += nt) {
        for (int i = b - 1; i >= 0; --i) {
            double2 acc = make_double2(i == c ? 1.0 : 0.0, 0.0);
            if (i > c) acc = make_double2(0.0, 0.0);
            for (int k = i + 1; k <= c; ++k) {
                const double2 r = G[i * b + k], z = Rinv[k * b + c];
                acc.x -= r.x * z.x - r.y * z.y;
                acc.y -= r.x * z.y + r.y * z.x;
            }
            const double d = G[i * b + i].x;
            Rinv[i * b + c] = (i > c) ? make_double2(0.0, 0.0) : make_double2(acc.x / d, acc.y / d);
        }
    }
}

void launch_cholesky_inv(double2* G, double2* Rinv, int b, int* status, cudaStream_t s) {
    MG_REQUIRE(b >= 1 && b <= 4096, MGMLMC_EINVAL, "cholesky: 1 <= b <= 4096");
    k_cholesky_inv<<<1, 1024, 0, s>>>(G, Rinv, b, status);
    MG_LAUNCHED();
}

void launch_jacobi_eig(double2* H, double2* W, double* lam, int b, int sweeps, cudaStream_t s, bool descending) {
    MG_REQUIRE(b >= 1 && b <= 1024, MGMLMC_EINVAL, "jacobi: 1 <= b <= 1024");
    const int bp = b + (b & 1);
    size_t sm = (size_t)((bp + 1) / 2 + 1) * sizeof(double) + 4 * (size_t)(bp / 2) * sizeof(double) + 64;
    if (sm < (size_t)(bp + 1) * sizeof(int)) sm = (bp + 1) * sizeof(int);
    k_jacobi<<<1, 1024, sm, s>>>(H, W, lam, b, sweeps, descending ? 1 : 0);
    MG_LAUNCHED();
}

#define INST(C)                                                                                         \
    template void launch_gemm_nn<C>(C*, const C*, const C*, int, int, int, bool, cudaStream_t);          \
    template void launch_gemm_hn<C>(double2*, const C*, const C*, long long, int, int, double2*, int,    \
                                    cudaStream_t);                                                       \
    template void launch_gauss_jordan<C>(C*, int, void*, cudaStream_t);
INST(double2)
INST(float2)

}  // namespace mg
