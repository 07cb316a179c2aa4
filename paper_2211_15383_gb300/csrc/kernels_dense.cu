// Dense complex kernels: GEMM (C = A B), tall-skinny inner products (C = A^H B),
// in-place Gauss-Jordan inversion of the coarsest operator, and a one-CTA
// cyclic Jacobi eigensolver for the small Hermitian Rayleigh-Ritz problems of
// the deflation setup.  FP64 instances run on the FP64 pipe, FP32 on the FP32
// pipe; the BF16 tensor-core coarsest solve lives in kernels_tc.cu.
#include <algorithm>

#include "kernels.cuh"

namespace mg {

// ------------------------------------------------------------------ GEMM nn
// Tile 64 x 32 (rows x cols), K step 16; thread (tx, ty) owns column tx and rows
// ty*8 .. ty*8+7.  All threads of a warp share ty, so A reads are broadcasts.
constexpr int GM = 64, GN = 32, GK = 16;

template <typename S, typename C>
__global__ void __launch_bounds__(256) k_gemm_nn(S* __restrict__ Cm, const S* __restrict__ A,
                                                 const S* __restrict__ B, int M, int K, int Nc, bool accumulate) {
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
            As[r][k] = (gr < M && gk < K) ? cvtc(A[(long long)gr * K + gk], C{}) : czero<C>();
        }
        for (int e = tid; e < GK * GN; e += 256) {
            const int k = e / GN, c = e % GN;
            const int gk = k0 + k, gc = col0 + c;
            Bs[k][c] = (gk < K && gc < Nc) ? cvtc(B[(long long)gk * Nc + gc], C{}) : czero<C>();
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
            const S v = cvtc(acc[r], S{});
            Cm[idx] = accumulate ? cadd(Cm[idx], v) : v;
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
    MG_REQUIRE((M + 15) / 16 <= 65535 || (Nc > 8 && (M + GM - 1) / GM <= 65535), MGMLMC_EINVAL, "gemm_nn: M too large");
    if (Nc <= 8) {
        dim3 g(1, (M + 15) / 16);
        k_gemm_nn8<C><<<g, dim3(8, 16), 0, s>>>(Cm, A, B, M, K, Nc, accumulate);
        MG_LAUNCHED();
        return;
    }
    dim3 g((Nc + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm_nn<C, C><<<g, dim3(32, 8), 0, s>>>(Cm, A, B, M, K, Nc, accumulate);
    MG_LAUNCHED();
}

void launch_gemm_nn_fp32(double2* Cm, const double2* A, const double2* B, int M, int K, int Nc, cudaStream_t s) {
    dim3 g((Nc + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm_nn<double2, float2><<<g, dim3(32, 8), 0, s>>>(Cm, A, B, M, K, Nc, false);
    MG_LAUNCHED();
}

// ------------------------------------------------------------------ GEMM hn
// part[g][a][b] = sum_{i in slice g} conj(A[i][a]) B[i][b]; tile 32 x 32, thread
// (tx = b, ty) owns a = ty*4 .. ty*4+3.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_gemm_hn(double2* __restrict__ part, const S* __restrict__ A,
                                                 const S* __restrict__ B, long long n, int ka, int kb,
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
            As[ii][c] = (gi < i_end && a0 + c < ka) ? cvtc(A[gi * ka + a0 + c], C{}) : czero<C>();
            Bs[ii][c] = (gi < i_end && b0 + c < kb) ? cvtc(B[gi * kb + b0 + c], C{}) : czero<C>();
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
    k_gemm_hn<C, C><<<g, dim3(32, 8), 0, s>>>(part, A, B, n, ka, kb, slice);
    MG_LAUNCHED();
    launch_finalize(Cm, part, groups, ka * kb, s);
}

// FP32 arithmetic on FP64 storage: each group's slice of rows is summed in FP32, the
// group partials in FP64.
int gemm_hn_fp32_groups(long long n, int ka, int kb) {
    const long long tiles = (long long)((ka + 31) / 32) * ((kb + 31) / 32);
    long long g = (4LL * kNumSM + tiles - 1) / tiles;
    g = std::max(g, (n + 16383) / 16384);                  // at most 16384 rows summed in FP32
    return (int)std::min(g, (n + 63) / 64);
}
void launch_gemm_hn_fp32(double2* Cm, const double2* A, const double2* B, long long n, int ka, int kb,
                         double2* part, int groups, cudaStream_t s) {
    long long slice = (n + groups - 1) / groups;
    slice = ((slice + 15) / 16) * 16;
    dim3 g((kb + 31) / 32, (ka + 31) / 32, groups);
    k_gemm_hn<double2, float2><<<g, dim3(32, 8), 0, s>>>(part, A, B, n, ka, kb, slice);
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
// Pivot candidate of one elimination CTA for the next column of the panel: the largest
// |A[i][k+1]|^2 over the CTA's rows i > k, ties to the smaller row index.
struct GJCand {
    double m;
    int i;
    int pad;
};
struct GJWork {
    int* perm;       // n
    GJCand* cand;    // (n + 7) / 8 candidates of the next column (16 B each, n slots)
    int* status;     // 1 = zero pivot met
    void* rows;      // B x n copy of the panel's pivot rows (type C)
};

// |v|^2 in FP64 with separately rounded products, so that the pivot search of the
// first column of a panel and the candidates of the others rank rows alike.
template <typename C>
__device__ __forceinline__ double gj_mag2(C v) {
    return __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
}
constexpr int kGJRowsPerCTA = 8;   // k_gj_eliminate: one warp per row

template <typename C> struct GJPanel;
template <> struct GJPanel<float2> { static constexpr int B = 32; };
template <> struct GJPanel<double2> { static constexpr int B = 16; };

// Step k of the panel [k0, k0 + kb): pivot search in column k (rows >= k), swap rows
// k and p within the panel columns, scale the panel part of row k.  The first column
// of a panel is searched row by row; for the others the elimination of the previous
// column left one candidate per CTA (ncand of them, in row order), which give the same
// pivot: the largest |A[i][k]|^2, ties to the smallest row index.
template <typename C>
__global__ void __launch_bounds__(1024) k_gj_pivot(C* A, int n, int k, int k0, int kb, GJWork w, int ncand) {
    __shared__ double best[1024];
    __shared__ int bidx[1024];
    double bv = -1.0;
    int bi = k;
    if (ncand > 0) {
        for (int g = threadIdx.x; g < ncand; g += blockDim.x) {
            const GJCand cd = w.cand[g];
            if (cd.m > bv) { bv = cd.m; bi = cd.i; }
        }
    } else {
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double m = gj_mag2(A[(long long)i * n + k]);
            if (m > bv) { bv = m; bi = i; }
        }
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
}

// Elimination of column k from every other row, within the panel columns: one warp
// per row, lanes over the columns (kb <= 32: lane L owns column k0 + L).  The
// multiplier is A[i][k] as the pivot step left it, read by every lane before the lane
// of column k overwrites it.  When column k + 1 is in the panel, the CTA also leaves
// the pivot candidate of that column among its rows i > k (w.cand[blockIdx.x]).
template <typename C>
__global__ void __launch_bounds__(32 * kGJRowsPerCTA) k_gj_eliminate(C* A, int n, int k, int k0, int kb, GJWork w) {
    __shared__ double cm[kGJRowsPerCTA];
    __shared__ int ci[kGJRowsPerCTA];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * kGJRowsPerCTA + wid;
    const bool next = k + 1 < k0 + kb;
    double m = -1.0;
    if (i < n && i != k) {
        const C f = A[(long long)i * n + k];
        __syncwarp();
        const int c = k0 + lane;
        if (c < k0 + kb) {
            const C pk = A[(long long)k * n + c];
            const long long idx = (long long)i * n + c;
            const C v = (c == k) ? czero<C>() : A[idx];
            const C r = csub(v, cmul(f, pk));
            A[idx] = r;
            if (c == k + 1 && i > k) m = gj_mag2(r);
        }
    }
    if (!next) return;                                   // uniform over the grid
    m = __shfl_sync(0xffffffffu, m, k + 1 - k0);
    if (lane == 0) {
        cm[wid] = m;
        ci[wid] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bm = -1.0;
        int bi = k + 1;
        for (int q = 0; q < kGJRowsPerCTA; ++q)
            if (cm[q] > bm) { bm = cm[q]; bi = ci[q]; }
        w.cand[blockIdx.x] = GJCand{bm, bi, 0};
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

// candidates (n slots of 16 B) | perm (n int) | status | pad to 256 B | pivot rows (B x n, 256 n bytes
// for both instances: 32 x 8 B and 16 x 16 B per column)
static size_t gj_rows_offset(int n) { return (((size_t)n * sizeof(double2) + (size_t)n * sizeof(int) + 64) + 255) / 256 * 256; }
size_t gauss_jordan_work_bytes(int n) { return gj_rows_offset(n) + (size_t)n * 256 + 256; }

template <typename C>
void launch_gauss_jordan(C* A, int n, void* work, cudaStream_t s) {
    constexpr int B = GJPanel<C>::B;
    static_assert(B * sizeof(C) == 256, "pivot-row buffer is 256 bytes per column");
    GJWork w;
    w.cand = reinterpret_cast<GJCand*>(work);
    w.perm = reinterpret_cast<int*>(reinterpret_cast<double2*>(work) + n);
    w.status = w.perm + n;
    w.rows = reinterpret_cast<char*>(work) + gj_rows_offset(n);
    MG_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s));
    long long launches = 0;
    const dim3 tiles((n + 63) / 64, (n + 63) / 64);
    const int ncand = (n + kGJRowsPerCTA - 1) / kGJRowsPerCTA;   // <= n slots of 16 B
    for (int k0 = 0; k0 < n; k0 += B) {
        const int kb = n - k0 < B ? n - k0 : B;
        for (int k = k0; k < k0 + kb; ++k) {
            k_gj_pivot<C><<<1, 1024, 0, s>>>(A, n, k, k0, kb, w, k > k0 ? ncand : 0);
            k_gj_eliminate<C><<<ncand, 32 * kGJRowsPerCTA, 0, s>>>(A, n, k, k0, kb, w);
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
// Cyclic Jacobi for a Hermitian b x b matrix H (row-major), one persistent
// cooperative kernel over the whole GPU.  A sweep is bp - 1 rounds (bp = b padded
// to even) of bp/2 disjoint index pairs in round-robin order: in round r pair k is
// (ord(k), ord(bp-1-k)) with ord(0) = 0 and ord(i) = 1 + (i - 1 + r) mod (bp - 1).
// Pair (p, q) gets the rotation G = diag(1, e^{-i phi}) [[c, s], [-s, c]] that
// removes H[p][q] = |h| e^{i phi}, with (c, s) from the symmetric 2x2 Schur
// decomposition (tau = (h_qq - h_pp)/(2|h|), t = sign(tau)/(|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1+t^2), s = t c).  Since the pairs of a round are disjoint, the whole
// round is H <- J^H H J with J block diagonal in the pairing: every 2x2 block (P, Q)
// of the pairing becomes G_P^H H(P, Q) G_Q, computed from a read-only copy of H
// (double buffer), and W(:, P) <- W(:, P) G_P in place.  One grid barrier per round.
// The sweeps stop when the off-diagonal Frobenius norm is below 1e-15 of the total.
// Eigenvalues come back sorted by increasing |lambda| (decreasing with descending),
// eigenvectors in the matching columns of W.
namespace jac {
constexpr int kThreads = 256;
constexpr long long kSpinLimit = 1LL << 24;   // x ~64 ns sleep: a barrier gives up after ~1 s

struct Sync {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

// Grid barrier for a cooperative launch (all CTAs resident); bounded wait: a CTA that
// waits too long records the failure and every CTA leaves at its next check.
__device__ __forceinline__ bool grid_barrier(Sync* sy, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &sy->gen;
        volatile int* verr = &sy->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&sy->count, 1u);
        if (arrived == nblocks - 1) {
            sy->count = 0;
            __threadfence();
            atomicAdd(&sy->gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g && *verr == 0) {
                if (++spins > kSpinLimit) {
                    atomicExch(&sy->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = (*verr == 0);
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int ord(int i, int r, int bp) { return i == 0 ? 0 : 1 + (i - 1 + r) % (bp - 1); }

__global__ void __launch_bounds__(kThreads) k_jacobi_grid(const double2* __restrict__ Hin, double2* A0, double2* A1,
                                                          double2* Wp, double* part, double* rot, Sync* sy, int b,
                                                          int bp, int sweeps) {
    extern __shared__ double sm_rot[];
    const int half = bp / 2;
    double* rc = sm_rot;                  // half each: c, s, Re e^{i phi}, Im e^{i phi}
    double* rs = rc + half;
    double* rpr = rs + half;
    double* rpi = rpr + half;
    int* rp = reinterpret_cast<int*>(rpi + half);   // pair indices p < q
    int* rq = rp + half;
    __shared__ double red_off[kThreads], red_tot[kThreads];
    __shared__ int stop;
    const unsigned G = gridDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)G * blockDim.x;
    const long long bb = (long long)bp * bp;
    for (long long e = tid; e < bb; e += nthr) {
        const int i = (int)(e / bp), j = (int)(e % bp);
        A0[e] = (i < b && j < b) ? Hin[(long long)i * b + j] : make_double2(0.0, 0.0);
        Wp[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    if (!grid_barrier(sy, G)) return;
    double2* cur = A0;
    double2* nxt = A1;
    for (int sw = 0; sw < sweeps; ++sw) {
        double lo = 0.0, lt = 0.0;
        for (long long e = tid; e < bb; e += nthr) {
            const double2 v = __ldcg(cur + e);
            const double m = v.x * v.x + v.y * v.y;
            lt += m;
            if (e / bp != e % bp) lo += m;
        }
        red_off[threadIdx.x] = lo;
        red_tot[threadIdx.x] = lt;
        __syncthreads();
        for (int st = kThreads / 2; st > 0; st >>= 1) {
            if ((int)threadIdx.x < st) {
                red_off[threadIdx.x] += red_off[threadIdx.x + st];
                red_tot[threadIdx.x] += red_tot[threadIdx.x + st];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = red_off[0];
            part[2 * blockIdx.x + 1] = red_tot[0];
        }
        if (!grid_barrier(sy, G)) return;
        if (threadIdx.x == 0) {
            double off = 0.0, tot = 0.0;       // same order in every CTA: the same decision
            for (unsigned g2 = 0; g2 < G; ++g2) {
                off += __ldcg(part + 2 * g2);
                tot += __ldcg(part + 2 * g2 + 1);
            }
            stop = (off <= 1e-30 * tot);
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < bp - 1; ++r) {
            // each rotation of the round once, grid-wide (FP64 square roots and divisions
            // run at 1/64 of the FP32 rate: computing all of them in every CTA cost more
            // than the block updates), published in rot[4][half] ...
            for (long long k = tid; k < half; k += nthr) {
                int p = ord((int)k, r, bp), q = ord(bp - 1 - (int)k, r, bp);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, sn = 0.0, pr = 1.0, pi = 0.0;
                if (q < b) {
                    const double2 hpq = __ldcg(cur + (long long)p * bp + q);
                    const double a = sqrt(hpq.x * hpq.x + hpq.y * hpq.y);
                    if (a > 0.0) {
                        const double hpp = __ldcg(cur + (long long)p * bp + p).x;
                        const double hqq = __ldcg(cur + (long long)q * bp + q).x;
                        const double tau = (hqq - hpp) / (2.0 * a);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                        pr = hpq.x / a;
                        pi = hpq.y / a;
                    }
                }
                rot[k] = c;
                rot[half + k] = sn;
                rot[2 * half + k] = pr;
                rot[3 * half + k] = pi;
            }
            if (!grid_barrier(sy, G)) return;
            // ... and staged by every CTA into shared memory with the pair indices
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p = ord(k, r, bp), q = ord(bp - 1 - k, r, bp);
                if (p > q) { const int t = p; p = q; q = t; }
                rc[k] = __ldcg(rot + k);
                rs[k] = __ldcg(rot + half + k);
                rpr[k] = __ldcg(rot + 2 * half + k);
                rpi[k] = __ldcg(rot + 3 * half + k);
                rp[k] = p;
                rq[k] = q;
            }
            __syncthreads();
            // 2x2 blocks (P, Q): out = G_P^H B G_Q
            const long long nblk = (long long)half * half;
            for (long long e = tid; e < nblk; e += nthr) {
                const int P = (int)(e / half), Q = (int)(e % half);
                const int p1 = rp[P], q1 = rq[P], p2 = rp[Q], q2 = rq[Q];
                const double c1 = rc[P], s1 = rs[P], c2 = rc[Q], s2 = rs[Q];
                const double2 f1 = make_double2(rpr[P], rpi[P]);
                const double2 f2c = make_double2(rpr[Q], -rpi[Q]);
                // written by other CTAs in the previous round: read through L2, not L1
                const double2 b00 = __ldcg(cur + (long long)p1 * bp + p2), b01 = __ldcg(cur + (long long)p1 * bp + q2);
                const double2 b10 = __ldcg(cur + (long long)q1 * bp + p2), b11 = __ldcg(cur + (long long)q1 * bp + q2);
                // rows: R0 = c1 B0 - s1 f1 B1, R1 = s1 B0 + c1 f1 B1
                const double2 fb10 = cmul(f1, b10), fb11 = cmul(f1, b11);
                const double2 r00 = make_double2(c1 * b00.x - s1 * fb10.x, c1 * b00.y - s1 * fb10.y);
                const double2 r01 = make_double2(c1 * b01.x - s1 * fb11.x, c1 * b01.y - s1 * fb11.y);
                const double2 r10 = make_double2(s1 * b00.x + c1 * fb10.x, s1 * b00.y + c1 * fb10.y);
                const double2 r11 = make_double2(s1 * b01.x + c1 * fb11.x, s1 * b01.y + c1 * fb11.y);
                // columns: O_i0 = c2 R_i0 - s2 conj(f2) R_i1, O_i1 = s2 R_i0 + c2 conj(f2) R_i1
                const double2 g01 = cmul(r01, f2c), g11 = cmul(r11, f2c);
                nxt[(long long)p1 * bp + p2] = make_double2(c2 * r00.x - s2 * g01.x, c2 * r00.y - s2 * g01.y);
                nxt[(long long)p1 * bp + q2] = make_double2(s2 * r00.x + c2 * g01.x, s2 * r00.y + c2 * g01.y);
                nxt[(long long)q1 * bp + p2] = make_double2(c2 * r10.x - s2 * g11.x, c2 * r10.y - s2 * g11.y);
                nxt[(long long)q1 * bp + q2] = make_double2(s2 * r10.x + c2 * g11.x, s2 * r10.y + c2 * g11.y);
            }
            // eigenvectors: W(:, P) <- W(:, P) G_P, in place (disjoint columns)
            const long long nw = (long long)bp * half;
            for (long long e = tid; e < nw; e += nthr) {
                const int i = (int)(e / half), P = (int)(e % half);
                const int p = rp[P], q = rq[P];
                const double c = rc[P], sn = rs[P];
                const double2 fc = make_double2(rpr[P], -rpi[P]);
                const double2 wp = __ldcg(Wp + (long long)i * bp + p);
                const double2 wq = cmul(__ldcg(Wp + (long long)i * bp + q), fc);
                Wp[(long long)i * bp + p] = make_double2(c * wp.x - sn * wq.x, c * wp.y - sn * wq.y);
                Wp[(long long)i * bp + q] = make_double2(sn * wp.x + c * wq.x, sn * wp.y + c * wq.y);
            }
            if (!grid_barrier(sy, G)) return;
            double2* t = cur;
            cur = nxt;
            nxt = t;
        }
    }
    // the diagonal of the last matrix goes to part[0 .. b) for the sorting kernel
    for (long long i = tid; i < b; i += nthr) part[2 * G + i] = __ldcg(cur + i * bp + i).x;
}

// rank of every eigenvalue by |lambda| (ties by index), then lam and the columns
// of W permuted to that order; a barrier failure is passed to the caller's flag.
__global__ void k_jacobi_rank(const double* diag, int* rank, int b, int descending) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= b) return;
    const double lc = descending ? -fabs(diag[col]) : fabs(diag[col]);
    int r = 0;
    for (int j = 0; j < b; ++j) {
        const double lj = descending ? -fabs(diag[j]) : fabs(diag[j]);
        r += (lj < lc || (lj == lc && j < col)) ? 1 : 0;
    }
    rank[col] = r;
}

__global__ void k_jacobi_permute(const double* diag, const int* rank, const double2* Wp, double2* W, double* lam,
                                 int b, int bp, const Sync* sy, int* err) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long e = tid; e < (long long)b * b; e += nthr) {
        const int row = (int)(e / b), col = (int)(e % b);
        W[(long long)row * b + rank[col]] = Wp[(long long)row * bp + col];
        if (row == 0) lam[rank[col]] = diag[col];
    }
    if (tid == 0 && err && sy->err) *err = 1;
}
}  // namespace jac

static int jacobi_grid_size() {
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, per = 0, coop = 0;
        MG_CUDA(cudaGetDevice(&dev));
        MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        MG_REQUIRE(coop, MGMLMC_ECUDA, "jacobi: the device does not support cooperative launches");
        const size_t sm = jacobi_smem_bytes(2048);
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jac::k_jacobi_grid, jac::kThreads, sm));
        MG_REQUIRE(per >= 1, MGMLMC_ECUDA, "jacobi: kernel cannot be resident");
        g = sms;   // one CTA per SM: every CTA resident, as the grid barrier requires
    }
    return g;
}

size_t jacobi_smem_bytes(int b) {
    const int bp = b + (b & 1);
    return (size_t)(bp / 2) * (4 * sizeof(double) + 2 * sizeof(int));
}

size_t jacobi_work_bytes(int b) {
    const size_t bp = (size_t)(b + (b & 1));
    return 3 * bp * bp * sizeof(double2) + (2 * (size_t)kNumSM * 4 + bp) * sizeof(double) + 256 + bp * sizeof(int) +
           2 * bp * sizeof(double) + 256;
}

// Cholesky factor of a Hermitian positive definite b x b matrix G = R^H R (R upper)
// and Rinv = R^{-1}, one cooperative kernel over all SMs.
//  Factorisation, right-looking, one grid barrier per column j: every thread reads
//  d = G[j][j] (final after the previous column), row j of R is G[j][.] / sqrt(d),
//  and the trailing upper triangle takes G[p][q] -= conj(R[j][p]) R[j][q] (p, q > j),
//  with R[j][.] formed on the fly from G's row j, which this column leaves untouched.
//  Inverse, one warp per column c of T = R^{-1} (back substitution from i = c down,
//  T[i][c] = (delta_ic - sum_{k>i} R[i][k] T[k][c]) / R[i][i], the sum split over the
//  lanes); T is kept transposed (Tt[c][k], coalesced along k) and written out at the end.
//  status[0] = 1 if a pivot was not positive (it is then replaced by 1e-300).
namespace chol {
__global__ void __launch_bounds__(jac::kThreads) k_cholesky_grid(double2* G, double2* Rinv, double2* R, double2* Tt,
                                                                 int b, int* status, jac::Sync* sy) {
    const unsigned NB = gridDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)NB * blockDim.x;
    for (int j = 0; j < b; ++j) {
        double d = __ldcg(G + (long long)j * b + j).x;
        if (!(d > 0.0)) {
            if (tid == 0) *status = 1;
            d = 1e-300;
        }
        const double rd = sqrt(d), inv = 1.0 / rd;
        for (long long i = tid; i < b; i += nthr) {
            double2 v = make_double2(0.0, 0.0);
            if (i == j) v = make_double2(rd, 0.0);
            else if (i > j) {
                const double2 g = __ldcg(G + (long long)j * b + i);
                v = make_double2(g.x * inv, g.y * inv);
            }
            R[(long long)j * b + i] = v;
        }
        const long long m = b - j - 1;
        for (long long e = tid; e < m * m; e += nthr) {
            const int p = j + 1 + (int)(e / m), q = j + 1 + (int)(e % m);
            if (q < p) continue;
            const double2 gp = __ldcg(G + (long long)j * b + p), gq = __ldcg(G + (long long)j * b + q);
            const double2 g = __ldcg(G + (long long)p * b + q);
            // conj(R[j][p]) R[j][q] = conj(gp) gq / d
            G[(long long)p * b + q] = make_double2(g.x - (gp.x * gq.x + gp.y * gq.y) / d,
                                                   g.y - (gp.x * gq.y - gp.y * gq.x) / d);
        }
        if (!jac::grid_barrier(sy, NB)) return;
    }
    const int lane = threadIdx.x & 31;
    const long long warp = tid >> 5, nwarps = nthr >> 5;
    for (long long c = warp; c < b; c += nwarps) {
        double2* t = Tt + c * b;
        for (int i = (int)c; i >= 0; --i) {
            double sr = 0.0, si = 0.0;
            for (int k = i + 1 + lane; k <= c; k += 32) {
                const double2 r = __ldcg(R + (long long)i * b + k), tk = t[k];
                sr += r.x * tk.x - r.y * tk.y;
                si += r.x * tk.y + r.y * tk.x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) {
                const double rii = __ldcg(R + (long long)i * b + i).x;
                t[i] = make_double2(((i == c ? 1.0 : 0.0) - sr) / rii, -si / rii);
            }
            __syncwarp();
        }
        for (int i = (int)c + 1 + lane; i < b; i += 32) t[i] = make_double2(0.0, 0.0);
    }
    if (!jac::grid_barrier(sy, NB)) return;
    for (long long e = tid; e < (long long)b * b; e += nthr) {
        const long long i = e / b, c = e % b;
        Rinv[e] = __ldcg(Tt + c * b + i);
    }
}

__global__ void k_flag(const jac::Sync* sy, int* err) {
    if (err && sy->err) *err = 1;
}
}  // namespace chol

size_t cholesky_work_bytes(int b) { return 2 * (size_t)b * b * sizeof(double2) + 256; }

void launch_cholesky_inv(double2* G, double2* Rinv, int b, void* work, int* status, int* err, cudaStream_t s) {
    MG_REQUIRE(b >= 1 && b <= 4096, MGMLMC_EINVAL, "cholesky: 1 <= b <= 4096");
    const int NB = jacobi_grid_size();
    double2* R = reinterpret_cast<double2*>(work);
    double2* Tt = R + (size_t)b * b;
    jac::Sync* sy = reinterpret_cast<jac::Sync*>(Tt + (size_t)b * b);
    MG_CUDA(cudaMemsetAsync(sy, 0, sizeof(jac::Sync), s));
    void* args[] = {(void*)&G, (void*)&Rinv, (void*)&R, (void*)&Tt, (void*)&b, (void*)&status, (void*)&sy};
    MG_CUDA(cudaLaunchCooperativeKernel((const void*)chol::k_cholesky_grid, dim3(NB), dim3(jac::kThreads), args, 0,
                                        s));
    MG_LAUNCHED();
    chol::k_flag<<<1, 1, 0, s>>>(sy, err);
    MG_LAUNCHED();
}

void launch_jacobi_eig(double2* H, double2* W, double* lam, int b, int sweeps, void* work, int* err, cudaStream_t s,
                       bool descending) {
    MG_REQUIRE(b >= 1 && b <= 2048, MGMLMC_EINVAL, "jacobi: 1 <= b <= 2048");
    const int bp = b + (b & 1);
    const int G = jacobi_grid_size();
    MG_REQUIRE(G <= 4 * kNumSM, MGMLMC_ECUDA, "jacobi: more SMs than the work space assumes");
    char* w = reinterpret_cast<char*>(work);
    const size_t mat = (size_t)bp * bp * sizeof(double2);
    double2* A0 = reinterpret_cast<double2*>(w);
    double2* A1 = reinterpret_cast<double2*>(w + mat);
    double2* Wp = reinterpret_cast<double2*>(w + 2 * mat);
    double* part = reinterpret_cast<double*>(w + 3 * mat);
    jac::Sync* sy = reinterpret_cast<jac::Sync*>(part + 2 * (size_t)kNumSM * 4 + bp);
    // after Sync: the rank array (bp ints), then the rotations (4 x bp/2 doubles)
    double* rot = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(reinterpret_cast<int*>(sy + 1) + bp) + 255) / 256 * 256);
    MG_CUDA(cudaMemsetAsync(sy, 0, sizeof(jac::Sync), s));
    const size_t sm = jacobi_smem_bytes(b);
    void* args[] = {(void*)&H, (void*)&A0, (void*)&A1, (void*)&Wp, (void*)&part, (void*)&rot, (void*)&sy, (void*)&b,
                    (void*)&bp, (void*)&sweeps};
    MG_CUDA(cudaLaunchCooperativeKernel((const void*)jac::k_jacobi_grid, dim3(G), dim3(jac::kThreads), args, sm, s));
    MG_LAUNCHED();
    int* rank = reinterpret_cast<int*>(sy + 1);
    jac::k_jacobi_rank<<<(b + 255) / 256, 256, 0, s>>>(part + 2 * G, rank, b, descending ? 1 : 0);
    MG_LAUNCHED();
    jac::k_jacobi_permute<<<2 * kNumSM, 256, 0, s>>>(part + 2 * G, rank, Wp, W, lam, b, bp, sy, err);
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
