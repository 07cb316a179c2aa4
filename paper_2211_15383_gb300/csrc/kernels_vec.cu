// Multi-RHS vector kernels: Z2 noise, BLAS1 with per-rhs coefficients and
// deterministic per-rhs reductions.  Layout [row][rhs]; block (32 rhs, 8 rows);
// grid (rhs tiles, row groups) with a grid-stride loop over rows.  Arithmetic
// runs in the vector's own precision (FP32 vectors stay on the FP32 pipe);
// only the cross-block partial sums are FP64.
#include "kernels.cuh"

namespace mg {

__device__ __forceinline__ uint64_t sm64(uint64_t z) {
    // One splitmix64 step (Steele, Lea & Flood 2014): add the golden gamma, then mix.
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename C>
__global__ void k_noise(C* __restrict__ x, long long n, int N, uint64_t seed, uint64_t term, int64_t first) {
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    const uint64_t ks = sm64(sm64(seed ^ term) ^ (uint64_t)(first + j));
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        const uint64_t h = sm64(ks ^ (uint64_t)i);
        C v;
        v.x = (h & 1ull) ? -1 : 1;
        v.y = 0;
        x[i * N + j] = v;
    }
}

template <typename C>
__global__ void k_probes(C* __restrict__ x, const int8_t* __restrict__ p, long long n, int N) {
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        C v;
        v.x = p[(long long)j * n + i];
        v.y = 0;
        x[i * N + j] = v;
    }
}

template <typename Cout, typename Cin>
__global__ void k_convert(Cout* __restrict__ y, const Cin* __restrict__ x, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = cvtc(x[i], Cout());
}

template <typename C>
__global__ void k_zero(C* __restrict__ x, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = czero<C>();
}

template <typename Cy, typename Cx_>
__global__ void k_scale_rhs(Cy* __restrict__ y, const Cx_* __restrict__ x, const double* __restrict__ scale,
                            bool invert, long long n, int N) {
    using R = re_t<Cy>;
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    double sc = scale[j];
    if (invert) sc = (sc != 0.0) ? 1.0 / sc : 0.0;
    const R s = (R)sc;
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        Cy v = cvtc(x[i * N + j], Cy());
        y[i * N + j] = mk(v.x * s, v.y * s);
    }
}

// w[:, j] *= s[j] for the rhs with s[j] != 0; the others are left untouched (and their
// threads return after one load).
template <typename C>
__global__ void k_scale_cols_if(C* __restrict__ w, const double* __restrict__ s, long long n, int N) {
    using R = re_t<C>;
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    const double sc = s[j];
    if (sc == 0.0) return;
    const R f = (R)sc;
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        const C v = w[i * N + j];
        w[i * N + j] = mk(v.x * f, v.y * f);
    }
}

template <typename Cy, typename Cx_>
__global__ void k_axpy_rhs(Cy* __restrict__ y, const double2* __restrict__ alpha, const double* __restrict__ beta,
                           double sign, const Cx_* __restrict__ x, long long n, int N) {
    using R = re_t<Cy>;
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    double2 a = alpha ? alpha[j] : make_double2(1.0, 0.0);
    const double b = (beta ? beta[j] : 1.0) * sign;
    const Cy ar = mk((R)(a.x * b), (R)(a.y * b));
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        Cy acc = y[i * N + j];
        cfma(acc, ar, cvtc(x[i * N + j], Cy()));
        y[i * N + j] = acc;
    }
}

// ---------------------------------------------------------------- reductions
template <typename Cx_, typename Cy>
__global__ void k_dot(double2* __restrict__ part, const Cx_* __restrict__ x, const Cy* __restrict__ y,
                      long long n, int N) {
    using R = re_t<Cx_>;
    __shared__ double2 sh[kRowLanes][kRhsTile + 1];
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    using Ca = cx_t<R>;
    Ca acc = czero<Ca>();
    if (j < N)
        for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
             i += (long long)gridDim.y * kRowLanes)
            cfmac(acc, x[i * N + j], cvtc(y[i * N + j], Ca()));
    sh[threadIdx.y][threadIdx.x] = to_d(acc);
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        double2 s = sh[0][threadIdx.x];
        for (int r = 1; r < kRowLanes; ++r) s = cadd(s, sh[r][threadIdx.x]);
        part[(long long)blockIdx.y * N + j] = s;
    }
}

template <typename C>
__global__ void k_norm2(double* __restrict__ part, const C* __restrict__ x, long long n, int N) {
    using R = re_t<C>;
    __shared__ double sh[kRowLanes][kRhsTile + 1];
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    R acc = 0;
    if (j < N)
        for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
             i += (long long)gridDim.y * kRowLanes) {
            C v = x[i * N + j];
            acc = fma(v.x, v.x, fma(v.y, v.y, acc));
        }
    sh[threadIdx.y][threadIdx.x] = (double)acc;
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        double s = sh[0][threadIdx.x];
        for (int r = 1; r < kRowLanes; ++r) s += sh[r][threadIdx.x];
        part[(long long)blockIdx.y * N + j] = s;
    }
}

// R rows per loop trip with all their loads issued first (few vectors leave too few
// loads in flight per row otherwise).
template <typename C, int MAXM>
__global__ void k_multidot(double2* __restrict__ part, const C* __restrict__ V, int m, const C* __restrict__ w,
                           long long n, int N) {
    constexpr int R = MAXM <= 4 ? 4 : (MAXM <= 8 ? 2 : 1);
    __shared__ double2 sh[kRowLanes][kRhsTile + 1];
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    const long long stride = n * (long long)N;
    const long long S = (long long)gridDim.y * kRowLanes;
    C acc[MAXM];
#pragma unroll
    for (int k = 0; k < MAXM; ++k) acc[k] = czero<C>();
    if (j < N && R == 1) {
        for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n; i += S) {
            const C wv = w[i * N + j];
#pragma unroll
            for (int k = 0; k < MAXM; ++k)
                if (k < m) cfmac(acc[k], V[k * stride + i * N + j], wv);
        }
    } else if (j < N) {
        for (long long i0 = (long long)blockIdx.y * kRowLanes + threadIdx.y; i0 < n; i0 += R * S) {
            C wv[R], vv[R][MAXM];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const long long i = i0 + r * S;
                const bool in = i < n;
                wv[r] = in ? w[i * N + j] : czero<C>();
#pragma unroll
                for (int k = 0; k < MAXM; ++k) vv[r][k] = (in && k < m) ? V[k * stride + i * N + j] : czero<C>();
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int k = 0; k < MAXM; ++k)
                    if (k < m) cfmac(acc[k], vv[r][k], wv[r]);
        }
    }
    for (int k = 0; k < m; ++k) {
        double2 v = czero<double2>();
#pragma unroll
        for (int kk = 0; kk < MAXM; ++kk)
            if (kk == k) v = to_d(acc[kk]);
        sh[threadIdx.y][threadIdx.x] = v;
        __syncthreads();
        if (threadIdx.y == 0 && j < N) {
            double2 s = sh[0][threadIdx.x];
            for (int r = 1; r < kRowLanes; ++r) s = cadd(s, sh[r][threadIdx.x]);
            part[((long long)blockIdx.y * m + k) * N + j] = s;
        }
        __syncthreads();
    }
}

template <typename C>
__global__ void k_multiaxpy(C* __restrict__ w, const double2* __restrict__ coef, int m, const C* __restrict__ V,
                            double sign, long long n, int N, double* __restrict__ norm_part,
                            const double* __restrict__ eta, int eta_pow, int accumulate,
                            const double* __restrict__ norm_div) {
    using R = re_t<C>;
    __shared__ C cf[64][kRhsTile];
    __shared__ double sh[kRowLanes][kRhsTile + 1];
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    const long long stride = n * (long long)N;
    for (int k = threadIdx.y; k < m; k += kRowLanes) {
        double2 c = (j < N) ? coef[(long long)k * N + j] : make_double2(0, 0);
        double f = sign;
        if (eta && j < N) {
            // coefficient of an unnormalised vector V_k = eta_k v_k: divided by eta_k^pow
            // (a zero vector contributes nothing)
            const double e = eta[(long long)k * N + j];
            const double d = eta_pow == 2 ? e * e : e;
            f = (d != 0.0) ? sign / d : 0.0;
        }
        cf[k][threadIdx.x] = mk((R)(c.x * f), (R)(c.y * f));
    }
    __syncthreads();
    // the norm is summed over w / norm_div[j] (FP32 squares of a small vector would
    // leave the normal range)
    R ns = (R)1;
    if (norm_div && j < N) {
        const double dv = norm_div[j];
        ns = (R)((dv != 0.0) ? 1.0 / dv : 1.0);
    }
    R nrm = 0;
    if (j < N)
        for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
             i += (long long)gridDim.y * kRowLanes) {
            C acc = accumulate ? w[i * N + j] : mk((R)0, (R)0);
            for (int k = 0; k < m; ++k) cfma(acc, cf[k][threadIdx.x], V[k * stride + i * N + j]);
            w[i * N + j] = acc;
            const R ax = acc.x * ns, ay = acc.y * ns;
            nrm = fma(ax, ax, fma(ay, ay, nrm));
        }
    if (norm_part) {
        // |w|^2 partials of the updated vector, as k_norm2 writes them
        sh[threadIdx.y][threadIdx.x] = (double)nrm;
        __syncthreads();
        if (threadIdx.y == 0 && j < N) {
            double t = sh[0][threadIdx.x];
            for (int r = 1; r < kRowLanes; ++r) t += sh[r][threadIdx.x];
            norm_part[(long long)blockIdx.y * N + j] = t;
        }
    }
}

// Partials reduction: block (32 outputs, 32 group lanes); lane ty adds groups
// ty, ty+32, ... in order, then a fixed-order sum over the 32 lanes, so the result
// does not depend on timing (deterministic).
template <typename T>
__device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ double2 zero_of<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double add_of(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add_of(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename T>
__global__ void __launch_bounds__(1024) k_finalize(T* __restrict__ out, const T* __restrict__ part, int groups,
                                                   int count) {
    __shared__ T sh[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    T acc = zero_of<T>();
    if (j < count) {
        int g = threadIdx.y;
#pragma unroll 8
        for (; g < groups; g += 32) acc = add_of(acc, part[(long long)g * count + j]);
    }
    sh[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && j < count) {
        T s = sh[0][threadIdx.x];
        for (int r = 1; r < 32; ++r) s = add_of(s, sh[r][threadIdx.x]);
        out[j] = s;
    }
}

// ------------------------------------------------------------------ launchers
static inline dim3 blk() { return dim3(kRhsTile, kRowLanes); }

template <typename C>
void launch_noise(C* x, long long n, int N, uint64_t seed, uint64_t term, int64_t first, cudaStream_t s) {
    k_noise<C><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, s>>>(x, n, N, seed, term, first);
    MG_LAUNCHED();
}
template <typename C>
void launch_probes(C* x, const int8_t* p, long long n, int N, cudaStream_t s) {
    k_probes<C><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, s>>>(x, p, n, N);
    MG_LAUNCHED();
}
template <typename Cout, typename Cin>
void launch_convert(Cout* y, const Cin* x, long long count, cudaStream_t s) {
    if (count <= 0) return;
    long long b = (count + 255) / 256;
    if (b > kNumSM * 16) b = kNumSM * 16;
    k_convert<Cout, Cin><<<(int)b, 256, 0, s>>>(y, x, count);
    MG_LAUNCHED();
}
template <typename C>
void launch_zero(C* x, long long count, cudaStream_t s) {
    if (count <= 0) return;
    long long b = (count + 255) / 256;
    if (b > kNumSM * 16) b = kNumSM * 16;
    k_zero<C><<<(int)b, 256, 0, s>>>(x, count);
    MG_LAUNCHED();
}
template <typename Cy, typename Cx_>
void launch_scale_rhs(Cy* y, const Cx_* x, const double* scale, bool invert, long long n, int N, cudaStream_t s) {
    k_scale_rhs<Cy, Cx_><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, s>>>(y, x, scale, invert, n, N);
    MG_LAUNCHED();
}
template <typename C>
void launch_scale_cols_if(C* w, const double* s, long long n, int N, cudaStream_t st) {
    k_scale_cols_if<C><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, st>>>(w, s, n, N);
    MG_LAUNCHED();
}
template <typename Cy, typename Cx_>
void launch_axpy_rhs(Cy* y, const double2* alpha, const double* beta, double sign, const Cx_* x, long long n, int N,
                     cudaStream_t s) {
    k_axpy_rhs<Cy, Cx_><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, s>>>(y, alpha, beta, sign, x, n, N);
    MG_LAUNCHED();
}

int reduce_groups(long long n, int N) { return row_groups(n, N, 4); }
// The axpy of Gram-Schmidt streams m + 2 vectors with few loads per row: 16 blocks
// per SM keep more of them in flight.
int axpy_groups(long long n, int N) { return row_groups(n, N, 16); }

// Row-major partials: out[i] = sum_g part[i * groups + g]; one warp per output,
// lanes add g = lane, lane + 32, ... in order, then a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_finalize_rows(double2* __restrict__ out, const double2* __restrict__ part,
                                                       int groups, int count) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= count) return;
    const double2* row = part + (long long)i * groups;
    double2 acc = make_double2(0.0, 0.0);
    for (int g = lane; g < groups; g += 32) acc = cadd(acc, row[g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) out[i] = acc;
}

void launch_finalize_rows(double2* out, const double2* part, int groups, int count, cudaStream_t s) {
    k_finalize_rows<<<(count + 7) / 8, 256, 0, s>>>(out, part, groups, count);
    MG_LAUNCHED();
}

void launch_finalize(double2* out, const double2* part, int groups, int count, cudaStream_t s) {
    k_finalize<double2><<<(count + 31) / 32, dim3(32, 32), 0, s>>>(out, part, groups, count);
    MG_LAUNCHED();
}
void launch_finalize(double* out, const double* part, int groups, int count, cudaStream_t s) {
    k_finalize<double><<<(count + 31) / 32, dim3(32, 32), 0, s>>>(out, part, groups, count);
    MG_LAUNCHED();
}

template <typename Cx_, typename Cy>
void launch_dot(double2* out, const Cx_* x, const Cy* y, long long n, int N, double2* part, cudaStream_t s) {
    const int G = reduce_groups(n, N);
    k_dot<Cx_, Cy><<<dim3(rhs_tiles(N), G), blk(), 0, s>>>(part, x, y, n, N);
    MG_LAUNCHED();
    launch_finalize(out, part, G, N, s);
}
template <typename C>
void launch_norm2(double* out, const C* x, long long n, int N, double* part, cudaStream_t s) {
    const int G = reduce_groups(n, N);
    k_norm2<C><<<dim3(rhs_tiles(N), G), blk(), 0, s>>>(part, x, n, N);
    MG_LAUNCHED();
    launch_finalize(out, part, G, N, s);
}
template <typename C>
void launch_multidot(double2* out, const C* V, int m, const C* w, long long n, int N, double2* part, cudaStream_t s) {
    MG_REQUIRE(m >= 1 && m <= 64, MGMLMC_EINVAL, "multidot: 1 <= m <= 64");
    const int G = reduce_groups(n, N);
    dim3 g(rhs_tiles(N), G);
    if (m <= 4) k_multidot<C, 4><<<g, blk(), 0, s>>>(part, V, m, w, n, N);
    else if (m <= 8) k_multidot<C, 8><<<g, blk(), 0, s>>>(part, V, m, w, n, N);
    else if (m <= 16) k_multidot<C, 16><<<g, blk(), 0, s>>>(part, V, m, w, n, N);
    else if (m <= 32) k_multidot<C, 32><<<g, blk(), 0, s>>>(part, V, m, w, n, N);
    else k_multidot<C, 64><<<g, blk(), 0, s>>>(part, V, m, w, n, N);
    MG_LAUNCHED();
    launch_finalize(out, part, G, m * N, s);
}
template <typename C>
void launch_multiaxpy(C* w, const double2* coef, int m, const C* V, double sign, long long n, int N, cudaStream_t s,
                      const double* eta, int eta_pow, bool accumulate) {
    MG_REQUIRE(m >= 1 && m <= 64, MGMLMC_EINVAL, "multiaxpy: 1 <= m <= 64");
    MG_REQUIRE(!eta || eta_pow == 1 || eta_pow == 2, MGMLMC_EINVAL, "multiaxpy: eta_pow is 1 or 2");
    k_multiaxpy<C><<<dim3(rhs_tiles(N), axpy_groups(n, N)), blk(), 0, s>>>(w, coef, m, V, sign, n, N, nullptr, eta,
                                                                          eta_pow, accumulate ? 1 : 0, nullptr);
    MG_LAUNCHED();
}
template <typename C>
void launch_multiaxpy_norm2(C* w, const double2* coef, int m, const C* V, double sign, long long n, int N,
                            double* norm2, double* part, cudaStream_t s, const double* eta, int eta_pow,
                            const double* norm_div) {
    MG_REQUIRE(m >= 1 && m <= 64, MGMLMC_EINVAL, "multiaxpy: 1 <= m <= 64");
    MG_REQUIRE(!eta || eta_pow == 1 || eta_pow == 2, MGMLMC_EINVAL, "multiaxpy: eta_pow is 1 or 2");
    const int G = axpy_groups(n, N);
    k_multiaxpy<C><<<dim3(rhs_tiles(N), G), blk(), 0, s>>>(w, coef, m, V, sign, n, N, part, eta, eta_pow, 1,
                                                            norm_div);
    MG_LAUNCHED();
    launch_finalize(norm2, part, G, N, s);
}

#define INST_C(C)                                                                                   \
    template void launch_noise<C>(C*, long long, int, uint64_t, uint64_t, int64_t, cudaStream_t);    \
    template void launch_probes<C>(C*, const int8_t*, long long, int, cudaStream_t);                 \
    template void launch_zero<C>(C*, long long, cudaStream_t);                                       \
    template void launch_scale_cols_if<C>(C*, const double*, long long, int, cudaStream_t);          \
    template void launch_norm2<C>(double*, const C*, long long, int, double*, cudaStream_t);         \
    template void launch_multidot<C>(double2*, const C*, int, const C*, long long, int, double2*,    \
                                     cudaStream_t);                                                  \
    template void launch_multiaxpy<C>(C*, const double2*, int, const C*, double, long long, int,     \
                                      cudaStream_t, const double*, int, bool);                       \
    template void launch_multiaxpy_norm2<C>(C*, const double2*, int, const C*, double, long long, int, \
                                            double*, double*, cudaStream_t, const double*, int,        \
                                            const double*);
INST_C(double2)
INST_C(float2)
#define INST_CC(A, B)                                                                               \
    template void launch_convert<A, B>(A*, const B*, long long, cudaStream_t);                       \
    template void launch_scale_rhs<A, B>(A*, const B*, const double*, bool, long long, int,          \
                                         cudaStream_t);                                              \
    template void launch_axpy_rhs<A, B>(A*, const double2*, const double*, double, const B*,         \
                                        long long, int, cudaStream_t);
INST_CC(double2, double2)
INST_CC(float2, float2)
INST_CC(double2, float2)
INST_CC(float2, double2)
template void launch_dot<double2, double2>(double2*, const double2*, const double2*, long long, int, double2*,
                                           cudaStream_t);
template void launch_dot<float2, float2>(double2*, const float2*, const float2*, long long, int, double2*,
                                         cudaStream_t);

}  // namespace mg

namespace mg {
// out[c][r] = in[r][c] for a rows x cols complex matrix (32 x 32 tiles).
__global__ void k_transpose(double2* __restrict__ out, const double2* __restrict__ in, long long rows, int cols) {
    __shared__ double2 t[32][33];
    const int c0 = blockIdx.x * 32;
    const long long nrb = (rows + 31) / 32;
    for (long long rb = blockIdx.y; rb < nrb; rb += gridDim.y) {      // grid-stride over 32-row blocks
        const long long r0 = rb * 32;
        __syncthreads();
        for (int k = threadIdx.y; k < 32; k += blockDim.y) {
            const long long r = r0 + k;
            const int cc = c0 + threadIdx.x;
            if (r < rows && cc < cols) t[k][threadIdx.x] = in[r * cols + cc];
        }
        __syncthreads();
        for (int k = threadIdx.y; k < 32; k += blockDim.y) {
            const int cc = c0 + k;
            const long long r = r0 + threadIdx.x;
            if (r < rows && cc < cols) out[(long long)cc * rows + r] = t[threadIdx.x][k];
        }
    }
}
void launch_transpose(double2* out, const double2* in, long long rows, int cols, cudaStream_t s) {
    const long long nrb = (rows + 31) / 32;
    dim3 g((cols + 31) / 32, (unsigned)(nrb < 65535 ? nrb : 65535));
    k_transpose<<<g, dim3(32, 8), 0, s>>>(out, in, rows, cols);
    MG_LAUNCHED();
}
}  // namespace mg
