// Stencil kernels: the fine Wilson-Schwinger operator D_1, the coarse 5-point
// block stencils D_l (l >= 2), restriction P^H, prolongation P, Gamma5 and the
// fused minimal-residual smoother update.
//
// The fine operator (the paper names the 2D Wilson-Schwinger discretisation,
// Sect. 1; its form is the standard Wilson one):
//   (D psi)(x) = (m0+2) psi(x) - 1/2 sum_mu [(1 - s_mu) U_mu(x) psi(x+mu)
//                                          + (1 + s_mu) U_mu(x-mu)^* psi(x-mu)]
// with s_0 = sigma_1, s_1 = sigma_2, antiperiodic in time.  Each hop needs a
// single complex multiply: (1 -+ s_mu) projects the 2-spinor onto one
// component (e.g. (1 - sigma_1) psi = (a, -a) with a = psi_0 - psi_1).
#include <algorithm>

#include "kernels.cuh"

namespace mg {

// Threads of the one-rhs-per-thread CTAs: 128, or fewer for narrower blocks so that
// no lane idles (N = 64: two warps).
static int cta_threads(int N) { return std::min(128, (N + 31) / 32 * 32); }

template <typename C, int MODE>
__global__ void __launch_bounds__(256) k_wilson(C* __restrict__ y, const C* __restrict__ x, const C* __restrict__ b,
                                                const C* __restrict__ U, re_t<C> mass, int lx, int lt, int N,
                                                double2* __restrict__ part) {
    using R = re_t<C>;
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    const int V = lx * lt;
    const R half = (R)0.5;
    C dyx = czero<C>();
    R dyy = 0;
    if (j < N) {
        for (int site = blockIdx.y * kRowLanes + threadIdx.y; site < V; site += gridDim.y * kRowLanes) {
            const int xx = site % lx, t = site / lx;
            const int sxp = (xx + 1 == lx ? 0 : xx + 1) + lx * t;
            const int sxm = (xx == 0 ? lx - 1 : xx - 1) + lx * t;
            const int stp = xx + lx * (t + 1 == lt ? 0 : t + 1);
            const int stm = xx + lx * (t == 0 ? lt - 1 : t - 1);
            const R sgp = (t + 1 == lt) ? (R)-0.5 : half;   // antiperiodic time boundary, times 1/2
            const R sgm = (t == 0) ? (R)-0.5 : half;
            const C u0 = U[2 * site], u1 = U[2 * site + 1];
            const C u0m = U[2 * sxm], u1m = U[2 * stm + 1];
            const long long N2 = 2LL * N;
            const C p0 = x[site * N2 + j], p1 = x[site * N2 + N + j];
            C o0 = mk(mass * p0.x, mass * p0.y), o1 = mk(mass * p1.x, mass * p1.y);
            {   // +x: (1 - sigma_1) psi = (a, -a), a = psi0 - psi1
                const C q0 = x[sxp * N2 + j], q1 = x[sxp * N2 + N + j];
                const C u = cscale(cmul(u0, csub(q0, q1)), half);
                o0 = csub(o0, u);
                o1 = cadd(o1, u);
            }
            {   // -x: (1 + sigma_1) psi = (c, c), c = psi0 + psi1
                const C q0 = x[sxm * N2 + j], q1 = x[sxm * N2 + N + j];
                const C u = cscale(cmulc(u0m, cadd(q0, q1)), half);
                o0 = csub(o0, u);
                o1 = csub(o1, u);
            }
            {   // +t: (1 - sigma_2) psi = (a, -i a), a = psi0 + i psi1
                const C q0 = x[stp * N2 + j], q1 = x[stp * N2 + N + j];
                const C u = cscale(cmul(u1, cadd(q0, ctimesi(q1))), sgp);
                o0 = csub(o0, u);
                o1 = cadd(o1, ctimesi(u));
            }
            {   // -t: (1 + sigma_2) psi = (c, i c), c = psi0 - i psi1
                const C q0 = x[stm * N2 + j], q1 = x[stm * N2 + N + j];
                const C u = cscale(cmulc(u1m, csub(q0, ctimesi(q1))), sgm);
                o0 = csub(o0, u);
                o1 = csub(o1, ctimesi(u));
            }
            if (MODE == 1) {
                o0 = csub(b[site * N2 + j], o0);
                o1 = csub(b[site * N2 + N + j], o1);
            }
            y[site * N2 + j] = o0;
            y[site * N2 + N + j] = o1;
            if (MODE == 2) {
                cfmac(dyx, o0, p0);
                cfmac(dyx, o1, p1);
                dyy = fma(o0.x, o0.x, fma(o0.y, o0.y, fma(o1.x, o1.x, fma(o1.y, o1.y, dyy))));
            }
        }
    }
    if (MODE == 2) {
        __shared__ double2 sh[2][kRowLanes][kRhsTile + 1];
        sh[0][threadIdx.y][threadIdx.x] = to_d(dyx);
        sh[1][threadIdx.y][threadIdx.x] = make_double2((double)dyy, 0.0);
        __syncthreads();
        if (threadIdx.y < 2 && j < N) {
            double2 s = sh[threadIdx.y][0][threadIdx.x];
            for (int r = 1; r < kRowLanes; ++r) s = cadd(s, sh[threadIdx.y][r][threadIdx.x]);
            part[((long long)threadIdx.y * N + j) * gridDim.y + blockIdx.y] = s;
        }
    }
}


// One block per coarse site (grid-stride): A[site] (5 d^2 complex) staged in
// shared memory, each thread owns one rhs and RPT output rows.
template <typename C, int RPT, int MODE>
__global__ void __launch_bounds__(256) k_block_stencil(C* __restrict__ y, const C* __restrict__ x,
                                                       const C* __restrict__ b, const C* __restrict__ A, int lx,
                                                       int lt, int d, int N, double2* __restrict__ part) {
    using R = re_t<C>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* As = reinterpret_cast<C*>(smem_raw);
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    const int V = lx * lt;
    const int nA = 5 * d * d;
    const int tid = threadIdx.y * kRhsTile + threadIdx.x;
    C dyx = czero<C>();
    R dyy = 0;
    for (int site = blockIdx.y; site < V; site += gridDim.y) {
        __syncthreads();
        for (int e = tid; e < nA; e += kRhsTile * kRowLanes) As[e] = A[(long long)site * nA + e];
        __syncthreads();
        if (j < N) {
            C acc[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) acc[r] = czero<C>();
            for (int dir = 0; dir < 5; ++dir) {
                const int nb = nbr_site(site, dir, lx, lt);
                const C* xn = x + (long long)nb * d * N + j;
                const C* Ad = As + dir * d * d;
                for (int bc = 0; bc < d; ++bc) {
                    const C xv = xn[(long long)bc * N];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        const int c = threadIdx.y + kRowLanes * r;
                        if (c < d) cfma(acc[r], Ad[c * d + bc], xv);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int c = threadIdx.y + kRowLanes * r;
                if (c < d) {
                    const long long idx = ((long long)site * d + c) * N + j;
                    C o = acc[r];
                    if (MODE == 1) o = csub(b[idx], o);
                    y[idx] = o;
                    if (MODE == 2) {
                        cfmac(dyx, o, x[idx]);
                        dyy = fma(o.x, o.x, fma(o.y, o.y, dyy));
                    }
                }
            }
        }
    }
    if (MODE == 2) {
        __syncthreads();
        double2* sh = reinterpret_cast<double2*>(smem_raw);   // reuse: [2][8][33]
        sh[(0 * kRowLanes + threadIdx.y) * (kRhsTile + 1) + threadIdx.x] = to_d(dyx);
        sh[(1 * kRowLanes + threadIdx.y) * (kRhsTile + 1) + threadIdx.x] = make_double2((double)dyy, 0.0);
        __syncthreads();
        if (threadIdx.y < 2 && j < N) {
            double2 s = sh[(threadIdx.y * kRowLanes) * (kRhsTile + 1) + threadIdx.x];
            for (int r = 1; r < kRowLanes; ++r)
                s = cadd(s, sh[(threadIdx.y * kRowLanes + r) * (kRhsTile + 1) + threadIdx.x]);
            part[((long long)threadIdx.y * N + j) * gridDim.y + blockIdx.y] = s;
        }
    }
}

// Site-per-thread-row variant for compile-time d: block = 128 rhs, each thread
// computes all d outputs of one site for its rhs, so every input value loaded
// is used d times.  The blocks are staged transposed, At[dir][b][c], so the
// inner loop over output rows reads consecutive shared-memory words (broadcast
// to the whole warp).
template <typename C, int D, int MODE>
__global__ void __launch_bounds__(128) k_block_stencil_d(C* __restrict__ y, const C* __restrict__ x,
                                                         const C* __restrict__ b, const C* __restrict__ A, int lx,
                                                         int lt, int N, double2* __restrict__ part) {
    using R = re_t<C>;
    __shared__ C At[5 * D * D];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int V = lx * lt;
    C dyx = czero<C>();
    R dyy = 0;
    for (int site = blockIdx.y; site < V; site += gridDim.y) {
        __syncthreads();
        for (int e = threadIdx.x; e < 5 * D * D; e += blockDim.x) {
            const int dir = e / (D * D), r = e % (D * D), c = r / D, bb = r % D;
            At[(dir * D + bb) * D + c] = A[(long long)site * 5 * D * D + e];
        }
        __syncthreads();
        if (j < N) {
            C acc[D];
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] = czero<C>();
#pragma unroll 1
            for (int dir = 0; dir < 5; ++dir) {
                const int nb = nbr_site(site, dir, lx, lt);
                const C* xn = x + (long long)nb * D * N + j;
                const C* Ad = At + dir * D * D;
#pragma unroll 4
                for (int bc = 0; bc < D; ++bc) {
                    const C xv = xn[(long long)bc * N];
#pragma unroll
                    for (int c = 0; c < D; ++c) cfma(acc[c], Ad[bc * D + c], xv);
                }
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const long long idx = ((long long)site * D + c) * N + j;
                C o = acc[c];
                if (MODE == 1) o = csub(b[idx], o);
                y[idx] = o;
                if (MODE == 2) {
                    cfmac(dyx, o, x[idx]);
                    dyy = fma(o.x, o.x, fma(o.y, o.y, dyy));
                }
            }
        }
    }
    if (MODE == 2) {
        // per-rhs partials: one thread per rhs, no cross-thread reduction needed
        if (j < N) {
            part[((long long)0 * N + j) * gridDim.y + blockIdx.y] = to_d(dyx);
            part[((long long)1 * N + j) * gridDim.y + blockIdx.y] = make_double2((double)dyy, 0.0);
        }
    }
}

// FP32 variant with two adjacent right-hand sides per thread: one 16-byte load
// brings x for both, and every shared-memory read of the block serves two rhs.
// Block = 128 threads = 256 rhs.  N must be even.
template <int D, int MODE>
__global__ void __launch_bounds__(128) k_block_stencil_f2(float2* __restrict__ y, const float2* __restrict__ x,
                                                          const float2* __restrict__ b, const float2* __restrict__ A,
                                                          int lx, int lt, int N, double2* __restrict__ part) {
    __shared__ float2 At[5 * D * D];
    // blockDim.x threads (32..128) x 2 rhs each: blocks of 64 rhs use one-warp CTAs
    const int j = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int V = lx * lt;
    float2 dyx0 = make_float2(0.f, 0.f), dyx1 = make_float2(0.f, 0.f);
    float dyy0 = 0.f, dyy1 = 0.f;
    for (int site = blockIdx.y; site < V; site += gridDim.y) {
        __syncthreads();
        for (int e = threadIdx.x; e < 5 * D * D; e += blockDim.x) {
            const int dir = e / (D * D), r = e % (D * D), c = r / D, bb = r % D;
            At[(dir * D + bb) * D + c] = A[(long long)site * 5 * D * D + e];
        }
        __syncthreads();
        if (j < N) {
            float2 a0[D], a1[D];
#pragma unroll
            for (int c = 0; c < D; ++c) a0[c] = a1[c] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int dir = 0; dir < 5; ++dir) {
                const int nb = nbr_site(site, dir, lx, lt);
                const float2* xn = x + (long long)nb * D * N + j;
                const float2* Ad = At + dir * D * D;
                // the neighbour's rows in groups of 4, loads first (latency of L2 hits)
#pragma unroll 1
                for (int b0 = 0; b0 < D; b0 += 4) {
                    float4 xv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) xv[q] = *reinterpret_cast<const float4*>(xn + (long long)(b0 + q) * N);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 x0 = make_float2(xv[q].x, xv[q].y), x1 = make_float2(xv[q].z, xv[q].w);
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            const float2 av = Ad[(b0 + q) * D + c];
                            cfma(a0[c], av, x0);
                            cfma(a1[c], av, x1);
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const long long idx = ((long long)site * D + c) * N + j;
                float2 o0 = a0[c], o1 = a1[c];
                if (MODE == 1) {
                    const float4 bv = *reinterpret_cast<const float4*>(b + idx);
                    o0 = make_float2(bv.x - o0.x, bv.y - o0.y);
                    o1 = make_float2(bv.z - o1.x, bv.w - o1.y);
                }
                *reinterpret_cast<float4*>(y + idx) = make_float4(o0.x, o0.y, o1.x, o1.y);
                if (MODE == 2) {
                    const float4 xv = *reinterpret_cast<const float4*>(x + idx);
                    cfmac(dyx0, o0, make_float2(xv.x, xv.y));
                    cfmac(dyx1, o1, make_float2(xv.z, xv.w));
                    dyy0 = fmaf(o0.x, o0.x, fmaf(o0.y, o0.y, dyy0));
                    dyy1 = fmaf(o1.x, o1.x, fmaf(o1.y, o1.y, dyy1));
                }
            }
        }
    }
    if (MODE == 2 && j < N) {
        const long long G = gridDim.y;
        part[((long long)0 * N + j) * G + blockIdx.y] = to_d(dyx0);
        part[((long long)0 * N + j + 1) * G + blockIdx.y] = to_d(dyx1);
        part[((long long)1 * N + j) * G + blockIdx.y] = make_double2((double)dyy0, 0.0);
        part[((long long)1 * N + j + 1) * G + blockIdx.y] = make_double2((double)dyy1, 0.0);
    }
}

// FP32 variant for d = 16 with four adjacent right-hand sides per thread and the 16
// output rows of a site split over the two halves of the CTA (half h, uniform per warp,
// computes rows 8h .. 8h + 7).  Each shared-memory read of a block entry serves four
// rhs, 16 FMA per 8 bytes read, twice as many as with two rhs per thread, whose FMA pipe
// waits on the shared-memory reads.  Per output the sums run in the same order as in
// k_block_stencil_f2, so y is the same; the MODE 2 dots add the two halves last.
// Block = 2 T threads with T = blockDim.x / 2 a multiple of 32; N % 4 == 0.
template <int MODE>
__global__ void __launch_bounds__(128) k_block_stencil_f4(float2* __restrict__ y, const float2* __restrict__ x,
                                                          const float2* __restrict__ b, const float2* __restrict__ A,
                                                          int lx, int lt, int N, double2* __restrict__ part) {
    constexpr int D = 16, H = 8;
    __shared__ float2 At[5 * D * D];
    __shared__ float red[MODE == 2 ? 64 * 12 : 1];     // half 1's dots, T <= 64
    const int T = blockDim.x >> 1;
    const int h = threadIdx.x >= T ? 1 : 0;
    const int tq = threadIdx.x - h * T;
    const int j = 4 * (blockIdx.x * T + tq);
    const int V = lx * lt;
    float2 dyx[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float dyy[4] = {0.f, 0.f, 0.f, 0.f};
    for (int site = blockIdx.y; site < V; site += gridDim.y) {
        __syncthreads();
        for (int e = threadIdx.x; e < 5 * D * D; e += blockDim.x) {
            const int dir = e / (D * D), r = e % (D * D), c = r / D, bb = r % D;
            At[(dir * D + bb) * D + c] = A[(long long)site * 5 * D * D + e];
        }
        __syncthreads();
        if (j < N) {
            float2 a[H][4];
#pragma unroll
            for (int c = 0; c < H; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) a[c][r] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int dir = 0; dir < 5; ++dir) {
                const int nb = nbr_site(site, dir, lx, lt);
                const float2* xn = x + (long long)nb * D * N + j;
                const float2* Ad = At + dir * D * D + h * H;
                // the neighbour's rows in groups of 4, loads first (latency of L2 hits)
#pragma unroll 1
                for (int b0 = 0; b0 < D; b0 += 4) {
                    float4 xv[4][2];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        xv[q][0] = *reinterpret_cast<const float4*>(xn + (long long)(b0 + q) * N);
                        xv[q][1] = *reinterpret_cast<const float4*>(xn + (long long)(b0 + q) * N + 2);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 x0 = make_float2(xv[q][0].x, xv[q][0].y), x1 = make_float2(xv[q][0].z, xv[q][0].w);
                        const float2 x2 = make_float2(xv[q][1].x, xv[q][1].y), x3 = make_float2(xv[q][1].z, xv[q][1].w);
#pragma unroll
                        for (int c = 0; c < H; ++c) {
                            const float2 av = Ad[(b0 + q) * D + c];
                            cfma(a[c][0], av, x0);
                            cfma(a[c][1], av, x1);
                            cfma(a[c][2], av, x2);
                            cfma(a[c][3], av, x3);
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < H; ++c) {
                const long long idx = ((long long)site * D + h * H + c) * N + j;
                float2 o[4] = {a[c][0], a[c][1], a[c][2], a[c][3]};
                if (MODE == 1) {
                    const float4 b0v = *reinterpret_cast<const float4*>(b + idx);
                    const float4 b1v = *reinterpret_cast<const float4*>(b + idx + 2);
                    o[0] = make_float2(b0v.x - o[0].x, b0v.y - o[0].y);
                    o[1] = make_float2(b0v.z - o[1].x, b0v.w - o[1].y);
                    o[2] = make_float2(b1v.x - o[2].x, b1v.y - o[2].y);
                    o[3] = make_float2(b1v.z - o[3].x, b1v.w - o[3].y);
                }
                *reinterpret_cast<float4*>(y + idx) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                *reinterpret_cast<float4*>(y + idx + 2) = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
                if (MODE == 2) {
                    const float4 x0v = *reinterpret_cast<const float4*>(x + idx);
                    const float4 x1v = *reinterpret_cast<const float4*>(x + idx + 2);
                    const float2 xs[4] = {make_float2(x0v.x, x0v.y), make_float2(x0v.z, x0v.w),
                                          make_float2(x1v.x, x1v.y), make_float2(x1v.z, x1v.w)};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        cfmac(dyx[r], o[r], xs[r]);
                        dyy[r] = fmaf(o[r].x, o[r].x, fmaf(o[r].y, o[r].y, dyy[r]));
                    }
                }
            }
        }
    }
    if (MODE == 2) {
        // half 1 hands its sums to half 0, which writes the per-rhs partials
        if (h == 1)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                red[tq * 12 + 3 * r] = dyx[r].x;
                red[tq * 12 + 3 * r + 1] = dyx[r].y;
                red[tq * 12 + 3 * r + 2] = dyy[r];
            }
        __syncthreads();
        if (h == 0 && j < N) {
            const long long G = gridDim.y;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float2 s = make_float2(dyx[r].x + red[tq * 12 + 3 * r], dyx[r].y + red[tq * 12 + 3 * r + 1]);
                part[((long long)0 * N + j + r) * G + blockIdx.y] = to_d(s);
                part[((long long)1 * N + j + r) * G + blockIdx.y] =
                    make_double2((double)(dyy[r] + red[tq * 12 + 3 * r + 2]), 0.0);
            }
        }
    }
}

// Narrow-block variant (few rhs, as in the setup solves): thread (tx < 8 rhs,
// ty < D output row); the blocks of the site are staged in shared memory.
template <typename C, int D, int MODE>
__global__ void __launch_bounds__(8 * D) k_block_stencil_narrow(C* __restrict__ y, const C* __restrict__ x,
                                                                const C* __restrict__ b, const C* __restrict__ A,
                                                                int lx, int lt, int N, double2* __restrict__ part) {
    using R = re_t<C>;
    __shared__ C As[5 * D * D];
    __shared__ double2 red[2][D][8];
    const int tx = threadIdx.x, c = threadIdx.y, tid = c * 8 + tx;
    const int j = blockIdx.x * 8 + tx;
    const int V = lx * lt;
    C dyx = czero<C>();
    R dyy = 0;
    for (int site = blockIdx.y; site < V; site += gridDim.y) {
        __syncthreads();
        for (int e = tid; e < 5 * D * D; e += 8 * D) As[e] = A[(long long)site * 5 * D * D + e];
        __syncthreads();
        if (j < N) {
            C acc = czero<C>();
            for (int dir = 0; dir < 5; ++dir) {
                const int nb = nbr_site(site, dir, lx, lt);
                const C* xn = x + (long long)nb * D * N + j;
                const C* Ar = As + (dir * D + c) * D;
#pragma unroll
                for (int bc = 0; bc < D; ++bc) cfma(acc, Ar[bc], xn[(long long)bc * N]);
            }
            const long long idx = ((long long)site * D + c) * N + j;
            if (MODE == 1) acc = csub(b[idx], acc);
            y[idx] = acc;
            if (MODE == 2) {
                cfmac(dyx, acc, x[idx]);
                dyy = fma(acc.x, acc.x, fma(acc.y, acc.y, dyy));
            }
        }
    }
    if (MODE == 2) {
        red[0][c][tx] = to_d(dyx);
        red[1][c][tx] = make_double2((double)dyy, 0.0);
        __syncthreads();
        if (c < 2 && j < N) {
            double2 s2 = red[c][0][tx];
            for (int r = 1; r < D; ++r) s2 = cadd(s2, red[c][r][tx]);
            part[((long long)c * N + j) * gridDim.y + blockIdx.y] = s2;
        }
    }
}

// y[s] (+)= Minv[s] x[s]: block = 128 rhs, one site per iteration, Minv[s] in
// shared memory; generic d (<= 32).
template <typename C>
__global__ void __launch_bounds__(128) k_block_diag_apply(C* __restrict__ y, const C* __restrict__ x,
                                                          const C* __restrict__ Minv, int nsites, int d, int N,
                                                          bool accumulate) {
    __shared__ C Ms[32 * 32];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int site = blockIdx.y; site < nsites; site += gridDim.y) {
        __syncthreads();
        for (int e = threadIdx.x; e < d * d; e += blockDim.x) Ms[e] = Minv[(long long)site * d * d + e];
        __syncthreads();
        if (j >= N) continue;
        C xv[32];
        for (int b = 0; b < d; ++b) xv[b] = x[((long long)site * d + b) * N + j];
        for (int c = 0; c < d; ++c) {
            C acc = accumulate ? y[((long long)site * d + c) * N + j] : czero<C>();
            for (int b = 0; b < d; ++b) cfma(acc, Ms[c * d + b], xv[b]);
            y[((long long)site * d + c) * N + j] = acc;
        }
    }
}

// The same with the block size fixed at compile time: the input column stays in
// registers (a runtime d puts it in local memory), all loads issued before the FMAs.
template <typename C, int D>
__global__ void __launch_bounds__(128) k_block_diag_apply_d(C* __restrict__ y, const C* __restrict__ x,
                                                            const C* __restrict__ Minv, int nsites, int N,
                                                            bool accumulate) {
    __shared__ C Ms[D * D];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int site = blockIdx.y; site < nsites; site += gridDim.y) {
        __syncthreads();
        for (int e = threadIdx.x; e < D * D; e += blockDim.x) Ms[e] = Minv[(long long)site * D * D + e];
        __syncthreads();
        if (j >= N) continue;
        C xv[D], acc[D];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            xv[b] = x[((long long)site * D + b) * N + j];
            acc[b] = accumulate ? y[((long long)site * D + b) * N + j] : czero<C>();
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
#pragma unroll
            for (int b = 0; b < D; ++b) cfma(acc[c], Ms[c * D + b], xv[b]);
            y[((long long)site * D + c) * N + j] = acc[c];
        }
    }
}

template <typename C>
void launch_block_diag_apply(C* y, const C* x, const C* Minv, int nsites, int d, int N, bool accumulate,
                             cudaStream_t s) {
    MG_REQUIRE(d <= 32, MGMLMC_EINVAL, "block-diagonal apply: d <= 32");
    const int th = cta_threads(N);
    const int tiles = (N + th - 1) / th;
    int G = 16 * kNumSM / tiles;
    if (G > nsites) G = nsites;
    if (G < 1) G = 1;
    if (d == 16) k_block_diag_apply_d<C, 16><<<dim3(tiles, G), th, 0, s>>>(y, x, Minv, nsites, N, accumulate);
    else if (d == 8) k_block_diag_apply_d<C, 8><<<dim3(tiles, G), th, 0, s>>>(y, x, Minv, nsites, N, accumulate);
    else k_block_diag_apply<C><<<dim3(tiles, G), th, 0, s>>>(y, x, Minv, nsites, d, N, accumulate);
    MG_LAUNCHED();
}

// xc[S][o] = sum_{site in S} sum_{a in spin block s(o)} conj(P[site][a][j(o)]) x[site][a]
template <typename C>
__global__ void k_restrict(C* __restrict__ xc, const C* __restrict__ x, const C* __restrict__ P, int lx, int lt,
                           int d, int ax, int at, int nvec, int N) {
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    const int cx = lx / ax, ct = lt / at, dc = 2 * nvec, hd = d / 2;
    for (int S = blockIdx.y; S < cx * ct; S += gridDim.y) {
        const int X = S % cx, T = S / cx;
        for (int o = threadIdx.y; o < dc; o += kRowLanes) {
            const int s = o / nvec, jv = o % nvec;
            C acc = czero<C>();
            for (int it = 0; it < at; ++it)
                for (int ix = 0; ix < ax; ++ix) {
                    const int site = (X * ax + ix) + lx * (T * at + it);
                    for (int a = s * hd; a < (s + 1) * hd; ++a)
                        cfmac(acc, P[((long long)site * d + a) * nvec + jv], x[((long long)site * d + a) * N + j]);
                }
            xc[((long long)S * dc + o) * N + j] = acc;
        }
    }
}

// x[site][a] (+)= sum_j P[site][a][j] xc[S(site)][s(a) nvec + j]
template <typename C>
__global__ void k_prolong(C* __restrict__ x, const C* __restrict__ xc, const C* __restrict__ P, int lx, int lt,
                          int d, int ax, int at, int nvec, int N, bool accumulate) {
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    const int cx = lx / ax, dc = 2 * nvec, hd = d / 2;
    const long long rows = (long long)lx * lt * d;
    for (long long row = (long long)blockIdx.y * kRowLanes + threadIdx.y; row < rows;
         row += (long long)gridDim.y * kRowLanes) {
        const int site = (int)(row / d), a = (int)(row % d);
        const int xx = site % lx, t = site / lx;
        const int S = xx / ax + cx * (t / at);
        const int s = a / hd;
        C acc = accumulate ? x[row * N + j] : czero<C>();
        const C* Pr = P + row * nvec;
        const C* xcs = xc + ((long long)S * dc + s * nvec) * N + j;
        for (int jv = 0; jv < nvec; ++jv) cfma(acc, Pr[jv], xcs[(long long)jv * N]);
        x[row * N + j] = acc;
    }
}

// Aggregate-per-block restriction / prolongation for compile-time nvec: block =
// 128 rhs, one coarse site S per block iteration; P restricted to S (ax*at*d*nvec
// values) staged in shared memory; each thread reads every fine value of its rhs
// once and keeps the 2 nvec coarse values in registers.
template <typename C, int NV>
__global__ void __launch_bounds__(128) k_restrict_nv(C* __restrict__ xc, const C* __restrict__ x,
                                                     const C* __restrict__ P, int lx, int lt, int d, int ax, int at,
                                                     int N) {
    extern __shared__ __align__(16) unsigned char smem_rp[];
    C* Ps = reinterpret_cast<C*>(smem_rp);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = lx / ax, ct = lt / at, hd = d / 2, na = ax * at;
    const int nP = na * d * NV;
    for (int S = blockIdx.y; S < cx * ct; S += gridDim.y) {
        const int X = S % cx, T = S / cx;
        __syncthreads();
        for (int e = threadIdx.x; e < nP; e += blockDim.x) {
            const int q = e / (d * NV), r = e % (d * NV);
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            Ps[e] = P[(long long)site * d * NV + r];
        }
        __syncthreads();
        if (j >= N) continue;
        C acc[2 * NV];
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) acc[o] = czero<C>();
        for (int q = 0; q < na; ++q) {
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            const C* xs = x + (long long)site * d * N + j;
            const C* Pq = Ps + q * d * NV;
            for (int a = 0; a < d; ++a) {
                const C xv = xs[(long long)a * N];
                const C* Pa = Pq + a * NV;
                if (a < hd) {
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfmac(acc[jv], Pa[jv], xv);
                } else {
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfmac(acc[NV + jv], Pa[jv], xv);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) xc[((long long)S * 2 * NV + o) * N + j] = acc[o];
    }
}

template <typename C, int NV>
__global__ void __launch_bounds__(128) k_prolong_nv(C* __restrict__ x, const C* __restrict__ xc,
                                                    const C* __restrict__ P, int lx, int lt, int d, int ax, int at,
                                                    int N, bool accumulate) {
    extern __shared__ __align__(16) unsigned char smem_rp[];
    C* Ps = reinterpret_cast<C*>(smem_rp);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = lx / ax, ct = lt / at, hd = d / 2, na = ax * at;
    const int nP = na * d * NV;
    for (int S = blockIdx.y; S < cx * ct; S += gridDim.y) {
        const int X = S % cx, T = S / cx;
        __syncthreads();
        for (int e = threadIdx.x; e < nP; e += blockDim.x) {
            const int q = e / (d * NV), r = e % (d * NV);
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            Ps[e] = P[(long long)site * d * NV + r];
        }
        __syncthreads();
        if (j >= N) continue;
        C cv[2 * NV];
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) cv[o] = xc[((long long)S * 2 * NV + o) * N + j];
        for (int q = 0; q < na; ++q) {
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            C* xs = x + (long long)site * d * N + j;
            const C* Pq = Ps + q * d * NV;
            for (int a = 0; a < d; ++a) {
                const C* Pa = Pq + a * NV;
                C acc = accumulate ? xs[(long long)a * N] : czero<C>();
                if (a < hd) {
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfma(acc, Pa[jv], cv[jv]);
                } else {
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfma(acc, Pa[jv], cv[NV + jv]);
                }
                xs[(long long)a * N] = acc;
            }
        }
    }
}

// The same two operators with the dofs per fine site (D) fixed at compile time: the
// loads of QB aggregate sites (QB * D values per thread) are issued together before
// the FMAs, instead of one load per loop trip.
template <typename C, int NV, int D, int QB>
__global__ void __launch_bounds__(128) k_restrict_nvd(C* __restrict__ xc, const C* __restrict__ x,
                                                      const C* __restrict__ P, int lx, int lt, int ax, int at, int N) {
    extern __shared__ __align__(16) unsigned char smem_rp[];
    C* Ps = reinterpret_cast<C*>(smem_rp);
    constexpr int HD = D / 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = lx / ax, ct = lt / at, na = ax * at;
    const int nP = na * D * NV;
    for (int S = blockIdx.y; S < cx * ct; S += gridDim.y) {
        const int X = S % cx, T = S / cx;
        __syncthreads();
        for (int e = threadIdx.x; e < nP; e += blockDim.x) {
            const int q = e / (D * NV), r = e % (D * NV);
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            Ps[e] = P[(long long)site * D * NV + r];
        }
        __syncthreads();
        if (j >= N) continue;
        C acc[2 * NV];
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) acc[o] = czero<C>();
        for (int q0 = 0; q0 < na; q0 += QB) {
            C xv[QB][D];
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) {
                const int q = q0 + qq;
                const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
#pragma unroll
                for (int a = 0; a < D; ++a)
                    xv[qq][a] = q < na ? x[((long long)site * D + a) * N + j] : czero<C>();
            }
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) {
                if (q0 + qq >= na) break;
                const C* Pq = Ps + (q0 + qq) * D * NV;
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfmac(acc[(a < HD ? 0 : NV) + jv], Pq[a * NV + jv], xv[qq][a]);
            }
        }
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) xc[((long long)S * 2 * NV + o) * N + j] = acc[o];
    }
}

template <typename C, int NV, int D, int QB>
__global__ void __launch_bounds__(128) k_prolong_nvd(C* __restrict__ x, const C* __restrict__ xc,
                                                     const C* __restrict__ P, int lx, int lt, int ax, int at, int N,
                                                     bool accumulate) {
    extern __shared__ __align__(16) unsigned char smem_rp[];
    C* Ps = reinterpret_cast<C*>(smem_rp);
    constexpr int HD = D / 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = lx / ax, ct = lt / at, na = ax * at;
    const int nP = na * D * NV;
    for (int S = blockIdx.y; S < cx * ct; S += gridDim.y) {
        const int X = S % cx, T = S / cx;
        __syncthreads();
        for (int e = threadIdx.x; e < nP; e += blockDim.x) {
            const int q = e / (D * NV), r = e % (D * NV);
            const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
            Ps[e] = P[(long long)site * D * NV + r];
        }
        __syncthreads();
        if (j >= N) continue;
        C cv[2 * NV];
#pragma unroll
        for (int o = 0; o < 2 * NV; ++o) cv[o] = xc[((long long)S * 2 * NV + o) * N + j];
        for (int q0 = 0; q0 < na; q0 += QB) {
            C ov[QB][D];
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) {
                const int q = q0 + qq;
                const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
#pragma unroll
                for (int a = 0; a < D; ++a)
                    ov[qq][a] = (accumulate && q < na) ? x[((long long)site * D + a) * N + j] : czero<C>();
            }
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) {
                const int q = q0 + qq;
                if (q >= na) break;
                const int site = (X * ax + q % ax) + lx * (T * at + q / ax);
                const C* Pq = Ps + q * D * NV;
#pragma unroll
                for (int a = 0; a < D; ++a) {
#pragma unroll
                    for (int jv = 0; jv < NV; ++jv) cfma(ov[qq][a], Pq[a * NV + jv], cv[(a < HD ? 0 : NV) + jv]);
                    x[((long long)site * D + a) * N + j] = ov[qq][a];
                }
            }
        }
    }
}

template <typename C>
__global__ void k_mr_update(C* __restrict__ e, C* __restrict__ r, const C* __restrict__ p,
                            const double2* __restrict__ dots, long long n, int N, bool e_is_zero) {
    using R = re_t<C>;
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    const double2 pr = dots[j];
    const double pp = dots[N + j].x;
    const double2 al = (pp > 0.0) ? make_double2(pr.x / pp, pr.y / pp) : make_double2(0.0, 0.0);
    const C a = mk((R)al.x, (R)al.y);
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < n;
         i += (long long)gridDim.y * kRowLanes) {
        const long long idx = i * N + j;
        const C rv = r[idx];
        C ev = e_is_zero ? czero<C>() : e[idx];
        cfma(ev, a, rv);
        e[idx] = ev;
        C rn = rv;
        C ap = cmul(a, p[idx]);
        r[idx] = csub(rn, ap);
    }
}

template <typename C>
__global__ void k_gamma5(C* __restrict__ y, const C* __restrict__ x, long long rows, int d, int N) {
    const int j = blockIdx.x * kRhsTile + threadIdx.x;
    if (j >= N) return;
    for (long long i = (long long)blockIdx.y * kRowLanes + threadIdx.y; i < rows;
         i += (long long)gridDim.y * kRowLanes) {
        const C v = x[i * N + j];
        y[i * N + j] = ((int)(i % d) < d / 2) ? v : mk(-v.x, -v.y);
    }
}

// --------------------------------------------------------------------- launchers
static inline dim3 blk() { return dim3(kRhsTile, kRowLanes); }

int stencil_groups(int nsites, int N) { return row_groups(nsites, N, 8); }
// k_wilson_bf16 launches N / 128 (four rhs per thread) or N / 64 column blocks of 256
// threads, three resident per SM: row groups for one wave of three CTAs per SM.
int stencil_groups_bf16(int nsites, int N) {
    const int gx = (N % 128 == 0) ? N / 128 : (N / 2 + kRhsTile - 1) / kRhsTile;
    const long long need = (nsites + kRowLanes - 1) / kRowLanes;
    return (int)std::max(1LL, std::min(need, 3LL * kNumSM / gx));
}

// FP32 Wilson operator with two rhs per thread: 16-byte loads and stores (a warp
// moves 512 B per access), half the index arithmetic per rhs.  N even.
template <int MODE>
__global__ void __launch_bounds__(256) k_wilson_f2(float2* __restrict__ y, const float2* __restrict__ x,
                                                   const float2* __restrict__ b, const float2* __restrict__ U,
                                                   float mass, int lx, int lt, int N, double2* __restrict__ part) {
    const int j = 2 * (blockIdx.x * kRhsTile + threadIdx.x);
    const int V = lx * lt;
    float2 dyx[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float dyy[2] = {0.f, 0.f};
    auto ld2 = [&](const float2* base, long long idx, float2& a, float2& c) {
        const float4 v = *reinterpret_cast<const float4*>(base + idx);
        a = make_float2(v.x, v.y);
        c = make_float2(v.z, v.w);
    };
    if (j < N) {
        const long long N2 = 2LL * N;
        for (int site = blockIdx.y * kRowLanes + threadIdx.y; site < V; site += gridDim.y * kRowLanes) {
            const int xx = site % lx, t = site / lx;
            const int sxp = (xx + 1 == lx ? 0 : xx + 1) + lx * t;
            const int sxm = (xx == 0 ? lx - 1 : xx - 1) + lx * t;
            const int stp = xx + lx * (t + 1 == lt ? 0 : t + 1);
            const int stm = xx + lx * (t == 0 ? lt - 1 : t - 1);
            const float sgp = (t + 1 == lt) ? -0.5f : 0.5f;   // antiperiodic time boundary, times 1/2
            const float sgm = (t == 0) ? -0.5f : 0.5f;
            const float2 u0 = U[2 * site], u1 = U[2 * site + 1];
            const float2 u0m = U[2 * sxm], u1m = U[2 * stm + 1];
            float2 p0[2], p1[2], a0[2], a1[2], c0[2], c1[2], e0[2], e1[2], f0[2], f1[2];
            ld2(x, site * N2 + j, p0[0], p0[1]);
            ld2(x, site * N2 + N + j, p1[0], p1[1]);
            ld2(x, sxp * N2 + j, a0[0], a0[1]);
            ld2(x, sxp * N2 + N + j, a1[0], a1[1]);
            ld2(x, sxm * N2 + j, c0[0], c0[1]);
            ld2(x, sxm * N2 + N + j, c1[0], c1[1]);
            ld2(x, stp * N2 + j, e0[0], e0[1]);
            ld2(x, stp * N2 + N + j, e1[0], e1[1]);
            ld2(x, stm * N2 + j, f0[0], f0[1]);
            ld2(x, stm * N2 + N + j, f1[0], f1[1]);
            float2 o0[2], o1[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                o0[r] = mk(mass * p0[r].x, mass * p0[r].y);
                o1[r] = mk(mass * p1[r].x, mass * p1[r].y);
                {   // +x: (1 - sigma_1) psi = (a, -a), a = psi0 - psi1
                    const float2 u = cscale(cmul(u0, csub(a0[r], a1[r])), 0.5f);
                    o0[r] = csub(o0[r], u);
                    o1[r] = cadd(o1[r], u);
                }
                {   // -x: (1 + sigma_1) psi = (c, c), c = psi0 + psi1
                    const float2 u = cscale(cmulc(u0m, cadd(c0[r], c1[r])), 0.5f);
                    o0[r] = csub(o0[r], u);
                    o1[r] = csub(o1[r], u);
                }
                {   // +t: (1 - sigma_2) psi = (a, -i a), a = psi0 + i psi1
                    const float2 u = cscale(cmul(u1, cadd(e0[r], ctimesi(e1[r]))), sgp);
                    o0[r] = csub(o0[r], u);
                    o1[r] = cadd(o1[r], ctimesi(u));
                }
                {   // -t: (1 + sigma_2) psi = (c, i c), c = psi0 - i psi1
                    const float2 u = cscale(cmulc(u1m, csub(f0[r], ctimesi(f1[r]))), sgm);
                    o0[r] = csub(o0[r], u);
                    o1[r] = csub(o1[r], ctimesi(u));
                }
            }
            if (MODE == 1) {
                float2 b0[2], b1[2];
                ld2(b, site * N2 + j, b0[0], b0[1]);
                ld2(b, site * N2 + N + j, b1[0], b1[1]);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    o0[r] = csub(b0[r], o0[r]);
                    o1[r] = csub(b1[r], o1[r]);
                }
            }
            *reinterpret_cast<float4*>(y + site * N2 + j) = make_float4(o0[0].x, o0[0].y, o0[1].x, o0[1].y);
            *reinterpret_cast<float4*>(y + site * N2 + N + j) = make_float4(o1[0].x, o1[0].y, o1[1].x, o1[1].y);
            if (MODE == 2) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    cfmac(dyx[r], o0[r], p0[r]);
                    cfmac(dyx[r], o1[r], p1[r]);
                    dyy[r] = fmaf(o0[r].x, o0[r].x, fmaf(o0[r].y, o0[r].y,
                                  fmaf(o1[r].x, o1[r].x, fmaf(o1[r].y, o1[r].y, dyy[r]))));
                }
            }
        }
    }
    if (MODE == 2) {
        __shared__ double2 sh[2][kRowLanes][2 * kRhsTile + 1];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            sh[0][threadIdx.y][2 * threadIdx.x + r] = to_d(dyx[r]);
            sh[1][threadIdx.y][2 * threadIdx.x + r] = make_double2((double)dyy[r], 0.0);
        }
        __syncthreads();
        // 64 rhs x 2 quantities: threads (x, y < 4) add the 8 row lanes of one each
        const int q = threadIdx.y >> 1, jj = 2 * threadIdx.x + (threadIdx.y & 1);
        const int jo = 2 * blockIdx.x * kRhsTile + jj;
        if (threadIdx.y < 4 && jo < N) {
            double2 acc = sh[q][0][jj];
            for (int r = 1; r < kRowLanes; ++r) acc = cadd(acc, sh[q][r][jj]);
            part[((long long)q * N + jo) * gridDim.y + blockIdx.y] = acc;
        }
    }
}

template <typename C>
static bool wilson_f2(C*, const C*, const C*, const C*, re_t<C>, int, int, int, int, double2*, int, cudaStream_t) {
    return false;
}
template <>
bool wilson_f2<float2>(float2* y, const float2* x, const float2* b, const float2* U, float mass, int lx, int lt, int N,
                       int mode, double2* part, int groups, cudaStream_t s) {
    if (N % 2) return false;
    dim3 g((N / 2 + kRhsTile - 1) / kRhsTile, groups);
    switch (mode) {
        case 0: k_wilson_f2<0><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
        case 1: k_wilson_f2<1><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
        default: k_wilson_f2<2><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
    }
    MG_LAUNCHED();
    return true;
}

// ---------------------------------------------------------------------------
// Fine-level smoother with the residual and its image held in BF16 ([row][rhs],
// one bf16x2 per complex value): the operator y = D x with the MR dots
// conj(y).x, |y|^2 (FP32 arithmetic, two rhs per thread, 8-byte accesses), the
// FP32 -> BF16 packing and the MR update e (=|+=) alpha r, r -= alpha p.
__device__ __forceinline__ float2 bf2_lo(uint32_t w) { return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u)); }
__device__ __forceinline__ uint32_t f2_bf(float2 v) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t*>(&b);
}

// Four rhs per thread: 16-byte accesses (four bf16x2 words), ten loads of a site in
// flight per thread.  N % 4 == 0.
// RPT right-hand sides per thread (4: 16-byte accesses, a warp spans 128 rhs; 2: 8-byte
// accesses, 64 rhs, so that a block of 64 keeps every lane busy).
template <int RPT>
__global__ void __launch_bounds__(256, 3) k_wilson_bf16(uint32_t* __restrict__ y, const uint32_t* __restrict__ x,
                                                        const float2* __restrict__ U, float mass, int lx, int lt,
                                                        int N, double2* __restrict__ part) {
    const int j = RPT * (blockIdx.x * kRhsTile + threadIdx.x);
    const int V = lx * lt;
    float2 dyx[RPT];
    float dyy[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        dyx[r] = make_float2(0.f, 0.f);
        dyy[r] = 0.f;
    }
    auto ld4 = [&](long long idx, float2* v) {
        if constexpr (RPT == 4) {
            const uint4 w = *reinterpret_cast<const uint4*>(x + idx);
            v[0] = bf2_lo(w.x);
            v[1] = bf2_lo(w.y);
            v[2] = bf2_lo(w.z);
            v[3] = bf2_lo(w.w);
        } else {
            const uint2 w = *reinterpret_cast<const uint2*>(x + idx);
            v[0] = bf2_lo(w.x);
            v[1] = bf2_lo(w.y);
        }
    };
    if (j < N) {
        const long long N2 = 2LL * N;
        for (int site = blockIdx.y * kRowLanes + threadIdx.y; site < V; site += gridDim.y * kRowLanes) {
            const int xx = site % lx, t = site / lx;
            const int sxp = (xx + 1 == lx ? 0 : xx + 1) + lx * t;
            const int sxm = (xx == 0 ? lx - 1 : xx - 1) + lx * t;
            const int stp = xx + lx * (t + 1 == lt ? 0 : t + 1);
            const int stm = xx + lx * (t == 0 ? lt - 1 : t - 1);
            const float sgp = (t + 1 == lt) ? -0.5f : 0.5f;   // antiperiodic time boundary, times 1/2
            const float sgm = (t == 0) ? -0.5f : 0.5f;
            const float2 u0 = U[2 * site], u1 = U[2 * site + 1];
            const float2 u0m = U[2 * sxm], u1m = U[2 * stm + 1];
            float2 p0[RPT], p1[RPT], a0[RPT], a1[RPT], c0[RPT], c1[RPT], e0[RPT], e1[RPT], f0[RPT], f1[RPT];
            ld4(site * N2 + j, p0);
            ld4(site * N2 + N + j, p1);
            ld4(sxp * N2 + j, a0);
            ld4(sxp * N2 + N + j, a1);
            ld4(sxm * N2 + j, c0);
            ld4(sxm * N2 + N + j, c1);
            ld4(stp * N2 + j, e0);
            ld4(stp * N2 + N + j, e1);
            ld4(stm * N2 + j, f0);
            ld4(stm * N2 + N + j, f1);
            uint32_t w0[RPT], w1[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                float2 o0 = mk(mass * p0[r].x, mass * p0[r].y), o1 = mk(mass * p1[r].x, mass * p1[r].y);
                {   // +x: (1 - sigma_1) psi = (a, -a), a = psi0 - psi1
                    const float2 u = cscale(cmul(u0, csub(a0[r], a1[r])), 0.5f);
                    o0 = csub(o0, u);
                    o1 = cadd(o1, u);
                }
                {   // -x: (1 + sigma_1) psi = (c, c), c = psi0 + psi1
                    const float2 u = cscale(cmulc(u0m, cadd(c0[r], c1[r])), 0.5f);
                    o0 = csub(o0, u);
                    o1 = csub(o1, u);
                }
                {   // +t: (1 - sigma_2) psi = (a, -i a), a = psi0 + i psi1
                    const float2 u = cscale(cmul(u1, cadd(e0[r], ctimesi(e1[r]))), sgp);
                    o0 = csub(o0, u);
                    o1 = cadd(o1, ctimesi(u));
                }
                {   // -t: (1 + sigma_2) psi = (c, i c), c = psi0 - i psi1
                    const float2 u = cscale(cmulc(u1m, csub(f0[r], ctimesi(f1[r]))), sgm);
                    o0 = csub(o0, u);
                    o1 = csub(o1, ctimesi(u));
                }
                cfmac(dyx[r], o0, p0[r]);
                cfmac(dyx[r], o1, p1[r]);
                dyy[r] = fmaf(o0.x, o0.x, fmaf(o0.y, o0.y, fmaf(o1.x, o1.x, fmaf(o1.y, o1.y, dyy[r]))));
                w0[r] = f2_bf(o0);
                w1[r] = f2_bf(o1);
            }
            if constexpr (RPT == 4) {
                *reinterpret_cast<uint4*>(y + site * N2 + j) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4*>(y + site * N2 + N + j) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            } else {
                *reinterpret_cast<uint2*>(y + site * N2 + j) = make_uint2(w0[0], w0[1]);
                *reinterpret_cast<uint2*>(y + site * N2 + N + j) = make_uint2(w1[0], w1[1]);
            }
        }
    }
    __shared__ double2 sh[2][kRowLanes][RPT * kRhsTile + 1];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        sh[0][threadIdx.y][RPT * threadIdx.x + r] = to_d(dyx[r]);
        sh[1][threadIdx.y][RPT * threadIdx.x + r] = make_double2((double)dyy[r], 0.0);
    }
    __syncthreads();
    // RPT * 32 rhs x 2 quantities: thread t < 2 * RPT * 32 adds the 8 row lanes of
    // quantity t / (RPT * 32), rhs t % (RPT * 32) of this block
    const int t = threadIdx.y * kRhsTile + threadIdx.x;
    if (t < 2 * RPT * kRhsTile) {
        const int q = t / (RPT * kRhsTile), jj = t % (RPT * kRhsTile);
        const int jo = RPT * blockIdx.x * kRhsTile + jj;
        if (jo < N) {
            double2 acc = sh[q][0][jj];
            for (int r = 1; r < kRowLanes; ++r) acc = cadd(acc, sh[q][r][jj]);
            part[((long long)q * N + jo) * gridDim.y + blockIdx.y] = acc;
        }
    }
}

__global__ void k_pack_bf16(uint32_t* __restrict__ y, const float2* __restrict__ x, long long count) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < count) y[i] = f2_bf(x[i]);
}

// Two rhs per thread: 8-byte BF16 and 16-byte FP32 accesses; two rows per loop trip
// with all their loads issued first.  N even.
__global__ void k_mr_update_fine_bf16(float2* __restrict__ e, uint32_t* __restrict__ r, const uint32_t* __restrict__ p,
                                      const double2* __restrict__ dots, long long n, int N, bool e_is_zero) {
    const int j = 2 * (blockIdx.x * kRhsTile + threadIdx.x);
    if (j >= N) return;
    float2 a[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const double2 pr = dots[j + q];
        const double pp = dots[N + j + q].x;
        a[q] = pp > 0.0 ? make_float2((float)(pr.x / pp), (float)(pr.y / pp)) : make_float2(0.f, 0.f);
    }
    const long long S = (long long)gridDim.y * kRowLanes;
    for (long long i0 = (long long)blockIdx.y * kRowLanes + threadIdx.y; i0 < n; i0 += 2 * S) {
        uint2 rw[2], pw[2];
        float4 ev[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long i = i0 + u * S;
            const bool in = i < n;
            const long long idx = i * N + j;
            rw[u] = in ? *reinterpret_cast<const uint2*>(r + idx) : make_uint2(0u, 0u);
            pw[u] = in ? *reinterpret_cast<const uint2*>(p + idx) : make_uint2(0u, 0u);
            ev[u] = (in && !e_is_zero) ? *reinterpret_cast<const float4*>(e + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long i = i0 + u * S;
            if (i >= n) break;
            const long long idx = i * N + j;
            const float2 r0 = bf2_lo(rw[u].x), r1 = bf2_lo(rw[u].y), p0 = bf2_lo(pw[u].x), p1 = bf2_lo(pw[u].y);
            float2 e0 = make_float2(ev[u].x, ev[u].y), e1 = make_float2(ev[u].z, ev[u].w);
            cfma(e0, a[0], r0);
            cfma(e1, a[1], r1);
            *reinterpret_cast<float4*>(e + idx) = make_float4(e0.x, e0.y, e1.x, e1.y);
            *reinterpret_cast<uint2*>(r + idx) =
                make_uint2(f2_bf(csub(r0, cmul(a[0], p0))), f2_bf(csub(r1, cmul(a[1], p1))));
        }
    }
}

void launch_wilson_bf16(uint32_t* y, const uint32_t* x, const float2* U, double m0, int lx, int lt, int N,
                        double2* part, int groups, cudaStream_t s) {
    MG_REQUIRE(N % 4 == 0, MGMLMC_EINVAL, "BF16 Wilson operator: N a multiple of 4");
    if (N % 128 == 0) {
        dim3 g(N / 128, groups);
        k_wilson_bf16<4><<<g, blk(), 0, s>>>(y, x, U, (float)(m0 + 2.0), lx, lt, N, part);
    } else {
        dim3 g((N / 2 + kRhsTile - 1) / kRhsTile, groups);
        k_wilson_bf16<2><<<g, blk(), 0, s>>>(y, x, U, (float)(m0 + 2.0), lx, lt, N, part);
    }
    MG_LAUNCHED();
}

void launch_pack_bf16(uint32_t* y, const float2* x, long long count, cudaStream_t s) {
    k_pack_bf16<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(y, x, count);
    MG_LAUNCHED();
}

void launch_mr_update_fine_bf16(float2* e, uint32_t* r, const uint32_t* p, const double2* dots, long long n, int N,
                                bool e_is_zero, cudaStream_t s) {
    MG_REQUIRE(N % 2 == 0, MGMLMC_EINVAL, "BF16 MR update: N even");
    // N / 64 column blocks (two rhs per thread): row groups for one wave of as many CTAs
    // per SM as are resident
    static int per_sm = 0;
    if (per_sm == 0) {
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mr_update_fine_bf16, kRhsTile * kRowLanes, 0));
        per_sm = std::max(1, per_sm);
    }
    const int gx = (N / 2 + kRhsTile - 1) / kRhsTile;
    const long long need = (n + kRowLanes - 1) / kRowLanes;
    const int gy = (int)std::max(1LL, std::min(need, (long long)per_sm * kNumSM / gx));
    k_mr_update_fine_bf16<<<dim3(gx, gy), blk(), 0, s>>>(e, r, p, dots, n, N, e_is_zero);
    MG_LAUNCHED();
}

template <typename C>
void launch_wilson(C* y, const C* x, const C* b, const C* U, double m0, int lx, int lt, int N, int mode,
                   double2* part, int groups, cudaStream_t s) {
    using R = re_t<C>;
    dim3 g(rhs_tiles(N), groups);
    const R mass = (R)(m0 + 2.0);
    if (wilson_f2<C>(y, x, b, U, mass, lx, lt, N, mode, part, groups, s)) return;
    switch (mode) {
        case 0: k_wilson<C, 0><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
        case 1: k_wilson<C, 1><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
        default: k_wilson<C, 2><<<g, blk(), 0, s>>>(y, x, b, U, mass, lx, lt, N, part); break;
    }
    MG_LAUNCHED();
}

template <typename C, int RPT>
static void bs_dispatch(C* y, const C* x, const C* b, const C* A, int lx, int lt, int d, int N, int mode,
                        double2* part, int groups, cudaStream_t s) {
    dim3 g(rhs_tiles(N), groups);
    size_t sm = (size_t)5 * d * d * sizeof(C);
    size_t smin = 2 * kRowLanes * (kRhsTile + 1) * sizeof(double2);
    if (sm < smin) sm = smin;
    if (sm > 48 * 1024) {
        MG_CUDA(cudaFuncSetAttribute(k_block_stencil<C, RPT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        MG_CUDA(cudaFuncSetAttribute(k_block_stencil<C, RPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        MG_CUDA(cudaFuncSetAttribute(k_block_stencil<C, RPT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    }
    switch (mode) {
        case 0: k_block_stencil<C, RPT, 0><<<g, blk(), sm, s>>>(y, x, b, A, lx, lt, d, N, part); break;
        case 1: k_block_stencil<C, RPT, 1><<<g, blk(), sm, s>>>(y, x, b, A, lx, lt, d, N, part); break;
        default: k_block_stencil<C, RPT, 2><<<g, blk(), sm, s>>>(y, x, b, A, lx, lt, d, N, part); break;
    }
    MG_LAUNCHED();
}

template <int D>
static bool bsd_f2(float2* y, const float2* x, const float2* b, const float2* A, int lx, int lt, int N, int mode,
                   double2* part, int groups, cudaStream_t s) {
    if (N % 2 != 0) return false;
    if (D == 16 && N % 4 == 0 && N >= 128) {
        // four rhs per thread; T threads per half of the output rows
        const int T = std::min(64, (N / 4 + 31) / 32 * 32);
        dim3 g((N / 4 + T - 1) / T, groups);
        switch (mode) {
            case 0: k_block_stencil_f4<0><<<g, 2 * T, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
            case 1: k_block_stencil_f4<1><<<g, 2 * T, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
            default: k_block_stencil_f4<2><<<g, 2 * T, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
        }
        MG_LAUNCHED();
        return true;
    }
    const int threads = std::min(128, (N / 2 + 31) / 32 * 32);
    dim3 g((N / 2 + threads - 1) / threads, groups);
    switch (mode) {
        case 0: k_block_stencil_f2<D, 0><<<g, threads, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
        case 1: k_block_stencil_f2<D, 1><<<g, threads, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
        default: k_block_stencil_f2<D, 2><<<g, threads, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
    }
    MG_LAUNCHED();
    return true;
}
template <int D>
static bool bsd_f2(double2*, const double2*, const double2*, const double2*, int, int, int, int, double2*, int,
                   cudaStream_t) {
    return false;
}

template <typename C, int D>
static void bsd_dispatch(C* y, const C* x, const C* b, const C* A, int lx, int lt, int N, int mode, double2* part,
                         int groups, cudaStream_t s) {
    if (bsd_f2<D>(y, x, b, A, lx, lt, N, mode, part, groups, s)) return;
    const int th = cta_threads(N);
    dim3 g((N + th - 1) / th, groups);
    switch (mode) {
        case 0: k_block_stencil_d<C, D, 0><<<g, th, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
        case 1: k_block_stencil_d<C, D, 1><<<g, th, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
        default: k_block_stencil_d<C, D, 2><<<g, th, 0, s>>>(y, x, b, A, lx, lt, N, part); break;
    }
    MG_LAUNCHED();
}

// The one-rhs-per-thread kernels need wide blocks; narrow blocks (the setup solves
// run 8 rhs) take the generic 32-rhs-tile kernel.
static bool use_site_kernel(int d, int N) { return (d == 8 || d == 16) && N >= 64; }
static bool use_narrow_kernel(int d, int N) { return (d == 8 || d == 16) && N <= 16; }

int block_stencil_groups(int nsites, int d, int N) {
    if (use_narrow_kernel(d, N)) return nsites < 32 * kNumSM ? nsites : 32 * kNumSM;   // grid-stride over sites
    if (use_site_kernel(d, N)) {
        // one site per CTA up to 16 CTAs per SM: staging and compute of different
        // sites overlap across CTAs
        const int tiles = (N + 127) / 128;
        int want = 16 * kNumSM / tiles;
        if (want < 1) want = 1;
        return nsites < want ? nsites : want;
    }
    int want = 8 * kNumSM / rhs_tiles(N);
    if (want < 1) want = 1;
    return nsites < want ? nsites : want;
}

template <typename C>
void launch_block_stencil(C* y, const C* x, const C* b, const C* A, int lx, int lt, int d, int N, int mode,
                          double2* part, int groups, cudaStream_t s) {
    MG_REQUIRE(d >= 2 && d <= 64, MGMLMC_EINVAL, "block stencil: 2 <= d <= 64");
    if (use_narrow_kernel(d, N)) {
        dim3 g((N + 7) / 8, groups);
        if (d == 16) {
            if (mode == 0) k_block_stencil_narrow<C, 16, 0><<<g, dim3(8, 16), 0, s>>>(y, x, b, A, lx, lt, N, part);
            else if (mode == 1) k_block_stencil_narrow<C, 16, 1><<<g, dim3(8, 16), 0, s>>>(y, x, b, A, lx, lt, N, part);
            else k_block_stencil_narrow<C, 16, 2><<<g, dim3(8, 16), 0, s>>>(y, x, b, A, lx, lt, N, part);
        } else {
            if (mode == 0) k_block_stencil_narrow<C, 8, 0><<<g, dim3(8, 8), 0, s>>>(y, x, b, A, lx, lt, N, part);
            else if (mode == 1) k_block_stencil_narrow<C, 8, 1><<<g, dim3(8, 8), 0, s>>>(y, x, b, A, lx, lt, N, part);
            else k_block_stencil_narrow<C, 8, 2><<<g, dim3(8, 8), 0, s>>>(y, x, b, A, lx, lt, N, part);
        }
        MG_LAUNCHED();
        return;
    }
    if (use_site_kernel(d, N) && d == 16) return bsd_dispatch<C, 16>(y, x, b, A, lx, lt, N, mode, part, groups, s);
    if (use_site_kernel(d, N) && d == 8) return bsd_dispatch<C, 8>(y, x, b, A, lx, lt, N, mode, part, groups, s);
    if (d <= 8) bs_dispatch<C, 1>(y, x, b, A, lx, lt, d, N, mode, part, groups, s);
    else if (d <= 16) bs_dispatch<C, 2>(y, x, b, A, lx, lt, d, N, mode, part, groups, s);
    else if (d <= 32) bs_dispatch<C, 4>(y, x, b, A, lx, lt, d, N, mode, part, groups, s);
    else bs_dispatch<C, 8>(y, x, b, A, lx, lt, d, N, mode, part, groups, s);
}

template <typename C, int NV>
static void rp_launch(bool restrict_op, C* xc_or_x, const C* in, const C* P, int lx, int lt, int d, int ax, int at,
                      int N, bool accumulate, cudaStream_t s) {
    const int ncs = (lx / ax) * (lt / at);
    const int th = cta_threads(N);
    const int tiles = (N + th - 1) / th;
    int G = 16 * kNumSM / tiles;
    if (G > ncs) G = ncs;
    if (G < 1) G = 1;
    const size_t sm = (size_t)ax * at * d * NV * sizeof(C);
    if (d == 2) {
        if (restrict_op) k_restrict_nvd<C, NV, 2, 4><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, ax, at, N);
        else k_prolong_nvd<C, NV, 2, 4><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, ax, at, N, accumulate);
        MG_LAUNCHED();
        return;
    }
    if (d == 16) {
        if (restrict_op) k_restrict_nvd<C, NV, 16, 1><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, ax, at, N);
        else k_prolong_nvd<C, NV, 16, 1><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, ax, at, N, accumulate);
        MG_LAUNCHED();
        return;
    }
    if (restrict_op)
        k_restrict_nv<C, NV><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, d, ax, at, N);
    else
        k_prolong_nv<C, NV><<<dim3(tiles, G), th, sm, s>>>(xc_or_x, in, P, lx, lt, d, ax, at, N, accumulate);
    MG_LAUNCHED();
}

template <typename C>
static bool rp_fast(bool restrict_op, C* out, const C* in, const C* P, int lx, int lt, int d, int ax, int at,
                    int nvec, int N, bool accumulate, cudaStream_t s) {
    if ((size_t)ax * at * d * nvec * sizeof(C) > 48 * 1024) return false;
    switch (nvec) {
        case 2: rp_launch<C, 2>(restrict_op, out, in, P, lx, lt, d, ax, at, N, accumulate, s); return true;
        case 4: rp_launch<C, 4>(restrict_op, out, in, P, lx, lt, d, ax, at, N, accumulate, s); return true;
        case 8: rp_launch<C, 8>(restrict_op, out, in, P, lx, lt, d, ax, at, N, accumulate, s); return true;
        default: return false;
    }
}

template <typename C>
void launch_restrict(C* xc, const C* x, const C* P, int lx, int lt, int d, int ax, int at, int nvec, int N,
                     cudaStream_t s) {
    if (rp_fast<C>(true, xc, x, P, lx, lt, d, ax, at, nvec, N, false, s)) return;
    const int ncs = (lx / ax) * (lt / at);
    int G = row_groups((long long)ncs * kRowLanes, N, 4);
    k_restrict<C><<<dim3(rhs_tiles(N), G), blk(), 0, s>>>(xc, x, P, lx, lt, d, ax, at, nvec, N);
    MG_LAUNCHED();
}

template <typename C>
void launch_prolong(C* x, const C* xc, const C* P, int lx, int lt, int d, int ax, int at, int nvec, int N,
                    bool accumulate, cudaStream_t s) {
    if (rp_fast<C>(false, x, xc, P, lx, lt, d, ax, at, nvec, N, accumulate, s)) return;
    const long long rows = (long long)lx * lt * d;
    k_prolong<C><<<dim3(rhs_tiles(N), row_groups(rows, N)), blk(), 0, s>>>(x, xc, P, lx, lt, d, ax, at, nvec, N,
                                                                             accumulate);
    MG_LAUNCHED();
}

template <typename C>
void launch_mr_update(C* e, C* r, const C* p, const double2* dots, long long n, int N, bool e_is_zero,
                      cudaStream_t s) {
    k_mr_update<C><<<dim3(rhs_tiles(N), row_groups(n, N)), blk(), 0, s>>>(e, r, p, dots, n, N, e_is_zero);
    MG_LAUNCHED();
}

template <typename C>
void launch_gamma5(C* y, const C* x, long long nsites, int d, int N, cudaStream_t s) {
    const long long rows = nsites * d;
    k_gamma5<C><<<dim3(rhs_tiles(N), row_groups(rows, N)), blk(), 0, s>>>(y, x, rows, d, N);
    MG_LAUNCHED();
}

#define INST(C)                                                                                        \
    template void launch_wilson<C>(C*, const C*, const C*, const C*, double, int, int, int, int, double2*, \
                                   int, cudaStream_t);                                                 \
    template void launch_block_stencil<C>(C*, const C*, const C*, const C*, int, int, int, int, int,    \
                                          double2*, int, cudaStream_t);                                 \
    template void launch_restrict<C>(C*, const C*, const C*, int, int, int, int, int, int, int,         \
                                     cudaStream_t);                                                     \
    template void launch_prolong<C>(C*, const C*, const C*, int, int, int, int, int, int, int, bool,    \
                                    cudaStream_t);                                                      \
    template void launch_mr_update<C>(C*, C*, const C*, const double2*, long long, int, bool,           \
                                      cudaStream_t);                                                    \
    template void launch_gamma5<C>(C*, const C*, long long, int, int, cudaStream_t);                  \
    template void launch_block_diag_apply<C>(C*, const C*, const C*, int, int, int, bool, cudaStream_t);
INST(double2)
INST(float2)

}  // namespace mg
