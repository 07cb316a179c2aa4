// Setup kernels (hierarchy construction, Sect. 3.1 / 4.2) and the small
// per-rhs kernels of FGMRES and of the sample assembly.  All FP64.
#include "kernels.cuh"

namespace mg {

// Block-stencil form of the fine operator: A[site][dir][a][b], dir = 0 self,
// 1 +x, 2 -x, 3 +t, 4 -t.  Hop blocks -1/2 U (1 - s_mu) forward and
// -1/2 U^* (1 + s_mu) backward, with the antiperiodic time sign.
__global__ void k_materialize_wilson(double2* A, const double2* U, double m0, int lx, int lt) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= lx * lt) return;
    const int xx = site % lx, t = site / lx;
    const int sxm = (xx == 0 ? lx - 1 : xx - 1) + lx * t;
    const int stm = xx + lx * (t == 0 ? lt - 1 : t - 1);
    const double sgp = (t + 1 == lt) ? -1.0 : 1.0, sgm = (t == 0) ? -1.0 : 1.0;
    double2* a = A + (long long)site * 20;
    const double2 z = make_double2(0, 0), one = make_double2(1, 0), i1 = make_double2(0, 1),
                  mi = make_double2(0, -1), m1 = make_double2(-1, 0);
    // self
    a[0] = make_double2(m0 + 2.0, 0); a[1] = z; a[2] = z; a[3] = make_double2(m0 + 2.0, 0);
    auto put = [&](int dir, double2 u, double2 b00, double2 b01, double2 b10, double2 b11) {
        const double2 f = make_double2(-0.5 * u.x, -0.5 * u.y);
        a[dir * 4 + 0] = cmul(f, b00);
        a[dir * 4 + 1] = cmul(f, b01);
        a[dir * 4 + 2] = cmul(f, b10);
        a[dir * 4 + 3] = cmul(f, b11);
    };
    const double2 u0 = U[2 * site], u1 = U[2 * site + 1];
    const double2 u0m = U[2 * sxm], u1m = U[2 * stm + 1];
    put(1, u0, one, m1, m1, one);                                           // 1 - sigma_1
    put(2, make_double2(u0m.x, -u0m.y), one, one, one, one);                // 1 + sigma_1
    put(3, make_double2(sgp * u1.x, sgp * u1.y), one, i1, mi, one);         // 1 - sigma_2
    put(4, make_double2(sgm * u1m.x, -sgm * u1m.y), one, mi, i1, one);      // 1 + sigma_2
}

void launch_materialize_wilson(double2* A, const double2* U, double m0, int lx, int lt, cudaStream_t s) {
    k_materialize_wilson<<<(lx * lt + 127) / 128, 128, 0, s>>>(A, U, m0, lx, lt);
    MG_LAUNCHED();
}

// Galerkin coarse operator D_{l+1} = P^H D_l P in two stages.
// Stage 1: T[x][fdir][a][o'] = sum_{b in spin block s'} Af[x][fdir][a][b] P[y][b][j'],
//          y the fine neighbour of x in direction fdir, o' = (s', j').
// Stage 2: Ac[S][dir][o][o'] = sum over fine sites x of aggregate S and fine hops x -> y
//          that leave S through side dir (dir 0: stay inside) of
//          sum_{a in spin block s} conj(P[x][a][j]) T[x][fdir][a][o'],  o = (s, j).
__device__ __forceinline__ int fine_nbr(int xx, int t, int fdir, int lx, int lt) {
    switch (fdir) {
        case 1: return (xx + 1 == lx ? 0 : xx + 1) + lx * t;
        case 2: return (xx == 0 ? lx - 1 : xx - 1) + lx * t;
        case 3: return xx + lx * (t + 1 == lt ? 0 : t + 1);
        case 4: return xx + lx * (t == 0 ? lt - 1 : t - 1);
        default: return xx + lx * t;
    }
}

__global__ void k_galerkin_t(double2* T, const double2* Af, const double2* P, int lx, int lt, int d, int nvec) {
    const int dc = 2 * nvec, hd = d / 2;
    const long long total = (long long)lx * lt * 5 * d * dc;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int op = (int)(e % dc), a = (int)((e / dc) % d), fdir = (int)((e / ((long long)dc * d)) % 5);
    const int site = (int)(e / (5LL * d * dc));
    const int xx = site % lx, t = site / lx;
    const int ysite = fine_nbr(xx, t, fdir, lx, lt);
    const int sp = op / nvec, jp = op % nvec;
    const double2* Ab = Af + ((long long)site * 5 + fdir) * d * d + (long long)a * d;
    double2 acc = make_double2(0, 0);
    for (int b = sp * hd; b < (sp + 1) * hd; ++b) cfma(acc, Ab[b], P[((long long)ysite * d + b) * nvec + jp]);
    T[e] = acc;
}

__global__ void k_galerkin_c(double2* Ac, const double2* T, const double2* P, int lx, int lt, int d, int ax, int at,
                             int nvec) {
    const int dc = 2 * nvec, hd = d / 2;
    const int cx = lx / ax, ct = lt / at;
    const long long total = (long long)cx * ct * 5 * dc * dc;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int op = (int)(e % dc), o = (int)((e / dc) % dc), dir = (int)((e / (dc * dc)) % 5);
    const int S = (int)(e / (5LL * dc * dc));
    const int X = S % cx, TT = S / cx;
    const int s = o / nvec, jj = o % nvec;
    double2 acc = make_double2(0, 0);
    for (int it = 0; it < at; ++it)
        for (int ix = 0; ix < ax; ++ix) {
            const int site = (X * ax + ix) + lx * (TT * at + it);
            for (int fdir = 0; fdir < 5; ++fdir) {
                int cdir;
                switch (fdir) {
                    case 1: cdir = (ix == ax - 1) ? 1 : 0; break;
                    case 2: cdir = (ix == 0) ? 2 : 0; break;
                    case 3: cdir = (it == at - 1) ? 3 : 0; break;
                    case 4: cdir = (it == 0) ? 4 : 0; break;
                    default: cdir = 0;
                }
                if (cdir != dir) continue;
                const double2* Tr = T + (((long long)site * 5 + fdir) * d) * dc + op;
                for (int a = s * hd; a < (s + 1) * hd; ++a)
                    cfmac(acc, P[((long long)site * d + a) * nvec + jj], Tr[(long long)a * dc]);
            }
        }
    Ac[e] = acc;
}

size_t galerkin_scratch_count(int lx, int lt, int d, int nvec) { return (size_t)lx * lt * 5 * d * 2 * nvec; }

void launch_galerkin(double2* Ac, const double2* Af, const double2* P, int lx, int lt, int d, int ax, int at,
                     int nvec, double2* T, cudaStream_t s) {
    const long long t1 = (long long)lx * lt * 5 * d * 2 * nvec;
    k_galerkin_t<<<(unsigned)((t1 + 127) / 128), 128, 0, s>>>(T, Af, P, lx, lt, d, nvec);
    MG_LAUNCHED();
    const long long total = (long long)(lx / ax) * (lt / at) * 5 * (2 * nvec) * (2 * nvec);
    k_galerkin_c<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(Ac, T, P, lx, lt, d, ax, at, nvec);
    MG_LAUNCHED();
}

// P[site][a][j]: test vector j restricted to (aggregate, spin block of a),
// orthonormalised by modified Gram-Schmidt in j order.  One thread per
// (aggregate, spin block); rows of the block ordered (site in aggregate, a).
__global__ void k_build_prolongator(double2* P, const double2* tv, int lx, int lt, int d, int ax, int at, int nvec,
                                    int* status) {
    const int cx = lx / ax, ct = lt / at, hd = d / 2;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= cx * ct * 2) return;
    const int S = id / 2, s = id % 2;
    const int X = S % cx, T = S / cx;
    const long long n = (long long)lx * lt * d;
    const int m = ax * at * hd;
    auto row_index = [&](int r) -> long long {   // fine dof of block row r
        const int sl = r / hd, a = s * hd + r % hd;
        const int site = (X * ax + sl % ax) + lx * (T * at + sl / ax);
        return (long long)site * d + a;
    };
    for (int r = 0; r < m; ++r) {
        const long long f = row_index(r);
        for (int j = 0; j < nvec; ++j) P[f * nvec + j] = tv[(long long)j * n + f];
    }
    for (int j = 0; j < nvec; ++j) {
        for (int i = 0; i < j; ++i) {
            double2 h = make_double2(0, 0);
            for (int r = 0; r < m; ++r) {
                const long long f = row_index(r);
                cfmac(h, P[f * nvec + i], P[f * nvec + j]);
            }
            for (int r = 0; r < m; ++r) {
                const long long f = row_index(r);
                P[f * nvec + j] = csub(P[f * nvec + j], cmul(h, P[f * nvec + i]));
            }
        }
        double nr = 0;
        for (int r = 0; r < m; ++r) {
            const double2 v = P[row_index(r) * nvec + j];
            nr += v.x * v.x + v.y * v.y;
        }
        nr = sqrt(nr);
        if (!(nr > 0.0)) {
            atomicExch(status, 1);
            nr = 1.0;
        }
        for (int r = 0; r < m; ++r) {
            const long long f = row_index(r);
            P[f * nvec + j] = cscale(P[f * nvec + j], 1.0 / nr);
        }
    }
}

void launch_build_prolongator(double2* P, const double2* tv, int lx, int lt, int d, int ax, int at, int nvec,
                              int* status, cudaStream_t s) {
    const int nb = (lx / ax) * (lt / at) * 2;
    k_build_prolongator<<<(nb + 127) / 128, 128, 0, s>>>(P, tv, lx, lt, d, ax, at, nvec, status);
    MG_LAUNCHED();
}

// ------------------------------------------------------------- FGMRES bookkeeping
// Per rhs r: H[r][i][j] (i <= j) the rotated upper-triangular Hessenberg,
// cs[r][j] real cosines, sn[r][j] complex sines, g[r][0..m] the rotated rhs.
__global__ void k_init_g(double2* g, const double* beta, int m, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    for (int i = 0; i <= m; ++i) g[(long long)r * (m + 1) + i] = make_double2(i == 0 ? beta[r] : 0.0, 0.0);
}

__global__ void k_arnoldi_column(double2* H, double* cs, double2* sn, double2* g, double* resid, const double2* h,
                                 const double* hnorm, int j, int m, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double2* Hr = H + (long long)r * (m + 1) * m;
    double* c_r = cs + (long long)r * m;
    double2* s_r = sn + (long long)r * m;
    double2* g_r = g + (long long)r * (m + 1);
    double2 col[65];
    for (int i = 0; i <= j; ++i) col[i] = h[(long long)i * N + r];
    col[j + 1] = make_double2(hnorm[r], 0.0);
    // previous rotations: (a, b) <- (c a + s b, -conj(s) a + c b)
    for (int i = 0; i < j; ++i) {
        const double c = c_r[i];
        const double2 s = s_r[i];
        const double2 a = col[i], b = col[i + 1];
        const double2 sb = cmul(s, b);
        const double2 sca = cmulc(s, a);
        col[i] = make_double2(c * a.x + sb.x, c * a.y + sb.y);
        col[i + 1] = make_double2(c * b.x - sca.x, c * b.y - sca.y);
    }
    // new rotation zeroing col[j+1]
    const double2 a = col[j], b = col[j + 1];
    const double na = sqrt(a.x * a.x + a.y * a.y), nb = sqrt(b.x * b.x + b.y * b.y);
    const double rho = sqrt(na * na + nb * nb);
    double c;
    double2 s, rr;
    if (rho == 0.0) {
        c = 1.0; s = make_double2(0, 0); rr = make_double2(0, 0);
    } else if (na == 0.0) {
        c = 0.0; s = make_double2(b.x / nb, -b.y / nb); rr = make_double2(nb, 0);   // s = conj(b)/|b|
    } else {
        const double2 ph = make_double2(a.x / na, a.y / na);
        c = na / rho;
        s = cmul(ph, make_double2(b.x / rho, -b.y / rho));      // (a/|a|) conj(b) / rho
        rr = make_double2(ph.x * rho, ph.y * rho);
    }
    c_r[j] = c;
    s_r[j] = s;
    col[j] = rr;
    for (int i = 0; i <= j; ++i) Hr[(long long)i * m + j] = col[i];
    const double2 gj = g_r[j];
    const double2 sg = cmulc(s, gj);
    g_r[j] = make_double2(c * gj.x, c * gj.y);
    g_r[j + 1] = make_double2(-sg.x, -sg.y);
    resid[r] = sqrt(sg.x * sg.x + sg.y * sg.y);
}

__global__ void k_back_substitute(double2* y, const double2* H, const double2* g, int j, int m, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double2* Hr = H + (long long)r * (m + 1) * m;
    const double2* g_r = g + (long long)r * (m + 1);
    double2 yv[64];
    for (int i = j; i >= 0; --i) {
        double2 acc = g_r[i];
        for (int l = i + 1; l <= j; ++l) acc = csub(acc, cmul(Hr[(long long)i * m + l], yv[l]));
        const double2 hd = Hr[(long long)i * m + i];
        const double den = hd.x * hd.x + hd.y * hd.y;
        yv[i] = (den > 0.0) ? make_double2((acc.x * hd.x + acc.y * hd.y) / den, (acc.y * hd.x - acc.x * hd.y) / den)
                            : make_double2(0, 0);
    }
    for (int i = 0; i <= j; ++i) y[(long long)i * N + r] = yv[i];
}

__global__ void k_max_ratio(double* out, const double* resid, const double* bnorm, int N) {
    __shared__ double sh[256];
    double m = 0;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        const double b = bnorm[r];
        double v = (b > 0.0) ? resid[r] / b : 0.0;
        if (v != v) v = __longlong_as_double(0x7ff8000000000000ll);   // keep NaN visible
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

void launch_init_g(double2* g, const double* beta, int m, int N, cudaStream_t s) {
    k_init_g<<<(N + 127) / 128, 128, 0, s>>>(g, beta, m, N);
    MG_LAUNCHED();
}
void launch_arnoldi_column(double2* H, double* cs, double2* sn, double2* g, double* resid, const double2* h,
                           const double* hnorm, int j, int m, int N, cudaStream_t s) {
    MG_REQUIRE(m <= 64, MGMLMC_EINVAL, "FGMRES restart length above 64");
    k_arnoldi_column<<<(N + 63) / 64, 64, 0, s>>>(H, cs, sn, g, resid, h, hnorm, j, m, N);
    MG_LAUNCHED();
}
void launch_back_substitute(double2* y, const double2* H, const double2* g, int j, int m, int N, cudaStream_t s) {
    k_back_substitute<<<(N + 63) / 64, 64, 0, s>>>(y, H, g, j, m, N);
    MG_LAUNCHED();
}
void launch_max_ratio(double* out, const double* resid, const double* bnorm, int N, cudaStream_t s) {
    k_max_ratio<<<1, 256, 0, s>>>(out, resid, bnorm, N);
    MG_LAUNCHED();
}

// ------------------------------------------------------------- sample assembly
// s[j] -= sum_i a_i conj(B[i][j]) A[i][j]   (deflated part of the coarsest term)
__global__ void k_deflation_correction(double2* s, const double2* A, const double2* B, const double* a, int k, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double2 t = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
        const double2 v = cmulc(B[(long long)i * N + j], A[(long long)i * N + j]);
        t.x += a[i] * v.x;
        t.y += a[i] * v.y;
    }
    s[j] = csub(s[j], t);
}

void launch_deflation_correction(double2* s, const double2* A, const double2* B, const double* a, int k, int N,
                                 cudaStream_t st) {
    k_deflation_correction<<<(N + 127) / 128, 128, 0, st>>>(s, A, B, a, k, N);
    MG_LAUNCHED();
}

// acc[0..2] += (sum re, sum im, sum |s|^2) over N samples, fixed summation order.
__global__ void k_sample_stats(double* acc, const double2* smp, int N) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0, b = 0, c = 0;
    for (int j = 0; j < N; ++j) {
        a += smp[j].x;
        b += smp[j].y;
        c += smp[j].x * smp[j].x + smp[j].y * smp[j].y;
    }
    acc[0] += a;
    acc[1] += b;
    acc[2] += c;
}

void launch_sample_stats(double* acc, const double2* smp, int N, cudaStream_t s) {
    k_sample_stats<<<1, 32, 0, s>>>(acc, smp, N);
    MG_LAUNCHED();
}

}  // namespace mg

namespace mg {
// One thread per row (site, a): Dd[row][nbr(site,dir) d + b] += A[site][dir][a][b]
// (Dd zeroed by the launcher).
__global__ void k_dense_from_blocks(double2* Dd, const double2* A, int lx, int lt, int d) {
    const long long n = (long long)lx * lt * d;
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int site = (int)(row / d), a = (int)(row % d);
    const int xx = site % lx, t = site / lx;
    for (int dir = 0; dir < 5; ++dir) {
        int nb;
        switch (dir) {
            case 1: nb = (xx + 1 == lx ? 0 : xx + 1) + lx * t; break;
            case 2: nb = (xx == 0 ? lx - 1 : xx - 1) + lx * t; break;
            case 3: nb = xx + lx * (t + 1 == lt ? 0 : t + 1); break;
            case 4: nb = xx + lx * (t == 0 ? lt - 1 : t - 1); break;
            default: nb = site;
        }
        const double2* Ab = A + ((long long)site * 5 + dir) * d * d + (long long)a * d;
        for (int b = 0; b < d; ++b) {
            double2& o = Dd[row * n + (long long)nb * d + b];
            o = cadd(o, Ab[b]);
        }
    }
}
void launch_dense_from_blocks(double2* Dd, const double2* A, int lx, int lt, int d, cudaStream_t s) {
    const long long n = (long long)lx * lt * d;
    MG_CUDA(cudaMemsetAsync(Dd, 0, sizeof(double2) * n * n, s));
    k_dense_from_blocks<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Dd, A, lx, lt, d);
    MG_LAUNCHED();
}
}  // namespace mg

namespace mg {
// Inverse of every site's self block A[s][0] (d x d complex, FP64), Gauss-Jordan
// with partial pivoting in global memory, one thread per site.  status = 1 on a
// zero pivot.
__global__ void k_block_diag_inverse(double2* Minv, double2* work, const double2* A, int nsites, int d,
                                     int* status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsites) return;
    double2* M = work + (long long)s * d * d;       // copy of the block, destroyed
    double2* I = Minv + (long long)s * d * d;
    const double2* B = A + (long long)s * 5 * d * d;  // dir 0
    for (int e = 0; e < d * d; ++e) {
        M[e] = B[e];
        I[e] = make_double2((e / d) == (e % d) ? 1.0 : 0.0, 0.0);
    }
    for (int k = 0; k < d; ++k) {
        int p = k;
        double best = -1.0;
        for (int i = k; i < d; ++i) {
            const double m = M[i * d + k].x * M[i * d + k].x + M[i * d + k].y * M[i * d + k].y;
            if (m > best) { best = m; p = i; }
        }
        if (!(best > 0.0)) { atomicExch(status, 1); return; }
        if (p != k)
            for (int c = 0; c < d; ++c) {
                double2 t = M[k * d + c]; M[k * d + c] = M[p * d + c]; M[p * d + c] = t;
                t = I[k * d + c]; I[k * d + c] = I[p * d + c]; I[p * d + c] = t;
            }
        const double2 pv = M[k * d + k];
        const double den = pv.x * pv.x + pv.y * pv.y;
        const double2 inv = make_double2(pv.x / den, -pv.y / den);
        for (int c = 0; c < d; ++c) {
            M[k * d + c] = cmul(M[k * d + c], inv);
            I[k * d + c] = cmul(I[k * d + c], inv);
        }
        for (int i = 0; i < d; ++i) {
            if (i == k) continue;
            const double2 f = M[i * d + k];
            for (int c = 0; c < d; ++c) {
                M[i * d + c] = csub(M[i * d + c], cmul(f, M[k * d + c]));
                I[i * d + c] = csub(I[i * d + c], cmul(f, I[k * d + c]));
            }
        }
    }
}

// Ahat[s][dir] = A[s][dir] Minv[nbr(s, dir)]: the block stencil of D M^{-1}.
__global__ void k_precondition_blocks(double2* Ahat, const double2* A, const double2* Minv, int lx, int lt, int d) {
    const long long total = (long long)lx * lt * 5 * d * d;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int cb = (int)(e % d), c = (int)((e / d) % d), dir = (int)((e / ((long long)d * d)) % 5);
    const int site = (int)(e / (5LL * d * d));
    const int xx = site % lx, t = site / lx;
    int nb;
    switch (dir) {
        case 1: nb = (xx + 1 == lx ? 0 : xx + 1) + lx * t; break;
        case 2: nb = (xx == 0 ? lx - 1 : xx - 1) + lx * t; break;
        case 3: nb = xx + lx * (t + 1 == lt ? 0 : t + 1); break;
        case 4: nb = xx + lx * (t == 0 ? lt - 1 : t - 1); break;
        default: nb = site;
    }
    const double2* Ar = A + (((long long)site * 5 + dir) * d + c) * d;
    const double2* Mn = Minv + (long long)nb * d * d;
    double2 acc = make_double2(0, 0);
    for (int b = 0; b < d; ++b) cfma(acc, Ar[b], Mn[b * d + cb]);
    Ahat[e] = acc;
}

void launch_block_diag_inverse(double2* Minv, double2* work, const double2* A, int nsites, int d, int* status,
                               cudaStream_t s) {
    k_block_diag_inverse<<<(nsites + 63) / 64, 64, 0, s>>>(Minv, work, A, nsites, d, status);
    MG_LAUNCHED();
}
void launch_precondition_blocks(double2* Ahat, const double2* A, const double2* Minv, int lx, int lt, int d,
                                cudaStream_t s) {
    const long long total = (long long)lx * lt * 5 * d * d;
    k_precondition_blocks<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(Ahat, A, Minv, lx, lt, d);
    MG_LAUNCHED();
}
}  // namespace mg
