// Tensor-core (tcgen05) BF16 GEMM for the coarsest-level solve of the mixed
// precision multigrid: y = D_L^{-1} r for a block of right-hand sides, with the
// stored inverse rounded to BF16 and FP32 accumulation in tensor memory.
//
// Complex product in real arithmetic: with A = D_L^{-1} = Ar + i Ai and the
// block X viewed as reals Xr[n][2N] (columns re/im of each rhs),
//     Y = [Ar | Ai] * [Xr ; Xr J],   (Xr J)[i][2j] = -Im X_ij, (Xr J)[i][2j+1] = Re X_ij,
// a real GEMM with M = n, K = 2n, N' = 2N.  A' = [Ar | Ai] is built once at
// setup; B' is packed per call, K-major (transposed), so both operands are
// K-major BF16 in the canonical no-swizzle shared-memory layout.
//
// Kernel: one CTA (4 warps) per 128 x NT output tile and K split.  Thread 0
// streams 128x64 (A) and NTx64 (B) stages with 1-D bulk copies into a ring of
// shared-memory stages (full/empty mbarrier pairs); thread 32 issues 4
// tcgen05.mma (K = 16 each) per stage and commits the stage back; the
// accumulator lives in TMEM (NT columns) and is read back with tcgen05.ld.
// Split-K partials are added in a fixed order by a second kernel.  Every
// mbarrier wait is bounded: on timeout the CTA records an error flag, frees TMEM
// and returns.
#include "kernels.cuh"

namespace mg {

namespace tc {

constexpr int BM = 128;         // rows per tile (TMEM lanes)
constexpr int BK = 64;          // K per stage (4 MMAs of K = 16)
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x
// 16 bytes; lbo = byte distance between core matrices adjacent along K, sbo =
// byte distance between 8-row groups; bits 46-48 hold the fixed version 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Canonical K-major layout of a rows x 64 BF16 tile: 8-row groups of 1024 B
// (eight 128-byte core matrices along K), rows 16 B apart inside a core matrix.
// Operands are stored pre-tiled in global memory: a 128 x 64 tile of A' (16 KB) or
// an NT x 64 tile of B' (NT * 128 B) is contiguous and already in the canonical
// layout above, so one 1-D bulk copy (cp.async.bulk, completing on an mbarrier)
// moves a whole stage operand.
__host__ __device__ __forceinline__ size_t tiled_off(int row, int k, int rows_per_tile, int ktiles) {
    const int tile_r = row / rows_per_tile, r = row % rows_per_tile;
    const int tile_k = k / 64, kk = k % 64;
    return ((size_t)tile_r * ktiles + tile_k) * (size_t)rows_per_tile * 128 +
           (size_t)((r >> 3) * 1024 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Warp-specialised main loop: thread 0 (warp 0) streams stages with bulk copies,
// thread 32 (warp 1) issues tcgen05.mma and commits each stage back to its empty
// barrier and the last one to `done`; then all four warps read TMEM (one lane
// quarter each) and store their rows.  K range: split blockIdx.z of gridDim.z.
template <int NT, int ST>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm_bf16(float* __restrict__ Y, const __nv_bfloat16* __restrict__ At, const __nv_bfloat16* __restrict__ Bt,
                   int M, int K, int Ncols, int* __restrict__ err) {
    constexpr int A_BYTES = BM * BK * 2;
    constexpr int B_BYTES = NT * BK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[ST], empty[ST], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.y, nt = blockIdx.x;
    const int ktiles = K / BK;
    const int per = (ktiles + gridDim.z - 1) / gridDim.z;
    const int k_begin = blockIdx.z * per;
    const int k_end = min(ktiles, k_begin + per);
    const int nk = max(0, k_end - k_begin);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const uint8_t* a_base = reinterpret_cast<const uint8_t*>(At) + (size_t)mt * ktiles * A_BYTES;
    const uint8_t* b_base = reinterpret_cast<const uint8_t*>(Bt) + (size_t)nt * ktiles * B_BYTES;

    if (tid == 0) {
        // producer
        for (int i = 0; i < nk; ++i) {
            const int s = i % ST, u = i / ST;
            if (u > 0 && !mbar_wait(&empty[s], (unsigned)((u - 1) & 1))) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (abort_flag) break;
            uint8_t* sa = smem + s * STAGE_BYTES;
            const int kt = k_begin + i;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            bulk_g2s(sa, a_base + (size_t)kt * A_BYTES, A_BYTES, &full[s]);
            bulk_g2s(sa + A_BYTES, b_base + (size_t)kt * B_BYTES, B_BYTES, &full[s]);
        }
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t IDESC = instr_desc(BM, NT);
        for (int i = 0; i < nk; ++i) {
            const int s = i % ST, u = i / ST;
            if (!mbar_wait(&full[s], (unsigned)(u & 1))) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (abort_flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t ad = smem_desc(sa + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(sb + ks * 256, 128, 1024);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[s])));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done)));
    }
    __syncwarp();
    // epilogue: wait for the last MMA, then every warp reads its 32 TMEM lanes
    bool ok = mbar_wait(&done, 0u);
    __syncthreads();
    if (!ok || abort_flag) {
        if (tid == 0) atomicExch(err, 1);
    } else if (nk == 0) {
        // empty K slice: its partial is zero
        const int row = mt * BM + warp * 32 + lane;
        float* out = Y + (size_t)blockIdx.z * (size_t)M * Ncols;
        if (row < M)
            for (int c = 0; c < NT; ++c) out[(size_t)row * Ncols + nt * NT + c] = 0.f;
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = mt * BM + warp * 32 + lane;
        float* out = Y + (size_t)blockIdx.z * (size_t)M * Ncols;
#pragma unroll 1
        for (int c = 0; c < NT; c += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float4* dst = reinterpret_cast<float4*>(out + (size_t)row * Ncols + nt * NT + c);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

// A' = [Re A | Im A] (n x 2n) written pre-tiled (128-row tiles).
__global__ void k_embed_a(__nv_bfloat16* __restrict__ E, const float2* __restrict__ A, int n) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e / n), k = (int)(e % n);
    const float2 v = A[e];
    const int kt = 2 * n / BK;
    E[tiled_off(i, k, BM, kt) / 2] = __float2bfloat16(v.x);
    E[tiled_off(i, n + k, BM, kt) / 2] = __float2bfloat16(v.y);
}

// B' (K-major, pre-tiled in NT-row tiles), col = 2j + p; zero for j >= N.
//   k <  n: p = 0 -> Re X[k][j],       p = 1 -> Im X[k][j]
//   k >= n: p = 0 -> -Im X[k-n][j],    p = 1 -> Re X[k-n][j]
__global__ void k_pack_bt(__nv_bfloat16* __restrict__ Bt, const float2* __restrict__ X, int n, int N, int Ncols,
                          int NT) {
    __shared__ float2 t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;   // rows of X, rhs
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && j < N) ? X[(size_t)i * N + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int kt = 2 * n / BK;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int i = i0 + threadIdx.x;
        if (i >= n || 2 * j + 1 >= Ncols) continue;
        const float2 v = (j < N) ? t[threadIdx.x][r] : make_float2(0.f, 0.f);
        Bt[tiled_off(2 * j, i, NT, kt) / 2] = __float2bfloat16(v.x);
        Bt[tiled_off(2 * j, n + i, NT, kt) / 2] = __float2bfloat16(-v.y);
        Bt[tiled_off(2 * j + 1, i, NT, kt) / 2] = __float2bfloat16(v.y);
        Bt[tiled_off(2 * j + 1, n + i, NT, kt) / 2] = __float2bfloat16(v.x);
    }
}

// Y[i][j] = sum over splits of Yp[z][i][c] (fixed order), complex output unpadded.
__global__ void k_reduce_y(float2* __restrict__ Y, const float* __restrict__ Yp, int n, int N, int Ncols, int splits) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * N) return;
    const long long i = e / N, j = e % N;
    float re = 0.f, im = 0.f;
    for (int z = 0; z < splits; ++z) {
        const float* p = Yp + (size_t)z * n * Ncols + i * Ncols + 2 * j;
        re += p[0];
        im += p[1];
    }
    Y[e] = make_float2(re, im);
}

}  // namespace tc

void launch_embed_bf16(__nv_bfloat16* E, const float2* A, int n, cudaStream_t s) {
    const long long tot = (long long)n * n;
    tc::k_embed_a<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(E, A, n);
    MG_LAUNCHED();
}

bool tc_coarse_supported(int n) { return n >= 128 && n % 128 == 0; }

static int pick_nt(int N) { return (2 * N >= 256) ? 256 : (2 * N > 64 ? 128 : 64); }

// Split-K factor: one CTA per SM (the stages fill ~192 KB of shared memory), so
// split the K range until the tiles cover the 152 SMs once.
static int pick_splits(int n, int Ncols, int NT) {
    const int tiles = (Ncols / NT) * (n / tc::BM);
    const int ktiles = 2 * n / tc::BK;
    int S = kNumSM / (tiles > 0 ? tiles : 1);
    if (S < 1) S = 1;
    if (S > ktiles) S = ktiles;
    if (S > 8) S = 8;
    const int per = (ktiles + S - 1) / S;     // every slice non-empty
    return (ktiles + per - 1) / per;
}

size_t coarse_inverse_bf16_scratch(int n, int N) {
    const int NT = pick_nt(N);
    const size_t ncols = (size_t)((2 * N + NT - 1) / NT) * NT;
    const int S = pick_splits(n, (int)ncols, NT);
    return ncols * 2 * n * sizeof(__nv_bfloat16) + (size_t)S * n * ncols * sizeof(float) + 256;
}

template <int NT, int ST>
static void launch_tc_st(float* Y, const __nv_bfloat16* A, const __nv_bfloat16* Bt, int M, int K, int Ncols,
                         int splits, int* err, cudaStream_t s) {
    constexpr int smem = ST * (tc::BM * tc::BK * 2 + NT * tc::BK * 2);
    MG_CUDA(cudaFuncSetAttribute(tc::k_tc_gemm_bf16<NT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 g(Ncols / NT, M / tc::BM, splits);
    tc::k_tc_gemm_bf16<NT, ST><<<g, 128, smem, s>>>(Y, A, Bt, M, K, Ncols, err);
    MG_LAUNCHED();
}

// Y (or split partials [splits][M][Ncols]) = A' B' for pre-tiled operands.
static void launch_tc(int NT, float* Y, const __nv_bfloat16* A, const __nv_bfloat16* Bt, int M, int K, int Ncols,
                      int splits, int* err, cudaStream_t s) {
    if (NT == 256) launch_tc_st<256, 4>(Y, A, Bt, M, K, Ncols, splits, err, s);
    else if (NT == 128) launch_tc_st<128, 6>(Y, A, Bt, M, K, Ncols, splits, err, s);
    else launch_tc_st<64, 8>(Y, A, Bt, M, K, Ncols, splits, err, s);
}

static void launch_pack(__nv_bfloat16* Bt, const float2* X, int n, int N, int Ncols, int NT, cudaStream_t s) {
    dim3 g((Ncols / 2 + 31) / 32, (n + 31) / 32);
    tc::k_pack_bt<<<g, dim3(32, 8), 0, s>>>(Bt, X, n, N, Ncols, NT);
    MG_LAUNCHED();
}

void launch_coarse_inverse_bf16(float2* Y, const float2* X, const __nv_bfloat16* E, int n, int N, void* scratch,
                                int* err, cudaStream_t s) {
    MG_REQUIRE(tc_coarse_supported(n), MGMLMC_EINVAL, "tensor-core coarsest solve needs n % 128 == 0");
    const int NT = pick_nt(N);
    const int Ncols = ((2 * N + NT - 1) / NT) * NT;
    const int S = pick_splits(n, Ncols, NT);
    __nv_bfloat16* Bt = reinterpret_cast<__nv_bfloat16*>(scratch);
    float* Yp = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(scratch) + (size_t)Ncols * 2 * n * 2);
    launch_pack(Bt, X, n, N, Ncols, NT, s);
    const bool direct = (Ncols == 2 * N && S == 1);
    launch_tc(NT, direct ? reinterpret_cast<float*>(Y) : Yp, E, Bt, n, 2 * n, Ncols, S, err, s);
    if (!direct) {
        const long long tot = (long long)n * N;
        tc::k_reduce_y<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Y, Yp, n, N, Ncols, S);
        MG_LAUNCHED();
    }
}


namespace tc {
// ------------------------------------------------------------------------------
// Deflation projections on the tensor cores (mg_precision 16).  For the traced
// operator's deflated part L diag(a) R^H (Sect. 2, Eq. splitting_defl_trace) a
// block of real probe vectors X [n][N] needs A = R^H X and B = L^H X.  With X real,
//     Re A = (Re R)^T X,  Im A = -(Im R)^T X  (and the same for B with L),
// so the four are one real GEMM  Y = W^T X  with W^T = [Re R | -Im R | Re L | -Im L]^T
// (M = 4k rows, padded to 128; K = n; N = the rhs), BF16 operands, FP32
// accumulation in TMEM.  W^T is rounded and pre-tiled once per deflation (the
// K-major layout of the GEMM above); X (+-1, exact in BF16) is packed per block.
// The samples then subtract sum_m a_m conj(B_m) A_m in FP64, and the estimate adds
// the deflated trace from the same rounded factors (k_defl_tau), which keeps it
// unbiased.

// W^T pre-tiled in 128-row tiles: row m < k: Re R[:, m]; k + m: -Im R; 2k + m: Re L;
// 3k + m: -Im L; rows >= 4k zero.  Rounding: FP64 -> FP32 -> BF16, both to nearest.
__global__ void k_embed_defl(__nv_bfloat16* __restrict__ W, const double2* __restrict__ R,
                             const double2* __restrict__ L, int n, int k, int Mpad) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * Mpad) return;
    const int i = (int)(e / Mpad), m = (int)(e % Mpad);
    float v = 0.f;
    if (m < 4 * k) {
        const int q = m / k, c = m % k;
        const double2 z = (q < 2 ? R : L)[(long long)i * k + c];
        v = (q & 1) ? -(float)z.y : (float)z.x;
    }
    W[tiled_off(m, i, BM, n / BK) / 2] = __float2bfloat16(v);
}

// X^T pre-tiled in NT-row tiles (row j = rhs, K = n): the real part of X, zero for j >= N.
__global__ void k_pack_x_real(__nv_bfloat16* __restrict__ Bt, const double2* __restrict__ X, int n, int N, int Ncols,
                              int NT) {
    __shared__ float t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && j < N) ? (float)X[(size_t)i * N + j].x : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < n && j < Ncols) Bt[tiled_off(j, i, NT, n / BK) / 2] = __float2bfloat16(t[threadIdx.x][r]);
    }
}

__device__ __forceinline__ double2 bf16_round(double2 z) {
    return make_double2((double)__bfloat162float(__float2bfloat16((float)z.x)),
                        (double)__bfloat162float(__float2bfloat16((float)z.y)));
}

// t[m] = R~_m^H L~_m in FP64 over the BF16-rounded factors (one CTA per m, fixed tree).
__global__ void k_defl_tau(double2* __restrict__ t, const double2* __restrict__ R, const double2* __restrict__ L,
                           int n, int k) {
    __shared__ double sr[256], si[256];
    const int m = blockIdx.x;
    double re = 0, im = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 r = bf16_round(R[(long long)i * k + m]), l = bf16_round(L[(long long)i * k + m]);
        re += r.x * l.x + r.y * l.y;
        im += r.x * l.y - r.y * l.x;
    }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            sr[threadIdx.x] += sr[threadIdx.x + st];
            si[threadIdx.x] += si[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) t[m] = make_double2(sr[0], si[0]);
}

// s[j] -= sum_m a_m conj(B_mj) A_mj from the split partials Yp[z][Mpad][Ncols] (one
// CTA per rhs, fixed order over splits and a fixed reduction tree over m).
__global__ void k_defl_correction_tc(double2* __restrict__ smp, const float* __restrict__ Yp,
                                     const double* __restrict__ a, int k, int Mpad, int Ncols, int splits) {
    __shared__ double sr[256], si[256];
    const int j = blockIdx.x;
    const size_t slab = (size_t)Mpad * Ncols;
    double re = 0, im = 0;
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double ar = 0, ai = 0, br = 0, bi = 0;
        for (int z = 0; z < splits; ++z) {
            const float* Y = Yp + z * slab;
            ar += Y[(size_t)m * Ncols + j];
            ai += Y[(size_t)(k + m) * Ncols + j];
            br += Y[(size_t)(2 * k + m) * Ncols + j];
            bi += Y[(size_t)(3 * k + m) * Ncols + j];
        }
        const double w = a[m];
        re += w * (br * ar + bi * ai);     // conj(B) A
        im += w * (br * ai - bi * ar);
    }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            sr[threadIdx.x] += sr[threadIdx.x + st];
            si[threadIdx.x] += si[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) smp[j] = make_double2(smp[j].x - sr[0], smp[j].y - si[0]);
}
}  // namespace tc

bool tc_deflation_supported(long long n, int k) { return n >= 64 && n % 64 == 0 && n <= 65535LL * 32 && k >= 1; }
int tc_deflation_rows(int k) { return (4 * k + tc::BM - 1) / tc::BM * tc::BM; }

void launch_embed_deflation_bf16(__nv_bfloat16* W, const double2* R, const double2* L, long long n, int k,
                                 cudaStream_t s) {
    MG_REQUIRE(tc_deflation_supported(n, k), MGMLMC_EINVAL, "tensor-core deflation needs n % 64 == 0");
    const int Mpad = tc_deflation_rows(k);
    const long long tot = n * Mpad;
    tc::k_embed_defl<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W, R, L, (int)n, k, Mpad);
    MG_LAUNCHED();
}

void launch_deflation_tau_bf16(double2* t, const double2* R, const double2* L, long long n, int k, cudaStream_t s) {
    tc::k_defl_tau<<<k, 256, 0, s>>>(t, R, L, (int)n, k);
    MG_LAUNCHED();
}

static int pick_nt_real(int N) { return N >= 256 ? 256 : (N > 64 ? 128 : 64); }

static int defl_splits(long long n, int Mpad, int Ncols, int NT) {
    const int tiles = (Ncols / NT) * (Mpad / tc::BM);
    const long long ktiles = n / tc::BK;
    long long S = kNumSM / (tiles > 0 ? tiles : 1);
    if (S < 1) S = 1;
    if (S > 16) S = 16;
    if (S > ktiles) S = ktiles;
    const long long per = (ktiles + S - 1) / S;
    return (int)((ktiles + per - 1) / per);
}

size_t deflation_bf16_scratch(long long n, int k, int N) {
    const int NT = pick_nt_real(N);
    const size_t Ncols = (size_t)((N + NT - 1) / NT) * NT;
    const int Mpad = tc_deflation_rows(k);
    const int S = defl_splits(n, Mpad, (int)Ncols, NT);
    return Ncols * (size_t)n * sizeof(__nv_bfloat16) + (size_t)S * Mpad * Ncols * sizeof(float) + 256;
}

void launch_deflation_correction_bf16(double2* smp, const double2* X, const __nv_bfloat16* W, const double* a,
                                      long long n, int k, int N, void* scratch, int* err, cudaStream_t s) {
    MG_REQUIRE(tc_deflation_supported(n, k), MGMLMC_EINVAL, "tensor-core deflation needs n % 64 == 0");
    const int NT = pick_nt_real(N);
    const int Ncols = (N + NT - 1) / NT * NT;
    const int Mpad = tc_deflation_rows(k);
    const int S = defl_splits(n, Mpad, Ncols, NT);
    __nv_bfloat16* Bt = reinterpret_cast<__nv_bfloat16*>(scratch);
    float* Yp = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(scratch) + (size_t)Ncols * n * 2);
    dim3 g((Ncols + 31) / 32, (unsigned)((n + 31) / 32));
    tc::k_pack_x_real<<<g, dim3(32, 8), 0, s>>>(Bt, X, (int)n, N, Ncols, NT);
    MG_LAUNCHED();
    launch_tc(NT, Yp, W, Bt, Mpad, (int)n, Ncols, S, err, s);
    tc::k_defl_correction_tc<<<N, 256, 0, s>>>(smp, Yp, a, k, Mpad, Ncols, S);
    MG_LAUNCHED();
}


namespace tc {
// ------------------------------------------------------------------------------
// Coarse block stencil on the tensor cores, d = 16 (the first coarse level of the
// workloads): y(s) = sum_dir A(s, dir) x(nbr(s, dir)), the operator that the
// block-Jacobi smoother's minimal-residual steps apply.
//
// Per site the product is taken transposed, with the rhs as the MMA's M:
//     Y_s^T (rhs x 32 reals) = sum_dir X_nb^T (rhs x 32 reals) * B(s, dir) (32 x 32),
// where a row of X_nb^T is the 16 complex components of one rhs at the
// neighbour (re, im interleaved, exactly as the FP32 vectors store them) and
// B(s, dir) is the real form of A(s, dir)^T:
//     B[(c,re)][(c',re)] =  Re A[c'][c]     B[(c,im)][(c',re)] = -Im A[c'][c]
//     B[(c,re)][(c',im)] =  Im A[c'][c]     B[(c,im)][(c',im)] =  Re A[c'][c]
// B is precomputed once per level in the canonical layout (2 KB per site and
// direction).
//
// The input of the stencil is not the FP32 vector itself but its BF16 copy
// stored in the MMA's own operand layout: per site and 128-rhs tile, an 8 KB
// K-major tile whose row j is the 16 complex components of rhs j (pad rows of a
// partial last tile are zero).  The kernels that produce the smoother's
// residuals write that copy as they go (k_pack_tiles for the first one,
// k_mr_update_tc for the next ones), so the stencil moves 8 KB blocks straight
// into shared memory and never converts.
//
// Warp-specialised and persistent: three CTAs per SM, each over one 128-rhs tile
// and a strided set of sites; a CTA's work is a sequence of jobs (site,
// direction).
//   warp 0 (one thread): streams each job's neighbour tile (8 KB) with a 1-D
//     bulk copy into a ring of 6 stage buffers, and with a site's first job the
//     site's 10 KB of B (two site slots alternate);
//   warp 1 (one thread): issues two MMAs (M = 128, N = 32, K = 16) per job
//     straight from the stage buffer into the site's TMEM accumulator (two sets
//     of 32 columns alternate by site) and commits them: to the stage's empty
//     barrier, and after a site's last job to the accumulator's;
//   warps 2-5 (thread = rhs): read a finished accumulator (tcgen05.ld, 32
//     columns = 16 complex outputs), hand it back, store y coalesced along the
//     rhs, and add the smoother's dots against the site's BF16 input row.
namespace tcs {
constexpr int D = 16;
constexpr int KD = 2 * D;                  // reals per row of X^T (K of one direction)
constexpr int TILE_A = 128 * KD * 2;       // 8 KB: one 128-rhs BF16 tile of X^T
constexpr int B_DIR = KD * KD * 2;         // 2 KB: one B(s, dir)
constexpr int B_SITE = 5 * B_DIR;          // 10 KB per site
constexpr int CH = 128;                    // rhs per CTA (one 128-row tile)
constexpr int NSTG = 6;                    // stage ring depth
constexpr int THREADS = 192;               // 6 warps
constexpr int kCtasPerSm = 3;              // three pipelines per SM
constexpr int SMEM = NSTG * TILE_A + 2 * B_SITE;   // 68 KB: three CTAs per SM
constexpr int TCOLS = 64;                  // two accumulators of 32 columns
constexpr int kMaxDevWait = 1 << 26;
// direction of the o-th job of a site: the neighbours first, the self block last
__device__ __forceinline__ int dir_of(int o) { return o == 4 ? 0 : o + 1; }

// Byte offset of (row, k) in a K-major, no-swizzle tile with K = 32: 8-row groups
// of 512 B, four 128-byte core matrices along K, rows 16 B apart.
__host__ __device__ __forceinline__ int kmaj32_off(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// B(s, dir) for every site: E[(s * 5 + dir) * 1024 + off / 2], element (n = output
// real, k = input real) of the real form of A(s, dir)^T.
__global__ void k_embed_stencil(__nv_bfloat16* __restrict__ E, const float2* __restrict__ A, int nsites) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nsites * 5 * KD * KD) return;
    const long long sd = e / (KD * KD);
    const int r = (int)(e % (KD * KD)), n = r / KD, k = r % KD;
    const int co = n >> 1, to = n & 1, ci = k >> 1, ti = k & 1;
    const float2 a = A[sd * D * D + co * D + ci];
    const float v = (ti == to) ? a.x : (ti == 1 ? -a.y : a.y);
    E[sd * (KD * KD) + kmaj32_off(n, k) / 2] = __float2bfloat16(v);
}

// BF16 tiles of x: rt[(site * T + t) * 4096 + off / 2], zero rows for rhs >= N.
// Thread = (site, component group of 4, rhs): four FP32 loads, one 16-byte store.
// Grid: x = (site, component group), y = 128-rhs tile.
__global__ void k_pack_tiles(__nv_bfloat16* __restrict__ rt, const float2* __restrict__ x, int nsites, int N) {
    const int T = gridDim.y, tt = blockIdx.y;
    const int j = tt * CH + threadIdx.x;
    const int site = blockIdx.x >> 2, cg = blockIdx.x & 3;
    float2 v[4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
        v[p] = (j < N) ? x[((size_t)site * D + 4 * cg + p) * N + j] : make_float2(0.f, 0.f);
    uint4 w;
    w.x = pack_bf16(v[0].x, v[0].y);
    w.y = pack_bf16(v[1].x, v[1].y);
    w.z = pack_bf16(v[2].x, v[2].y);
    w.w = pack_bf16(v[3].x, v[3].y);
    uint8_t* tile = reinterpret_cast<uint8_t*>(rt) + ((size_t)site * T + tt) * TILE_A;
    *reinterpret_cast<uint4*>(tile + kmaj32_off(threadIdx.x, 8 * cg)) = w;
    (void)nsites;
}

// Minimal-residual update of the block-Jacobi smoother (alpha = dots[j] / dots[N + j]):
// yh (=|+=) alpha r, r -= alpha p, and (rt != null) the BF16 tiles of the new r.
// Thread = (site, rhs): the 16 rows of the site, four 16-byte tile pieces.
__global__ void __launch_bounds__(CH) k_mr_update_tc(float2* __restrict__ yh, float2* __restrict__ r,
                                                    const float2* __restrict__ p, const double2* __restrict__ dots,
                                                    int N, bool first, __nv_bfloat16* __restrict__ rt) {
    const int T = gridDim.y, tt = blockIdx.y;     // grid: x = site, y = 128-rhs tile
    const int j = tt * CH + threadIdx.x;
    const int site = blockIdx.x;
    float ax = 0.f, ay = 0.f;
    if (j < N) {
        const double2 pr = dots[j];
        const double pp = dots[N + j].x;
        if (pp > 0.0) {
            ax = (float)(pr.x / pp);
            ay = (float)(pr.y / pp);
        }
    }
    uint8_t* tile = rt ? reinterpret_cast<uint8_t*>(rt) + ((size_t)site * T + tt) * TILE_A : nullptr;
    // all loads of the thread first (memory-level parallelism), then the arithmetic
    float2 rv[D], pv[D], ev[D];
    const size_t base = (size_t)site * D * N + j;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const bool in = j < N;
        rv[c] = in ? r[base + (size_t)c * N] : make_float2(0.f, 0.f);
        pv[c] = in ? p[base + (size_t)c * N] : make_float2(0.f, 0.f);
        ev[c] = (in && !first) ? yh[base + (size_t)c * N] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        ev[c].x = fmaf(ax, rv[c].x, fmaf(-ay, rv[c].y, ev[c].x));
        ev[c].y = fmaf(ax, rv[c].y, fmaf(ay, rv[c].x, ev[c].y));
        rv[c] = make_float2(rv[c].x - fmaf(ax, pv[c].x, -ay * pv[c].y), rv[c].y - fmaf(ax, pv[c].y, ay * pv[c].x));
        if (j < N) {
            yh[base + (size_t)c * N] = ev[c];
            r[base + (size_t)c * N] = rv[c];
        }
    }
    if (tile) {
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            uint4 w;
            w.x = pack_bf16(rv[4 * cg].x, rv[4 * cg].y);
            w.y = pack_bf16(rv[4 * cg + 1].x, rv[4 * cg + 1].y);
            w.z = pack_bf16(rv[4 * cg + 2].x, rv[4 * cg + 2].y);
            w.w = pack_bf16(rv[4 * cg + 3].x, rv[4 * cg + 3].y);
            *reinterpret_cast<uint4*>(tile + kmaj32_off(threadIdx.x, 8 * cg)) = w;
        }
    }
}

// Minimal-residual update with r and p held only as BF16 tiles (the smoother's
// residual needs no more than a few digits): yh (=|+=) alpha r (FP32), r -= alpha p
// (BF16 tiles, in place).  Thread = (site, rhs): one row of each tile.
__global__ void __launch_bounds__(CH) k_mr_update_bf16(float2* __restrict__ yh, __nv_bfloat16* __restrict__ rt,
                                                      const __nv_bfloat16* __restrict__ pt,
                                                      const double2* __restrict__ dots, int N, bool first) {
    const int T = gridDim.y, tt = blockIdx.y;     // grid: x = site, y = 128-rhs tile
    const int jl = threadIdx.x, j = tt * CH + jl;
    const int site = blockIdx.x;
    if (j >= N) return;                           // pad rows stay zero
    const double2 pr = dots[j];
    const double pp = dots[N + j].x;
    const float ax = pp > 0.0 ? (float)(pr.x / pp) : 0.f, ay = pp > 0.0 ? (float)(pr.y / pp) : 0.f;
    const size_t toff = ((size_t)site * T + tt) * TILE_A;
    uint8_t* rrow = reinterpret_cast<uint8_t*>(rt) + toff;
    const uint8_t* prow = reinterpret_cast<const uint8_t*>(pt) + toff;
    uint4 rw[4], pw[4];
#pragma unroll
    for (int cg = 0; cg < 4; ++cg) {
        rw[cg] = *reinterpret_cast<const uint4*>(rrow + kmaj32_off(jl, 8 * cg));
        pw[cg] = *reinterpret_cast<const uint4*>(prow + kmaj32_off(jl, 8 * cg));
    }
    const size_t base = (size_t)site * D * N + j;
    float2 ev[D];
#pragma unroll
    for (int c = 0; c < D; ++c) ev[c] = first ? make_float2(0.f, 0.f) : yh[base + (size_t)c * N];
#pragma unroll
    for (int cg = 0; cg < 4; ++cg) {
        uint32_t rr[4] = {rw[cg].x, rw[cg].y, rw[cg].z, rw[cg].w};
        const uint32_t pq[4] = {pw[cg].x, pw[cg].y, pw[cg].z, pw[cg].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 4 * cg + q;
            const float rx = __uint_as_float(rr[q] << 16), ry = __uint_as_float(rr[q] & 0xFFFF0000u);
            const float px = __uint_as_float(pq[q] << 16), py = __uint_as_float(pq[q] & 0xFFFF0000u);
            ev[c].x = fmaf(ax, rx, fmaf(-ay, ry, ev[c].x));
            ev[c].y = fmaf(ax, ry, fmaf(ay, rx, ev[c].y));
            rr[q] = pack_bf16(rx - fmaf(ax, px, -ay * py), ry - fmaf(ax, py, ay * px));
        }
        *reinterpret_cast<uint4*>(rrow + kmaj32_off(jl, 8 * cg)) = make_uint4(rr[0], rr[1], rr[2], rr[3]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) yh[base + (size_t)c * N] = ev[c];
}

// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, unsigned parity, volatile int* abort_flag) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < kMaxDevWait; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// FORM 0: y = A x as FP32 rows, with the dots; 1: y as BF16 tiles (yt), with the dots;
// 2: the residual b - A x as BF16 tiles (yt), b FP32 rows, no dots.
template <int FORM>
__global__ void __launch_bounds__(THREADS, kCtasPerSm)
    k_block_stencil_tc(float2* __restrict__ y, __nv_bfloat16* __restrict__ yt, const float2* __restrict__ b,
                       const __nv_bfloat16* __restrict__ xt, const __nv_bfloat16* __restrict__ E, int lx, int lt, int N,
                       double2* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[NSTG], empty[NSTG], afull[2], aempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    uint8_t* stg = smem;                          // NSTG x 8 KB BF16 operand tiles
    uint8_t* bbuf = smem + NSTG * TILE_A;         // 2 x 10 KB B of a site
    volatile int* abrt = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int V = lx * lt;
    const int G = gridDim.x;
    const int T = gridDim.y;                      // 128-rhs tiles
    const int t = blockIdx.y;                     // this CTA's tile
    const int nsite = (V - (int)blockIdx.x + G - 1) / G;   // sites of this CTA
    const int njobs = 5 * nsite;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < NSTG; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&afull[q], 1);
            mbar_init(&aempty[q], 4);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const uint8_t* xtb = reinterpret_cast<const uint8_t*>(xt);

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int q = 0;
            for (; q < njobs; ++q) {
                const int si = q / 5, o = q % 5, slot = q % NSTG, as = si & 1;
                if (q >= NSTG && !mbar_wait_ab(&empty[slot], (unsigned)((q / NSTG - 1) & 1), abrt)) break;
                // the B slot is free once the MMAs of the site two back are done
                if (o == 0 && si >= 2 && !mbar_wait_ab(&afull[as], (unsigned)(((si - 2) >> 1) & 1), abrt)) break;
                const int site = blockIdx.x + si * G;
                const int nb = nbr_site(site, dir_of(o), lx, lt);
                mbar_expect_tx(&full[slot], (uint32_t)TILE_A + (o == 0 ? (uint32_t)B_SITE : 0u));
                bulk_g2s(stg + slot * TILE_A, xtb + ((size_t)nb * T + t) * TILE_A, (uint32_t)TILE_A, &full[slot]);
                if (o == 0)
                    bulk_g2s(bbuf + as * B_SITE, E + (size_t)site * (B_SITE / 2), (uint32_t)B_SITE, &full[slot]);
            }
            if (*abrt) {
                // copies still in flight land before the shared memory goes back: the
                // last job issued to each slot (earlier ones completed before reuse)
                for (int q2 = max(0, q - NSTG); q2 < q; ++q2) mbar_wait(&full[q2 % NSTG], (unsigned)((q2 / NSTG) & 1));
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = instr_desc(128, 32);
            int last = -1;
            for (int q = 0; q < njobs; ++q) {
                const int si = q / 5, o = q % 5, slot = q % NSTG, as = si & 1;
                if (o == 0 && si >= 2 && !mbar_wait_ab(&aempty[as], (unsigned)(((si >> 1) - 1) & 1), abrt)) break;
                if (!mbar_wait_ab(&full[slot], (unsigned)((q / NSTG) & 1), abrt)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(stg + slot * TILE_A);
                const uint32_t sb = smem_u32(bbuf + as * B_SITE + dir_of(o) * B_DIR);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ad = smem_desc(sa + ks * 256, 128, 512);
                    const uint64_t bd = smem_desc(sb + ks * 256, 128, 512);
                    const uint32_t acc = (o > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + as * 32),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty[slot])));
                if (o == 4)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&afull[as])));
                last = q;
            }
            if (*abrt && last >= 0) {
                // MMAs in flight complete before the TMEM and shared memory go back
                mbar_wait(&empty[last % NSTG], (unsigned)((last / NSTG) & 1));
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int quarter = warp & 3;             // TMEM lanes this warp may read
        const int jl = quarter * 32 + lane;
        const int j = t * CH + jl;
        float2 dyx = make_float2(0.f, 0.f);
        float dyy = 0.f;
        bool ok = true;
        for (int si = 0; si < nsite; ++si) {
            const int as = si & 1;
            if (!mbar_wait_ab(&afull[as], (unsigned)((si >> 1) & 1), abrt)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(as * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&aempty[as]);      // accumulator may be overwritten
            if (FORM != 0 && j >= N) {
                // pad rows of a partial tile stay zero
                uint8_t* yrow = reinterpret_cast<uint8_t*>(yt) + ((size_t)(blockIdx.x + si * G) * T + t) * TILE_A;
#pragma unroll
                for (int cg = 0; cg < 4; ++cg)
                    *reinterpret_cast<uint4*>(yrow + kmaj32_off(jl, 8 * cg)) = make_uint4(0u, 0u, 0u, 0u);
            }
            if (j < N) {
                const int site = blockIdx.x + si * G;
                float2 ov[D];
#pragma unroll
                for (int co = 0; co < D; ++co) {
                    ov[co] = make_float2(__uint_as_float(r[2 * co]), __uint_as_float(r[2 * co + 1]));
                    if (FORM == 2) {
                        const float2 bv = b[((size_t)site * D + co) * N + j];
                        ov[co] = make_float2(bv.x - ov[co].x, bv.y - ov[co].y);
                    }
                }
                if (FORM != 0) {
                    uint8_t* yrow = reinterpret_cast<uint8_t*>(yt) + ((size_t)site * T + t) * TILE_A;
#pragma unroll
                    for (int cg = 0; cg < 4; ++cg) {
                        uint4 w;
                        w.x = pack_bf16(ov[4 * cg].x, ov[4 * cg].y);
                        w.y = pack_bf16(ov[4 * cg + 1].x, ov[4 * cg + 1].y);
                        w.z = pack_bf16(ov[4 * cg + 2].x, ov[4 * cg + 2].y);
                        w.w = pack_bf16(ov[4 * cg + 3].x, ov[4 * cg + 3].y);
                        *reinterpret_cast<uint4*>(yrow + kmaj32_off(jl, 8 * cg)) = w;
                    }
                }
                if (FORM == 2) continue;
                // the site's own BF16 input row (16 components of rhs j) for the dots
                const uint8_t* own = xtb + ((size_t)site * T + t) * TILE_A;
                uint4 xw[4];
#pragma unroll
                for (int cg = 0; cg < 4; ++cg) xw[cg] = *reinterpret_cast<const uint4*>(own + kmaj32_off(jl, 8 * cg));
#pragma unroll
                for (int co = 0; co < D; ++co) {
                    if (FORM == 0) y[((size_t)site * D + co) * N + j] = ov[co];
                    const uint32_t wbits = (co & 3) == 0 ? xw[co >> 2].x
                                           : (co & 3) == 1 ? xw[co >> 2].y
                                           : (co & 3) == 2 ? xw[co >> 2].z : xw[co >> 2].w;
                    const float2 xv = make_float2(__uint_as_float(wbits << 16), __uint_as_float(wbits & 0xFFFF0000u));
                    // conj(y) * x, accumulated per rhs
                    dyx.x = fmaf(ov[co].x, xv.x, fmaf(ov[co].y, xv.y, dyx.x));
                    dyx.y = fmaf(ov[co].x, xv.y, fmaf(-ov[co].y, xv.x, dyx.y));
                    dyy = fmaf(ov[co].x, ov[co].x, fmaf(ov[co].y, ov[co].y, dyy));
                }
            }
        }
        if (FORM != 2 && ok && j < N) {
            part[((long long)0 * N + j) * G + blockIdx.x] = make_double2((double)dyx.x, (double)dyx.y);
            part[((long long)1 * N + j) * G + blockIdx.x] = make_double2((double)dyy, 0.0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0 && abort_flag) atomicExch(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}
}  // namespace tcs
}  // namespace tc

bool tc_stencil_supported(int d, int N) { return d == tc::tcs::D && N >= 1 && N <= 65535 * tc::tcs::CH; }

void launch_embed_stencil_bf16(__nv_bfloat16* E, const float2* A, int nsites, cudaStream_t s) {
    const long long tot = (long long)nsites * 5 * tc::tcs::KD * tc::tcs::KD;
    tc::tcs::k_embed_stencil<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(E, A, nsites);
    MG_LAUNCHED();
}

static int tc_tiles(int N) { return (N + tc::tcs::CH - 1) / tc::tcs::CH; }

size_t tc_tiles_bytes(int nsites, int N) { return (size_t)nsites * tc_tiles(N) * tc::tcs::TILE_A; }

void launch_pack_tiles_bf16(__nv_bfloat16* rt, const float2* x, int nsites, int N, cudaStream_t s) {
    MG_REQUIRE(nsites >= 1 && nsites <= (1 << 28) && tc_tiles(N) <= 65535, MGMLMC_EINVAL, "BF16 tiles: size");
    tc::tcs::k_pack_tiles<<<dim3(4 * nsites, tc_tiles(N)), tc::tcs::CH, 0, s>>>(rt, x, nsites, N);
    MG_LAUNCHED();
}

void launch_mr_update_tc(float2* yh, float2* r, const float2* p, const double2* dots, int nsites, int N, bool first,
                         __nv_bfloat16* rt, cudaStream_t s) {
    MG_REQUIRE(nsites >= 1 && nsites <= (1 << 30) && tc_tiles(N) <= 65535, MGMLMC_EINVAL, "BF16 tiles: size");
    tc::tcs::k_mr_update_tc<<<dim3(nsites, tc_tiles(N)), tc::tcs::CH, 0, s>>>(yh, r, p, dots, N, first, rt);
    MG_LAUNCHED();
}

// Three persistent CTAs per SM (68 KB of shared memory each) over the 128-rhs tiles.
int block_stencil_tc_groups(int nsites, int N) {
    int g = tc::tcs::kCtasPerSm * kNumSM / tc_tiles(N);
    if (g < 1) g = 1;
    return nsites < g ? nsites : g;
}

template <int FORM>
static void bstc_launch(float2* y, __nv_bfloat16* yt, const float2* b, const __nv_bfloat16* xt,
                        const __nv_bfloat16* E, int lx, int lt, int N, double2* part, int groups, int* err,
                        cudaStream_t s) {
    MG_CUDA(cudaFuncSetAttribute(tc::tcs::k_block_stencil_tc<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::tcs::SMEM));
    dim3 g(groups, tc_tiles(N));
    tc::tcs::k_block_stencil_tc<FORM><<<g, tc::tcs::THREADS, tc::tcs::SMEM, s>>>(y, yt, b, xt, E, lx, lt, N, part, err);
    MG_LAUNCHED();
}

void launch_block_stencil_tc(float2* y, __nv_bfloat16* yt, const float2* b, const __nv_bfloat16* xt,
                             const __nv_bfloat16* E, int lx, int lt, int N, double2* part, int groups, int* err,
                             cudaStream_t s) {
    MG_REQUIRE(tc_stencil_supported(16, N), MGMLMC_EINVAL, "tensor-core stencil: d = 16");
    MG_REQUIRE(groups >= 1 && groups <= lx * lt, MGMLMC_EINVAL, "tensor-core stencil: bad grid");
    MG_REQUIRE((y != nullptr) != (yt != nullptr) && !(b && y), MGMLMC_EINVAL, "tensor-core stencil: one output form");
    MG_REQUIRE(((uintptr_t)xt & 15) == 0 && ((uintptr_t)E & 15) == 0 && ((uintptr_t)yt & 15) == 0, MGMLMC_EINVAL,
               "tensor-core stencil: operands must be 16-byte aligned");
    if (y) bstc_launch<0>(y, yt, b, xt, E, lx, lt, N, part, groups, err, s);
    else if (!b) bstc_launch<1>(y, yt, b, xt, E, lx, lt, N, part, groups, err, s);
    else bstc_launch<2>(y, yt, b, xt, E, lx, lt, N, part, groups, err, s);
}

void launch_mr_update_bf16(float2* yh, __nv_bfloat16* rt, const __nv_bfloat16* pt, const double2* dots, int nsites,
                           int N, bool first, cudaStream_t s) {
    MG_REQUIRE(nsites >= 1 && nsites <= (1 << 30) && tc_tiles(N) <= 65535, MGMLMC_EINVAL, "BF16 tiles: size");
    tc::tcs::k_mr_update_bf16<<<dim3(nsites, tc_tiles(N)), tc::tcs::CH, 0, s>>>(yh, rt, pt, dots, N, first);
    MG_LAUNCHED();
}

}  // namespace mg

// ------------------------------------------------------------------------------
// Allocation-free variant of the coarsest solve.  The packed operand B' lives in
// a file-scope device array instead of context work space, so the call itself
// never allocates.  Its address is looked up once per device with
// cudaGetSymbolAddress (host code must not use the symbol as a device pointer).
#include <mutex>

#include "context.h"

namespace mg {
namespace tc {
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB: B' for n_L * nrhs <= 2^20
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ int g_noalloc_err;

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[kMaxDevices];
static int* g_noalloc_err_ptr[kMaxDevices];

// Device addresses of the static scratch and error flag for the current device.
static void noalloc_symbols(void** scratch, int** err) {
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    MG_REQUIRE(dev >= 0 && dev < kMaxDevices, MGMLMC_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        void* e = nullptr;
        MG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        MG_CUDA(cudaGetSymbolAddress(&e, g_noalloc_err));
        g_noalloc_err_ptr[dev] = reinterpret_cast<int*>(e);
        g_noalloc_ptr[dev] = p;
    }
    *scratch = g_noalloc_ptr[dev];
    *err = g_noalloc_err_ptr[dev];
}
}  // namespace tc
}  // namespace mg

extern "C" int mgmlmc_coarse_inverse_noalloc(mgmlmc_ctx* h, int nrhs, const float* x, float* y, void* stream) {
    if (!h) return MGMLMC_EINVAL;
    mg::Ctx& c = h->c;
    c.err.clear();
    try {
        MG_REQUIRE(c.have_hier, MGMLMC_ESTATE, "coarse_inverse_noalloc: no hierarchy");
        const mg::Level& L = c.lev[c.L - 1];
        MG_REQUIRE(L.Dinv16 != nullptr, MGMLMC_ESTATE,
                   "coarse_inverse_noalloc: needs mg_precision 32 or 16 and a coarsest level with n_L % 128 == 0");
        MG_REQUIRE(x && y && x != y, MGMLMC_EINVAL, "coarse_inverse_noalloc: x, y must be distinct device pointers");
        // the kernel stores y with 16-byte vector stores and reads x as 8-byte pairs
        MG_REQUIRE(((uintptr_t)y & 15) == 0 && ((uintptr_t)x & 7) == 0, MGMLMC_EINVAL,
                   "coarse_inverse_noalloc: y must be 16-byte and x 8-byte aligned");
        MG_REQUIRE(nrhs >= 32 && nrhs % 32 == 0, MGMLMC_EINVAL, "coarse_inverse_noalloc: nrhs must be a multiple of 32");
        const int n = (int)L.n;
        const size_t need = (size_t)2 * nrhs * 2 * n * sizeof(__nv_bfloat16);
        MG_REQUIRE(need <= mg::tc::kNoAllocScratchBytes, MGMLMC_EINVAL,
                   "coarse_inverse_noalloc: n_L * nrhs above 2^20 (static scratch of 8 MiB)");
        void* scratch = nullptr;
        int* err = nullptr;
        mg::tc::noalloc_symbols(&scratch, &err);
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const int Ncols = 2 * nrhs;
        MG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        const int NT = (Ncols % 256 == 0) ? 256 : (Ncols % 128 == 0 ? 128 : 64);
        mg::launch_pack(reinterpret_cast<__nv_bfloat16*>(scratch), reinterpret_cast<const float2*>(x), n, nrhs, Ncols,
                        NT, s);
        const __nv_bfloat16* Bt = reinterpret_cast<const __nv_bfloat16*>(scratch);
        mg::launch_tc(NT, y, L.Dinv16, Bt, n, 2 * n, Ncols, 1, err, s);
        int herr = 0;
        MG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        MG_REQUIRE(herr == 0, MGMLMC_ETIMEOUT, "coarse_inverse_noalloc: a bounded mbarrier wait gave up");
    } catch (const mg::Error& e) {
        c.err = e.what();
        return e.code;
    }
    return MGMLMC_OK;
}
