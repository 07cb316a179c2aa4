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
// Kernel: one CTA (4 warps) per 128 x NT output tile.  A 4-stage cp.async
// pipeline stages 128x64 (A) and NTx64 (B) tiles; thread 0 issues 4
// tcgen05.mma (K = 16 each) per stage and commits them to the stage's
// mbarrier; the accumulator lives in TMEM (NT columns) and is read back with
// tcgen05.ld.  Every mbarrier wait is bounded: on timeout the CTA records an
// error flag, drains its copies, frees TMEM and returns.
#include "kernels.cuh"

namespace mg {

namespace tc {

constexpr int BM = 128;         // rows per tile (TMEM lanes)
constexpr int BK = 64;          // K per stage (4 MMAs of K = 16)
constexpr int STAGES = 4;
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Canonical K-major layout of a rows x 64 BF16 tile: 8-row groups of 1024 B
// (eight 128-byte core matrices along K), rows 16 B apart inside a core matrix.
__device__ __forceinline__ uint32_t tile_off(int row, int kchunk) {
    return (uint32_t)((row >> 3) * 1024 + kchunk * 128 + (row & 7) * 16);
}

template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm_bf16(float* __restrict__ Y, const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Bt,
                   int M, int K, int Ncols, int* __restrict__ err) {
    constexpr int A_BYTES = BM * BK * 2;
    constexpr int B_BYTES = NT * BK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[STAGES];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * NT;
    const int nk = K / BK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&mbar[s], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    auto load_stage = [&](int kt, int s) {
        uint8_t* sa = smem + s * STAGE_BYTES;
        uint8_t* sb = sa + A_BYTES;
        const int k0 = kt * BK;
        for (int c = tid; c < BM * 8; c += 128) {
            const int r = c >> 3, kc = c & 7;
            cp_async16(sa + tile_off(r, kc), A + (size_t)(m0 + r) * K + k0 + kc * 8);
        }
        for (int c = tid; c < NT * 8; c += 128) {
            const int r = c >> 3, kc = c & 7;
            cp_async16(sb + tile_off(r, kc), Bt + (size_t)(n0 + r) * K + k0 + kc * 8);
        }
    };

    constexpr uint32_t IDESC = instr_desc(BM, NT);
    bool ok = true;
    // prologue: stages 0 .. STAGES-2
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int s = kt % STAGES;
        // refill the stage consumed STAGES-1 iterations ago, once its MMAs are done
        const int kn = kt + STAGES - 1;
        if (kn < nk) {
            const int sn = kn % STAGES;
            if (kn >= STAGES) {
                if (!mbar_wait(&mbar[sn], (unsigned)((kn / STAGES - 1) & 1))) {
                    ok = false;
                    atomicExch(&abort_flag, 1);
                }
            }
            if (ok) load_stage(kn, sn);
        }
        cp_async_commit();
        cp_async_wait<STAGES - 1>();             // tile kt has landed (this thread's part)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) { ok = false; break; }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t ad = smem_desc(sa + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(sb + ks * 256, 128, 1024);
                const uint32_t acc = (kt > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[s])));
        }
    }
    cp_async_wait<0>();
    if (ok && nk > 0) {
        const int last = nk - 1;
        if (!mbar_wait(&mbar[last % STAGES], (unsigned)((last / STAGES) & 1))) ok = false;
    }
    __syncthreads();
    if (!ok) abort_flag = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!abort_flag) {
        // epilogue: warp w owns TMEM lanes 32w .. 32w+31 = output rows
        const int row = m0 + warp * 32 + lane;
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
                float4* dst = reinterpret_cast<float4*>(Y + (size_t)row * Ncols + n0 + c);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

// A'[i][k] = Re A[i][k], A'[i][n + k] = Im A[i][k]   (A complex FP32 n x n)
__global__ void k_embed_a(__nv_bfloat16* __restrict__ E, const float2* __restrict__ A, int n) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const long long i = e / n, k = e % n;
    const float2 v = A[e];
    E[i * 2 * n + k] = __float2bfloat16(v.x);
    E[i * 2 * n + n + k] = __float2bfloat16(v.y);
}

// Bt[col][k] (K-major B' of the real embedding), col = 2j + p; zero for col >= 2N.
//   k <  n: p = 0 -> Re X[k][j],       p = 1 -> Im X[k][j]
//   k >= n: p = 0 -> -Im X[k-n][j],    p = 1 -> Re X[k-n][j]
__global__ void k_pack_bt(__nv_bfloat16* __restrict__ Bt, const float2* __restrict__ X, int n, int N, int Ncols) {
    __shared__ float2 t[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;   // rows of X, rhs
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && j < N) ? X[(size_t)i * N + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int K = 2 * n;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int i = i0 + threadIdx.x;
        if (i >= n || 2 * j + 1 >= Ncols) continue;
        const float2 v = (j < N) ? t[threadIdx.x][r] : make_float2(0.f, 0.f);
        Bt[(size_t)(2 * j) * K + i] = __float2bfloat16(v.x);
        Bt[(size_t)(2 * j) * K + n + i] = __float2bfloat16(-v.y);
        Bt[(size_t)(2 * j + 1) * K + i] = __float2bfloat16(v.y);
        Bt[(size_t)(2 * j + 1) * K + n + i] = __float2bfloat16(v.x);
    }
}

__global__ void k_unpad_y(float2* __restrict__ Y, const float* __restrict__ Yp, int n, int N, int Ncols) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * N) return;
    const long long i = e / N, j = e % N;
    Y[e] = make_float2(Yp[i * Ncols + 2 * j], Yp[i * Ncols + 2 * j + 1]);
}

}  // namespace tc

void launch_embed_bf16(__nv_bfloat16* E, const float2* A, int n, cudaStream_t s) {
    const long long tot = (long long)n * n;
    tc::k_embed_a<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(E, A, n);
    MG_LAUNCHED();
}

bool tc_coarse_supported(int n) { return n >= 128 && n % 128 == 0; }

static int pick_nt(int N) { return (2 * N >= 256) ? 256 : (2 * N > 64 ? 128 : 64); }

size_t coarse_inverse_bf16_scratch(int n, int N) {
    const int NT = pick_nt(N);
    const size_t ncols = (size_t)((2 * N + NT - 1) / NT) * NT;
    return ncols * 2 * n * sizeof(__nv_bfloat16) + (size_t)n * ncols * sizeof(float) + 256;
}

template <int NT>
static void launch_tc(float* Y, const __nv_bfloat16* A, const __nv_bfloat16* Bt, int M, int K, int Ncols, int* err,
                      cudaStream_t s) {
    constexpr int smem = tc::STAGES * (tc::BM * tc::BK * 2 + NT * tc::BK * 2);
    MG_CUDA(cudaFuncSetAttribute(tc::k_tc_gemm_bf16<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 g(Ncols / NT, M / tc::BM);
    tc::k_tc_gemm_bf16<NT><<<g, 128, smem, s>>>(Y, A, Bt, M, K, Ncols, err);
    MG_LAUNCHED();
}

void launch_coarse_inverse_bf16(float2* Y, const float2* X, const __nv_bfloat16* E, int n, int N, void* scratch,
                                int* err, cudaStream_t s) {
    MG_REQUIRE(tc_coarse_supported(n), MGMLMC_EINVAL, "tensor-core coarsest solve needs n % 128 == 0");
    const int NT = pick_nt(N);
    const int Ncols = ((2 * N + NT - 1) / NT) * NT;
    __nv_bfloat16* Bt = reinterpret_cast<__nv_bfloat16*>(scratch);
    float* Yp = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(scratch) + (size_t)Ncols * 2 * n * 2);
    {
        dim3 g((Ncols / 2 + 31) / 32, (n + 31) / 32);
        tc::k_pack_bt<<<g, dim3(32, 8), 0, s>>>(Bt, X, n, N, Ncols);
        MG_LAUNCHED();
    }
    const bool direct = (Ncols == 2 * N);
    float* out = direct ? reinterpret_cast<float*>(Y) : Yp;
    if (NT == 256) launch_tc<256>(out, E, Bt, n, 2 * n, Ncols, err, s);
    else if (NT == 128) launch_tc<128>(out, E, Bt, n, 2 * n, Ncols, err, s);
    else launch_tc<64>(out, E, Bt, n, 2 * n, Ncols, err, s);
    if (!direct) {
        const long long tot = (long long)n * N;
        tc::k_unpad_y<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Y, Yp, n, N, Ncols);
        MG_LAUNCHED();
    }
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
                   "coarse_inverse_noalloc: needs mg_precision = 32 and a coarsest level with n_L % 128 == 0");
        MG_REQUIRE(x && y && x != y, MGMLMC_EINVAL, "coarse_inverse_noalloc: x, y must be distinct device pointers");
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
        {
            dim3 g((Ncols / 2 + 31) / 32, (n + 31) / 32);
            mg::tc::k_pack_bt<<<g, dim3(32, 8), 0, s>>>(reinterpret_cast<__nv_bfloat16*>(scratch),
                                                       reinterpret_cast<const float2*>(x), n, nrhs, Ncols);
            MG_LAUNCHED();
        }
        const __nv_bfloat16* Bt = reinterpret_cast<const __nv_bfloat16*>(scratch);
        if (Ncols % 256 == 0) mg::launch_tc<256>(y, L.Dinv16, Bt, n, 2 * n, Ncols, err, s);
        else if (Ncols % 128 == 0) mg::launch_tc<128>(y, L.Dinv16, Bt, n, 2 * n, Ncols, err, s);
        else mg::launch_tc<64>(y, L.Dinv16, Bt, n, 2 * n, Ncols, err, s);
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
