// Shared helpers of the CUDA path: error handling, complex arithmetic on
// float2/double2, launch geometry.  Part of the product library; independent
// of the CPU oracle.
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "mgmlmc.h"

namespace mg {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define MG_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            throw ::mg::Error(MGMLMC_ECUDA, std::string(#call) + ": " +                 \
                                                cudaGetErrorString(e_));               \
    } while (0)

// Kernel launches issued by this library (process-wide), for launch accounting.
std::atomic<long long>& launch_counter();   // all contexts, thread-safe

#define MG_LAUNCHED()                                                                  \
    do {                                                                               \
        ++::mg::launch_counter();                                                      \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess)                                                         \
            throw ::mg::Error(MGMLMC_ECUDA, std::string("kernel launch in ") +         \
                                                __func__ + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define MG_REQUIRE(cond, code, msg)                                                    \
    do {                                                                               \
        if (!(cond)) throw ::mg::Error((code), (msg));                                  \
    } while (0)

// ---- complex type per real type --------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <typename R> using cx_t = typename Cx<R>::T;
template <typename C> struct Re;
template <> struct Re<double2> { using T = double; };
template <> struct Re<float2> { using T = float; };
template <typename C> using re_t = typename Re<C>::T;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
// a * b
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <typename C> __host__ __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { return mk(a.x * s, a.y * s); }
// i * a
template <typename C> __host__ __device__ __forceinline__ C ctimesi(C a) { return mk(-a.y, a.x); }

__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename C> __host__ __device__ __forceinline__ C cvt(double2 a);
template <> __host__ __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ float2 cvtc(float2 a, float2) { return a; }
__host__ __device__ __forceinline__ float2 cvtc(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 cvtc(float2 a, double2) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 cvtc(double2 a, double2) { return a; }
template <typename C> __device__ __forceinline__ C from_d(double2 a);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---- launch geometry ---------------------------------------------------------------
constexpr int kNumSM = 152;          // GB300: 2 dies x 76 SMs
constexpr int kRhsTile = 32;         // right-hand sides per warp (threadIdx.x)
constexpr int kRowLanes = 8;         // rows per block (threadIdx.y)

inline int rhs_tiles(int N) { return (N + kRhsTile - 1) / kRhsTile; }
// Number of row groups for grid-stride kernels: about 4 resident blocks per SM.
inline int row_groups(long long rows, int N, int per_sm = 4) {
    long long want = (long long)kNumSM * per_sm / rhs_tiles(N);
    if (want < 1) want = 1;
    long long need = (rows + kRowLanes - 1) / kRowLanes;
    return (int)(need < want ? need : want);
}

}  // namespace mg
