// Measurement helper: fused multiply-add throughput of the device (used to
// state the ALU roofline of the FP64 kernels next to the measured HBM and
// tensor peaks).  Eight independent FMA chains per thread, every SM busy.
#include <cstdio>

#include "common.cuh"

namespace mg {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_peak(R* out, int iters, R a, R b) {
    R x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (R)-12345.0) out[0] = s;   // keeps the chains alive
}

template <typename R>
static double run_peak(int iters) {
    cudaStream_t st;
    MG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    R* out = nullptr;
    MG_CUDA(cudaMalloc(&out, sizeof(R)));
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    const int blocks = kNumSM * 8, threads = 256;
    k_fma_peak<R><<<blocks, threads, 0, st>>>(out, iters / 8, (R)0.9999999, (R)1e-7);
    MG_LAUNCHED();
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        MG_CUDA(cudaEventRecord(e0, st));
        k_fma_peak<R><<<blocks, threads, 0, st>>>(out, iters, (R)0.9999999, (R)1e-7);
        MG_LAUNCHED();
        MG_CUDA(cudaEventRecord(e1, st));
        MG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double fl = 2.0 * 8.0 * (double)iters * blocks * threads;
        if (ms > 0 && fl / (ms * 1e-3) > best) best = fl / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaStreamDestroy(st);
    return best;
}

}  // namespace mg

extern "C" int mgmlmc_fma_peak(int precision, double* flops_per_s) {
    if (!flops_per_s || (precision != 64 && precision != 32)) return MGMLMC_EINVAL;
    try {
        *flops_per_s = precision == 64 ? mg::run_peak<double>(8192) : mg::run_peak<float>(262144);
    } catch (const mg::Error& e) {
        return e.code;
    }
    return MGMLMC_OK;
}
