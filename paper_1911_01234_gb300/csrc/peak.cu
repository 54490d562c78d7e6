// Peak FMA throughput of the current GPU in FP32 and FP64, measured by a
// kernel of independent fused multiply-add chains (the denominator of the ALU
// roofline of the transforms: the plain path is FP32 arithmetic on the CUDA
// cores, with FP64 reductions).  The paper has no counterpart; this is a
// measurement of the machine, not a step of the method.
//
// Each thread runs 8 independent chains x <- x a + b (a just below 1, so the
// values stay near b / (1 - a) and never become subnormal), unrolled 16 deep,
// which hides the FMA latency with 8 warps per scheduler.  The grid is 4
// resident 256-thread CTAs per SM.  FLOPs = 2 per FMA.
#include <algorithm>
#include <string>

#include "../../include/vdamp.h"
#include "vdamp_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(T* sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1) sink[blockIdx.x] = s;   // never true: keeps the chains live
}

template <typename T>
vdamp_status run(int iters, cudaStream_t st, double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        vdamp::set_last_error(cudaGetErrorString(e));
        return VDAMP_ECUDA;
    }
    const int blocks = 4 * sms;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 0.f;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one warm-up launch, then the faster of three timed launches
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fma_peak_kernel<T><<<blocks, kThreads, 0, st>>>(nullptr, iters, (T)0.999999, (T)1e-6);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        vdamp::set_last_error(cudaGetErrorString(e));
        return VDAMP_ECUDA;
    }
    const double flops = 2.0 * kChains * kUnroll * (double)iters * kThreads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return VDAMP_OK;
}

}  // namespace

extern "C" vdamp_status vdamp_fma_peak(int precision, int iters, double* tflops, double* ms,
                                       void* stream) {
    if (!tflops || iters < 1 || (precision != 32 && precision != 64)) {
        vdamp::set_last_error("vdamp_fma_peak: precision must be 32 or 64, iters >= 1");
        return VDAMP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return precision == 32 ? run<float>(iters, st, tflops, ms) : run<double>(iters, st, tflops, ms);
}
