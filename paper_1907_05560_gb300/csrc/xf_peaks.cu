// xf_peaks.cu -- microbenchmarks that give the ALU roofline denominators:
// FP64 and FP32 FMA throughput, measured with CUDA events on this GPU; and
// the throughput of the FP64 functions the 3x3 propagator calls besides its
// counted arithmetic (reciprocal square root, sine-cosine pair), which prices
// them in FMA issue slots.
#include <cuda_runtime.h>

#include "../../include/xf.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void fma_kernel(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.678) out[0] = s; // keeps the chains alive
}

// 8 independent chains per thread of y = rsqrt(fma(y, a, b)) (arguments stay
// near 1), or of (s, c) = sincos(y), y = fma(s, a, c) (arguments in [-2, 2]).
template <int OP>
__global__ void func_kernel(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 0.01 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (OP == 0) {
                x[c] = rsqrt(fma(x[c], a, b));
            } else {
                double sn, cs;
                sincos(x[c], &sn, &cs);
                x[c] = fma(sn, a, cs);
            }
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
}

template <int OP>
int run_func(double *ops_per_s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return XF_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return XF_E_NOMEM;
    const int threads = 256, blocks = sms * 8, iters = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    func_kernel<OP><<<blocks, threads>>>(out, iters, 0.5, 0.75); // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        func_kernel<OP><<<blocks, threads>>>(out, iters, 0.5, 0.75);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return XF_E_CUDA;
    // one rsqrt (plus its FMA) or one sine-cosine pair (plus its FMA) per chain step
    *ops_per_s = (double)kChains * iters * threads * blocks / (best * 1e-3);
    return XF_OK;
}

template <typename T>
int run(double *flops_per_s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return XF_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return XF_E_NOMEM;
    const int threads = 256, blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7); // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        fma_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return XF_E_CUDA;
    *flops_per_s = 2.0 * kChains * (double)iters * threads * blocks / (best * 1e-3);
    return XF_OK;
}

} // namespace

extern "C" int xf_peak(int which, double *value)
{
    if (!value) return XF_E_ARG;
    if (which == XF_PEAK_FP64_FMA) return run<double>(value);
    if (which == XF_PEAK_FP32_FMA) return run<float>(value);
    if (which == XF_PEAK_FP64_RSQRT) return run_func<0>(value);
    if (which == XF_PEAK_FP64_SINCOS) return run_func<1>(value);
    return XF_E_ARG;
}
