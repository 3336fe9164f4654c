// FMA throughput of the SM's SIMT pipes (FP32 and FP64), measured: the
// denominator of the ALU-bound block inversion's roofline beside the figure
// from unit counts (lanes x 2 flops x clock).
//
// Every thread runs kChains independent FMA chains x <- x * b + c (|b| < 1,
// so the values stay finite and the compiler cannot fold the loop), enough
// chains per warp to cover the pipe latency; the grid fills every SM to its
// thread limit. Each thread writes its sum, so no chain is dead code.
#include <cuda_runtime.h>

#include "dev.cuh"
#include "kernels.h"

namespace ipcb {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;

template <class T>
__global__ void __launch_bounds__(512) k_fma_chains(T b, T c, int iters, T* out) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = x[i] * b + c;  // contracted to one FMA
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

template <class T>
int measure_fma_peak(double target_ms, double* tflops) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int threads = 512;
    const int blocks = sms * (per_sm / threads);
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = (T)0.999999, c = (T)1e-6;
    // calibrate on a short run, then time one launch of about target_ms
    int iters = 64;
    float ms = 0.f;
    int rc = 0;
    for (int round = 0; round < 2 && rc == 0; ++round) {
        KL(k_fma_chains<T><<<blocks, threads>>>(b, c, iters, out));  // warm-up at this size
        cudaEventRecord(e0);
        KL(k_fma_chains<T><<<blocks, threads>>>(b, c, iters, out));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = -1;
        cudaEventElapsedTime(&ms, e0, e1);
        if (round == 0) {
            const double scale = target_ms / (ms > 1e-3f ? ms : 1e-3f);
            iters = (int)fmin(fmax(iters * scale, 64.0), 1 << 24);
        }
    }
    if (cudaGetLastError() != cudaSuccess) rc = -1;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
    *tflops = rc == 0 && ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

template int measure_fma_peak<float>(double, double*);
template int measure_fma_peak<double>(double, double*);

}  // namespace ipcb
