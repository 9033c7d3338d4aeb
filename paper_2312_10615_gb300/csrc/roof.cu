// roof.cu -- measured arithmetic roof of the CUDA cores (FP64 or FP32 fused multiply-add rate).
//
// The FP64 kernels of the path (the operator apply of Alg. 4 and the SQMR vector recurrences) are
// bound by the FP64 pipe, not by HBM; their roofline needs the rate this part really sustains.
// The probe runs a grid of 152 SMs x resident blocks, each thread carrying kChains independent FMA
// chains through kIters dependent steps (enough independent work to fill the pipe's latency), and
// times it with CUDA events on the caller's stream.  The chains' values feed a store guarded by a
// condition that never holds, so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include "stokesmg.h"

namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T seed) {
    T a[kChains];
    const T m = T(0.999999) + seed * T(1e-9), c = T(1e-7);
#pragma unroll
    for (int u = 0; u < kChains; ++u) a[u] = T(threadIdx.x + u) * T(1e-3) + seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int u = 0; u < kChains; ++u) s += a[u];
    if (s == T(-12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true
}

template <class T> int measure(double *rate, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STOKES_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, 256, 0);
    if (sms <= 0 || per_sm <= 0) return STOKES_ERR_CUDA;
    const int blocks = sms * per_sm;
    const int iters = sizeof(T) == 8 ? 256 : 8192;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * 256) != cudaSuccess) {
        cudaGetLastError();
        return STOKES_ERR_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_probe<T><<<blocks, 256, 0, s>>>(out, iters, T(0.5));  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_probe<T><<<blocks, 256, 0, s>>>(out, iters, T(0.5));
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return STOKES_ERR_CUDA;
    const double flops = 2.0 * kChains * 16.0 * iters * 256.0 * blocks;
    *rate = flops / (best * 1e-3);
    return STOKES_OK;
}

}  // namespace

extern "C" int stokes_measure_fma_peak(int fp64, double *flops_per_s, void *stream) {
    if (!flops_per_s) return STOKES_ERR_INVALID_ARG;
    return fp64 ? measure<double>(flops_per_s, (cudaStream_t)stream) : measure<float>(flops_per_s, (cudaStream_t)stream);
}
