// FMA throughput probe (measurement only, not part of libpfc.so): the FP32 and FP64 rates of the
// GPU's plain (non-tensor) FMA pipes, against which the transform-bound FP64 path is reported.
// Every thread runs 8 independent FMA chains, so the pipes, not the dependency latency, bound
// the rate; blocks fill every SM several times over.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)12345.678) out[blockIdx.x] = s;   // keeps the chains live
}

template <typename T> int probe(double *flops_per_s) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = nsm * 8, threads = 256, iters = sizeof(T) == 4 ? 4096 : 256;
    T *out = nullptr;
    if (cudaMalloc(&out, blocks * sizeof(T)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999, b = (T)1e-4;
    k_fma_chains<T><<<blocks, threads>>>(out, iters, a, b);
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, threads>>>(out, iters, a, b);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 8 * 4 * (double)iters * blocks * threads;
        if (ms > 0.f && flops / (ms * 1e-3) > best) best = flops / (ms * 1e-3);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return 1;
    *flops_per_s = best;
    return 0;
}

}  // namespace

// Best of 5 timed launches, FLOP/s (an FMA counts 2). Returns 0 on success.
extern "C" int pfcp_fma_peak(int fp64, double *flops_per_s) {
    return fp64 ? probe<double>(flops_per_s) : probe<float>(flops_per_s);
}
