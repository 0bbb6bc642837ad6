// probe.cu -- pipe-throughput microbenchmark (include/lisa_probe.h): independent FMA or
// MUFU chains per thread on every SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/lisa_probe.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void fma_chains(T *out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x * 1e-3 + k);
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int r = 0; r < 8; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = x[k] * a + b;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void mufu_chains(float *out, int iters) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int r = 0; r < 8; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = __sinf(x[k]);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" lisa_status lisa_probe_pipes(int device, double *out) {
    if (!out) return LISA_ERR_ARG;
    int nsm = 0, clk_khz = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
    if (e != cudaSuccess) return LISA_ERR_CUDA;
    const int threads = 256, blocks = nsm * 8;
    const size_t n = (size_t)threads * blocks;
    double *od = nullptr;
    float *of = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    float ms[3] = {0.0f, 0.0f, 0.0f};
    const int it[3] = {64, 2048, 512};
    if ((e = cudaMalloc(&od, n * sizeof(double))) == cudaSuccess &&
        (e = cudaMalloc(&of, n * sizeof(float))) == cudaSuccess &&
        (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) == cudaSuccess) {
        for (int k = 0; k < 3 && e == cudaSuccess; k++) {
            for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // warm-up, then timed
                const int iters = rep == 0 ? 2 : it[k];
                cudaEventRecord(e0, s);
                if (k == 0) fma_chains<double><<<blocks, threads, 0, s>>>(od, iters, 1.0000001, 1e-9);
                if (k == 1) fma_chains<float><<<blocks, threads, 0, s>>>(of, iters, 1.0000001f, 1e-9f);
                if (k == 2) mufu_chains<<<blocks, threads, 0, s>>>(of, iters);
                cudaEventRecord(e1, s);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess && rep == 1) e = cudaEventElapsedTime(&ms[k], e0, e1);
            }
        }
    }
    if (od) cudaFree(od);
    if (of) cudaFree(of);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return LISA_ERR_CUDA;
    for (int k = 0; k < 3; k++) out[k] = (double)n * it[k] * 8 * kChains / (ms[k] * 1e-3);
    out[3] = clk_khz * 1e3;
    return LISA_OK;
}
