// sph_probe.cu -- measured FP32 FMA throughput (the ALU roofline of the pair passes).
#include <cuda_runtime.h>

#include "sph.h"

namespace {

constexpr int PROBE_BLOCK = 256;
constexpr int PROBE_CHAINS = 8;  // independent FMA chains per thread: hides the FMA latency

// Every thread runs PROBE_CHAINS independent recurrences a = a * b + c (one
// FP32 fused multiply-add each, 2 flops).  b and c are kernel arguments so
// that nothing folds; with 0 < b < 1 the values stay bounded.  The store
// behind an impossible comparison keeps the chains live.
__global__ void __launch_bounds__(PROBE_BLOCK) k_fma_probe(float* out, int iters, float b, float c) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" sph_status sph_fma_peak(void* stream, int reps, double* tflops, double* ms) {
    if (!tflops || reps < 1) return SPH_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, PROBE_BLOCK, 0) != cudaSuccess ||
        sms < 1 || per_sm < 1)
        return SPH_ECUDA;
    const int grid = sms * per_sm;  // one full wave of resident blocks
    const int iters = 4096;         // x 16 x PROBE_CHAINS FMAs per thread
    float* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * PROBE_BLOCK * sizeof(float)) != cudaSuccess) return SPH_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 0.f;
    if (err == cudaSuccess) {
        k_fma_probe<<<grid, PROBE_BLOCK, 0, s>>>(out, iters, 0.9999f, 1e-4f);  // warm-up
        err = cudaGetLastError();
    }
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        k_fma_probe<<<grid, PROBE_BLOCK, 0, s>>>(out, iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float t = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
        if (err == cudaSuccess && t > 0.f && (best == 0.f || t < best)) best = t;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || best <= 0.f) return SPH_ECUDA;
    const double flops = 2.0 * (double)grid * PROBE_BLOCK * iters * 16.0 * PROBE_CHAINS;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return SPH_OK;
}
