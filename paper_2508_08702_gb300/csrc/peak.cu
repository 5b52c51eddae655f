// peak.cu -- FP64 fused multiply-add throughput of this GPU, the measured
// denominator of the enumeration kernel's roofline.  Every thread runs
// eight independent dependency chains of fmas, so that the FP64 pipe, not
// latency, limits the rate; the result is written out so nothing is dead.
#include <cuda_runtime.h>

namespace msp {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 12345.678) out[0] = s;   // practically never taken; keeps the chains live
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

cudaError_t fp64_peak(double* dfma_per_s, int sms, cudaStream_t st) {
    double* out = nullptr;
    cudaError_t e = cudaMalloc(&out, 2 * sizeof(double));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_kernel, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    const int iters = 4096;
    fp64_fma_kernel<<<blocks, 256, 0, st>>>(out, 64, 0.999, 1e-3);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        fp64_fma_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999, 1e-3);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    *dfma_per_s = (double)blocks * 256.0 * iters * kChains / (best * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace msp
