// fp64_peak.cu -- measured FP64 fused-multiply-add throughput of the GPU.
//
// The particle map is bound by the FP64 pipe, so its roofline is the rate at
// which this GPU retires DFMA instructions.  Each thread runs eight independent
// FMA chains (enough to cover the pipe latency); the launch covers every SM
// with two 256-thread blocks.  clock64() brackets give the SM clock the kernel
// actually ran at.
#include <cuda_runtime.h>

#include "glisse_internal.h"

namespace glisse {

__global__ void __launch_bounds__(256) dfma_chain_kernel(double* out, long long* cycles, int iters, double a,
                                                           double b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.0 + 1e-3 * (double)((t + j) & 1023);
    const long long c0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    const long long c1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[t] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

}  // namespace glisse

extern "C" int glisse_fp64_peak(int32_t iterations, double* dfma_per_s, double* sm_mhz) {
    using namespace glisse;
    if (iterations <= 0) return GLISSE_E_INVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLISSE_E_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GLISSE_E_CUDA;
    const int blocks = 2 * nsm, threads = 256;
    double* out = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GLISSE_OK;
    float ms = 0.f;
    long long* hc = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
        rc = GLISSE_E_NOMEM;
        goto done;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = GLISSE_E_CUDA;
        goto done;
    }
    dfma_chain_kernel<<<blocks, threads>>>(out, cyc, 8, 0.999999, 1e-6);  // warm-up
    cudaEventRecord(e0);
    dfma_chain_kernel<<<blocks, threads>>>(out, cyc, iterations, 0.999999, 1e-6);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = GLISSE_E_CUDA;
        goto done;
    }
    hc = new long long[blocks];
    if (cudaMemcpy(hc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = GLISSE_E_CUDA;
        goto done;
    }
    {
        double mean = 0.0;
        for (int b = 0; b < blocks; ++b) mean += (double)hc[b];
        mean /= blocks;
        const double ops = (double)blocks * threads * (double)iterations * 8.0;
        if (dfma_per_s) *dfma_per_s = ops / (ms * 1e-3);
        if (sm_mhz) *sm_mhz = mean / (ms * 1e3);
    }
done:
    delete[] hc;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    return rc;
}
