// selftest.cu -- test hooks, not used by the map itself: elementwise
// evaluation of the device arithmetic helpers (device_math.cuh) on device
// arrays, so that tests can check each one against exact arithmetic; and a
// run of each task launch whose bounded wait is made to run out.
#include <cuda_runtime.h>

#include "device_math.cuh"
#include "glisse_internal.h"

namespace glisse {
cudaError_t particle_wait_selftest(int polls, char* scratch, int* status, cudaStream_t s);
cudaError_t diff_wait_selftest(int which, int polls, char* scratch, int* status, cudaStream_t s);

namespace {

__global__ void math_kernel(int fn, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i], k = b ? b[i] : 1.0;
    double r = 0.0;
    switch (fn) {
        case GLISSE_MATH_RSQRT: r = rsqrt_full(x); break;
        case GLISSE_MATH_RCP: r = rcp_full(x); break;
        case GLISSE_MATH_RCP40: r = rcp_40(x); break;
        case GLISSE_MATH_KRCUBE: r = k_rcube(x, k); break;
        case GLISSE_MATH_FLOAT_SQUARE: {
            double s2, s3;
            r = float_powers(d2f_bits(x), s2, s3) ? s2 : __longlong_as_double(0x7FF8000000000000ll);
            break;
        }
        case GLISSE_MATH_FLOAT_CUBE: {
            double s2, s3;
            r = float_powers(d2f_bits(x), s2, s3) ? s3 : __longlong_as_double(0x7FF8000000000000ll);
            break;
        }
        case GLISSE_MATH_D2F: r = (double)d2f_bits(x); break;
        default: r = __longlong_as_double(0x7FF8000000000000ll); break;
    }
    out[i] = r;
}

}  // namespace
}  // namespace glisse

using namespace glisse;

extern "C" int glisse_selftest_math(int32_t fn, const double* a, const double* b, double* out, int64_t n,
                                    void* stream) {
    if (n < 0 || fn < GLISSE_MATH_RSQRT || fn > GLISSE_MATH_D2F) return GLISSE_E_INVAL;
    if (n == 0) return GLISSE_OK;
    if (!a || !out) return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    math_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fn, a, b, out, n);
    if (cudaGetLastError() != cudaSuccess) return GLISSE_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GLISSE_E_CUDA;
    return GLISSE_OK;
}

extern "C" int glisse_selftest_wait(int32_t which, int32_t polls, int32_t* status, void* stream) {
    if (which < GLISSE_WAIT_PARTICLE_TASKS || which > GLISSE_WAIT_DIFF_BACKWARD || polls < 1 || !status)
        return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // task counter (8 bytes), the two groups' counters (8), then the status word
    constexpr size_t kBytes = 64;
    char* buf = nullptr;
    if (cudaMalloc(&buf, kBytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    int* d_status = reinterpret_cast<int*>(buf + 32);
    cudaError_t e = cudaMemsetAsync(buf, 0, kBytes, s);
    if (e == cudaSuccess)
        e = which == GLISSE_WAIT_PARTICLE_TASKS ? particle_wait_selftest(polls, buf, d_status, s)
                                                : diff_wait_selftest(which, polls, buf, d_status, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    *status = h;
    return GLISSE_OK;
}
