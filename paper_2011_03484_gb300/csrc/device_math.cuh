// device_math.cuh -- FP64 building blocks that keep work off the FP64 pipe.
//
// On GB300 the FP64 pipe retires about 1.7 DFMA per clock per SM while the
// FP32, integer and MUFU pipes run tens of times faster alongside it.  Every
// double-precision conversion (F2F) and comparison (DSETP) also occupies the
// FP64 pipe.  These helpers therefore
//   - take reciprocal / reciprocal-square-root seeds from the MUFU unit
//     (rcp.approx.ftz.f64, rsqrt.approx.ftz.f64: about 2^-20 relative error,
//     the low 32 bits of the result are zero) and finish them with one
//     polynomial correction in FP64;
//   - move values between double and float with integer bit operations;
//   - compare non-negative doubles as 64-bit integers.
#pragma once
#include <cstdint>

namespace glisse {

__device__ __forceinline__ double rsqrt_seed(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

__device__ __forceinline__ double rcp_seed(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/sqrt(x) for normal x > 0 to within a fraction of an ulp.
// With y = seed and e = 1 - x y^2 (|e| < 2^-19, computed exactly by one FMA
// since y^2 is exact):
//   x^(-1/2) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + O(e^3)).
// The e^2 term is below 2^-39 relative, so it is formed in FP32.
// 4 FP64 instructions.
__device__ __forceinline__ double rsqrt_full(double x);

// k * x^(-3/2) for normal x > 0 (the inverse-cube distance factor of a kick).
// y = seed (20 significant bits, so y*y is exact), e = 1 - x y^2:
//   x^(-3/2) = y^3 (1 - e)^(-3/2) = y^3 (1 + 3e/2 + 15e^2/8 + O(e^3)).
// 6 FP64 instructions.
__device__ __forceinline__ double k_rcube(double x, double k);

// 1/x to about 2^-40 from the MUFU seed and one Newton step (2 FP64 instructions).
__device__ __forceinline__ double rcp_40(double x) {
    double y = rcp_seed(x);
    double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// Refine an approximation y of 1/x by one Newton step: relative error e -> e^2.
__device__ __forceinline__ double rcp_refine(double x, double y) {
    double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// double -> float by truncating the significand, using integer operations only.
// Exact exponent mapping for |x| in the float normal range; values below it
// become signed zero, values above it (and inf / NaN) become signed infinity.
__device__ __forceinline__ float d2f_bits(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int e = ((hi >> 20) & 0x7FF) - 1023 + 127;
    const unsigned mant = (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
    unsigned bits = sign | ((unsigned)e << 23) | mant;
    bits = (e <= 0) ? sign : bits;
    bits = (e >= 255) ? (sign | 0x7F800000u) : bits;
    return __uint_as_float(bits);
}

// float -> double exactly, using integer operations only (normal floats and zero).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned m = b & 0x7FFFFFu;
    unsigned hi = sign | ((e + (1023u - 127u)) << 20) | (m >> 3);
    unsigned lo = m << 29;
    hi = (e == 0u) ? sign : hi;
    lo = (e == 0u) ? 0u : lo;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double rsqrt_full(double x) {
    const double y = rsqrt_seed(x);
    const double y2 = y * y;
    const double e = fma(-x, y2, 1.0);
    const float ef = d2f_bits(e);
    const double c = fma(0.5, e, f2d_bits(0.375f * ef * ef));
    return fma(y, c, y);
}

__device__ __forceinline__ double k_rcube(double x, double k) {
    const double y = rsqrt_seed(x);
    const double y2 = y * y;
    const double e = fma(-x, y2, 1.0);
    const double w = (y2 * y) * k;
    const float ef = d2f_bits(e);
    const double c = fma(1.5, e, f2d_bits(1.875f * ef * ef));
    return fma(w, c, w);
}

// 1/x to full precision from the MUFU seed: e = 1 - x y (|e| < 2^-19),
// 1/x = y (1 + e + e^2 + O(e^3)); e^2 in FP32.  3 FP64 instructions.
__device__ __forceinline__ double rcp_full(double x) {
    const double y = rcp_seed(x);
    const double e = fma(-x, y, 1.0);
    const float ef = d2f_bits(e);
    const double c = e + f2d_bits(ef * ef);
    return fma(y, c, y);
}

// a < b for non-negative doubles (including +0 and +inf) as a 64-bit integer compare.
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}

// True when x is +-inf or NaN (exponent field all ones), integer test.
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return (__double2hiint(x) & 0x7FF00000) == 0x7FF00000;
}

// Biased exponent of |x| (0 for zero / subnormal), integer test.
__device__ __forceinline__ int exp_bits(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// Multiply by 2^k (k small, result normal) by adjusting the exponent field: no FP64 instruction.
__device__ __forceinline__ double ldexp_bits(double x, int k) {
    return __hiloint2double(__double2hiint(x) + (k << 20), __double2loint(x));
}

}  // namespace glisse
