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
// The e^2 term is below 2^-39 relative, so it is formed in FP32; y^2 comes
// from integer arithmetic (seed_square).  3 FP64 instructions.
__device__ __forceinline__ double rsqrt_full(double x);

// k * x^(-3/2) for normal x > 0 (the inverse-cube distance factor of a kick).
// y = seed, e = 1 - x y^2:
//   x^(-3/2) = y^3 (1 - e)^(-3/2) = y^3 (1 + 3e/2 + 15e^2/8 + O(e^3)).
// y^2 (exact) and k y^3 (correctly rounded) come from integer arithmetic on
// the seed's 21-bit significand and k's 53-bit one (seed_square_kcube), so 3
// FP64 instructions remain.
__device__ __forceinline__ double k_rcube(double x, double k);

// 1/x to about 2^-40 from the MUFU seed and one Newton step (2 FP64 instructions).
__device__ __forceinline__ double rcp_40(double x) {
    double y = rcp_seed(x);
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

// t^2 exactly for t with at most 21 significant bits (the low 32 bits of its
// encoding zero, as the MUFU seeds are), by an integer square of the
// significand (42 bits).  Valid for |t| in [2^-511, 2^511]; NaN outside.
__device__ __forceinline__ double seed_square(double t) {
    const int hi = __double2hiint(t);
    const int et = (hi >> 20) & 0x7FF;
    const unsigned m = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
    const unsigned long long m2 = (unsigned long long)m * m;  // [2^40, 2^42)
    const int a = (int)(m2 >> 41);
    const double t2 = __longlong_as_double(((long long)(2 * et - 1024 + a) << 52) + (long long)(m2 << (12 - a)));
    return (unsigned)(et - 512) <= 1022u ? t2 : __longlong_as_double(0x7FF8000000000000ll);
}

// For t with at most 21 significant bits (the low 32 bits of its encoding
// zero, as the MUFU seeds are) and k >= 0: t^2
// exactly and k t^3 correctly rounded (ties away from zero) by integer
// arithmetic.  The 53-bit significand of k times m^3 (63 bits, exact) is a
// 116-bit product; its top 64 bits come from one 64 x 64 high multiply
// (the low bits can only matter for an exact tie) and are rounded to 53.
// k = 0 (or subnormal) gives 0.  Returns false (kt3 unspecified) when t is
// outside [2^-300, 2^300] or not normal, k is not finite, or k t^3 leaves
// the normal range.
__device__ __forceinline__ bool seed_square_kcube(double t, double k, double& t2, double& kt3) {
    const int hi = __double2hiint(t);
    const int et = (hi >> 20) & 0x7FF;  // t = m 2^(et - 1043)
    const unsigned m = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
    const unsigned long long m2 = (unsigned long long)m * m;  // [2^40, 2^42)
    const unsigned long long m3 = m2 * m;                     // [2^60, 2^63)
    const int a = (int)(m2 >> 41);
    t2 = __longlong_as_double(((long long)(2 * et - 1024 + a) << 52) + (long long)(m2 << (12 - a)));
    const long long kb = __double_as_longlong(k);
    const int ek = (int)((kb >> 52) & 0x7FF);  // k = km 2^(ek - 1075)
    const unsigned long long km = ((unsigned long long)kb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long p = __umul64hi(km << 11, m3 << 1);  // floor(km m3 / 2^52) in [2^60, 2^64)
    const int sh = 11 - __clzll(p);                               // leading bit at 52 + sh
    const unsigned long long q = ((p >> (sh - 1)) + 1) >> 1;      // 53 bits, rounded
    const int be = sh + ek + 3 * et - 3077;                       // biased exponent of k t^3
    kt3 = (ek == 0) ? 0.0 : __longlong_as_double(((long long)(be - 1) << 52) + (long long)q);
    return (unsigned)(et - 723) <= 600u && ek != 0x7FF && (ek == 0 || (unsigned)(be - 1) < 2045u);
}

// |s|^2 exactly and s^3 correctly rounded (ties away from zero) for a float s,
// as doubles, by integer multiplication of the 24-bit significand m: m^2 has
// 48 bits, m^3 = 2^32 H + L is formed from two 32 x 32 products and rounded
// to 53 bits.  Returns false (results unspecified) when s is zero,
// subnormal or non-finite.
__device__ __forceinline__ bool float_powers(float s, double& s2, double& s3) {
    const unsigned bits = __float_as_uint(s);
    const int ef = (int)((bits >> 23) & 0xFFu);  // s = m 2^(ef - 150)
    const unsigned m = (bits & 0x7FFFFFu) | 0x800000u;
    const unsigned long long m2 = (unsigned long long)m * m;  // [2^46, 2^48)
    // s^2 = m2 2^(2 ef - 300): leading bit of m2 at 46 + a, significand
    // m2 << (6 - a) in [2^52, 2^53), biased exponent 2 ef + 769 + a
    const int a = (int)(m2 >> 47);
    const long long e2 = (long long)(2 * ef + 768 + a) << 52;
    s2 = __longlong_as_double(e2 + (long long)(m2 << (6 - a)));
    // m^3 = m2 m = 2^32 H + L with H = m2_hi m + (m2_lo m >> 32) in [2^37, 2^40)
    const unsigned long long p1 = (unsigned long long)(unsigned)m2 * m;
    const unsigned long long H0 = (unsigned long long)(unsigned)(m2 >> 32) * m + (p1 >> 32);
    const int b = min((int)(H0 >> 38), 2);  // leading bit of m^3 at 69 + b
    const int sh = 17 + b;                  // keep 53 bits
    const unsigned long long L = (p1 & 0xFFFFFFFFull) + (1ull << (sh - 1));
    const unsigned long long H = H0 + (L >> 32);
    const unsigned long long q3 = (H << (32 - sh)) | ((L & 0xFFFFFFFFull) >> sh);  // [2^52, 2^53]
    const long long e3 = (long long)(3 * ef + 641 + b) << 52;
    const long long sign = (long long)(bits & 0x80000000u) << 32;
    s3 = __longlong_as_double((e3 + (long long)q3) | sign);
    return (unsigned)(ef - 1) < 254u;
}

__device__ __forceinline__ double rsqrt_full(double x) {
    const double y = rsqrt_seed(x);
    const double y2 = seed_square(y);
    const double e = fma(-x, y2, 1.0);
    const float ef = d2f_bits(e);
    const double c = fma(0.5, e, f2d_bits(0.375f * ef * ef));
    return fma(y, c, y);
}

__device__ __forceinline__ double k_rcube(double x, double k) {
    const double y = rsqrt_seed(x);
    double y2, ky3;
    const bool ok = seed_square_kcube(y, k, y2, ky3);
    const double e = fma(-x, y2, 1.0);
    const double w = ok ? ky3 : __longlong_as_double(0x7FF8000000000000ll);
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
