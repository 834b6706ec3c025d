// sampling.cu -- osculating elements and resonance libration flags of the live
// particles at one sample step (section 3: elements logged at a fixed
// interval; a particle librates in the p:q resonance with a planet when
//   phi = p lambda - q lambda_N - (p - q) varpi
// never comes within a window (10 degrees) of 0, or never within it of 180
// degrees, over the samples; lambda = varpi + M, varpi = Omega + omega).
//
// Frames: heliocentric (mu = G m0 for particles, G (m0 + m_j) for planet j)
// or barycentric (positions and velocities relative to the barycentre of star
// and planets, mu = G (m0 + sum m_j) for every body).  Angles in [0, 2 pi);
// e = 0 puts the pericentre at the node, i = 0 the node on the x axis;
// hyperbolic orbits report M = e sinh F - F unwrapped and do not enter the
// libration test.  Runs once per sample (every thousands of steps), so it
// uses the library's FP64 functions; it is not on the per-step path.
#include <algorithm>
#include <cmath>

#include "glisse_internal.h"

namespace glisse {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.1415926535897932384626433832795;
constexpr int kSampleBlock = 128;

__device__ double wrap_angle(double x) {
    double y = fmod(x, kTwoPi);
    return y < 0.0 ? y + kTwoPi : y;
}

// Osculating elements a, e, i, Omega, omega, M of the two-body orbit about mu.
__device__ bool osculating(double mu, const double s[6], double el[6]) {
    const double r = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    const double v2 = s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
    // specific angular momentum and its projection on the reference plane
    const double h[3] = {s[1] * s[5] - s[2] * s[4], s[2] * s[3] - s[0] * s[5], s[0] * s[4] - s[1] * s[3]};
    const double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (!(r > 0.0) || !(hn > 0.0) || !(mu > 0.0)) return false;
    const double hp = sqrt(h[0] * h[0] + h[1] * h[1]);
    // Laplace-Runge-Lenz direction: e = (v x h) / mu - r / |r|
    double ev[3];
    const double vxh[3] = {s[4] * h[2] - s[5] * h[1], s[5] * h[0] - s[3] * h[2], s[3] * h[1] - s[4] * h[0]};
    for (int d = 0; d < 3; ++d) ev[d] = vxh[d] / mu - s[d] / r;
    const double e = sqrt(ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2]);
    const double a = 1.0 / (2.0 / r - v2 / mu);
    const double inc = atan2(hp, h[2]);
    const double node = hp > 0.0 ? atan2(h[0], -h[1]) : 0.0;
    // unit vectors in the orbital plane: p along the node line, q = h_hat x p
    const double cn = cos(node), sn = sin(node);
    const double q[3] = {-h[2] * sn / hn, h[2] * cn / hn, (h[0] * sn - h[1] * cn) / hn};
    const double lat = atan2(s[0] * q[0] + s[1] * q[1] + s[2] * q[2], s[0] * cn + s[1] * sn);
    const double peri = e > 0.0 ? atan2(ev[0] * q[0] + ev[1] * q[1] + ev[2] * q[2], ev[0] * cn + ev[1] * sn) : 0.0;
    const double f = lat - peri;
    double M;
    if (e < 1.0) {
        const double E = atan2(sqrt((1.0 - e) * (1.0 + e)) * sin(f), e + cos(f));
        M = wrap_angle(E - e * sin(E));
    } else if (e > 1.0) {
        const double F = 2.0 * atanh(sqrt((e - 1.0) / (e + 1.0)) * tan(0.5 * f));
        M = e * sinh(F) - F;
    } else {
        const double D = tan(0.5 * f);
        M = D + D * D * D / 3.0;
    }
    el[0] = a;
    el[1] = e;
    el[2] = inc;
    el[3] = wrap_angle(node);
    el[4] = wrap_angle(peri);
    el[5] = M;
    return true;
}

__global__ void __launch_bounds__(kSampleBlock) sample_kernel(const SampleArgs a) {
    // frame offset, particle mu and the planet's mean longitude: the same for every thread
    __shared__ double s_off[6];
    __shared__ double s_mu, s_lam;
    __shared__ int s_resok;
    if (threadIdx.x == 0) {
        const PlanetConsts& pc = *a.pc;
        double mt = pc.m0;
        for (int j = 0; j < pc.np; ++j) mt += pc.m[j];
        for (int d = 0; d < 6; ++d) {
            double acc = 0.0;
            if (a.frame == GLISSE_FRAME_BARY)
                for (int j = 0; j < pc.np; ++j) acc += pc.m[j] * a.planets[6 * j + d];
            s_off[d] = acc / mt;
        }
        s_mu = pc.G * (a.frame == GLISSE_FRAME_BARY ? mt : pc.m0);
        s_resok = 0;
        s_lam = 0.0;
        if (a.res_planet >= 0) {
            double sp[6], el[6];
            for (int d = 0; d < 6; ++d) sp[d] = a.planets[6 * a.res_planet + d] - s_off[d];
            const double mup = a.frame == GLISSE_FRAME_BARY ? s_mu : pc.G * (pc.m0 + pc.m[a.res_planet]);
            if (osculating(mup, sp, el) && el[1] < 1.0) {
                s_lam = el[3] + el[4] + el[5];
                s_resok = 1;
            }
        }
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!a.alive[i]) continue;
        const int64_t pid = a.id[i];
        double s[6], el[6];
        for (int d = 0; d < 6; ++d) s[d] = a.sync[6 * pid + d] - s_off[d];
        const bool ok = osculating(s_mu, s, el);
        if (a.elem) {
            double* o = a.elem + 6 * pid;
            for (int d = 0; d < 6; ++d) o[d] = ok ? el[d] : __longlong_as_double(0x7FF8000000000000ll);
        }
        if (a.res_planet >= 0 && s_resok && ok && el[1] < 1.0) {
            const double varpi = el[3] + el[4];
            const double lam = varpi + el[5];
            const double phi = wrap_angle(a.res_p * lam - a.res_q * s_lam - (a.res_p - a.res_q) * varpi);
            const double d0 = fmin(phi, kTwoPi - phi);
            const double d180 = fabs(phi - kPi);
            if (d0 < a.avoid) a.near0[pid] = 1;
            if (d180 < a.avoid) a.near180[pid] = 1;
            a.count[pid] += 1;
        }
    }
}

}  // namespace

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((a.n + kSampleBlock - 1) / kSampleBlock, 152 * 16);
    sample_kernel<<<(unsigned)blocks, kSampleBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace glisse
