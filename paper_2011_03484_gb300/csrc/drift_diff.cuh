// drift_diff.cuh -- derivatives of the Kepler drift (tangent, adjoint and
// second-order tangent maps) for the differentiable map (diff.cu).
//
// With G_n(s, beta) = s^n c_n(beta s^2):  dG_n/ds = G_{n-1} (dG_0/ds = -beta G_1)
// and dG_n/dbeta = -(s G_{n+1} - n G_{n+2}) / 2 (from the series term by term).
// s solves T(s) = r0 G1 + u G2 + mu G3 = tau with tau = dt - k P(beta),
// P = 2 pi mu beta^(-3/2), so by implicit differentiation
//   ds = (dtau - G1 dr0 - G2 du - T_beta dbeta) / R,   R = T'(s),
//   T_beta = r0 G1_beta + u G2_beta + mu G3_beta,   dtau = 1.5 k P dbeta / beta,
// and r0 = |r|, u = r . v, beta = 2 mu / r0 - v . v.
//
// The tangent map and the G-function evaluation are templates over the scalar
// type.  With T = double they are the tangent map.  With T = ad::Dual (a value
// and its derivative along one direction of the state) the same code gives the
// derivative of the tangent map itself, d(M(x) t)/dx [dx] = M(x) dt +
// (dM(x)[dx]) t: the second-order term that the gradient of the tangent-growth
// indicator needs.
#pragma once
#include "kepler.cuh"

namespace glisse {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers: v + d eps with eps^2 = 0.  Overloads live in
// namespace ad and are found by argument-dependent lookup, so unqualified
// calls on doubles keep resolving to the plain functions.
// ---------------------------------------------------------------------------
namespace ad {
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator+(const Dual& a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, const Dual& b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(const Dual& a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, const Dual& b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator-(const Dual& a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
    return {a.v * b.v, ::fma(a.v, b.d, a.d * b.v)};
}
__device__ __forceinline__ Dual operator*(const Dual& a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, const Dual& b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) {
    const double q = a.v / b.v;
    return {q, ::fma(-q, b.d, a.d) / b.v};
}
__device__ __forceinline__ Dual operator/(const Dual& a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual fma(const Dual& a, const Dual& b, const Dual& c) {
    return {::fma(a.v, b.v, c.v), ::fma(a.v, b.d, ::fma(a.d, b.v, c.d))};
}
__device__ __forceinline__ Dual fma(double a, const Dual& b, const Dual& c) {
    return {::fma(a, b.v, c.v), ::fma(a, b.d, c.d)};
}
__device__ __forceinline__ Dual fma(const Dual& a, double b, const Dual& c) {
    return {::fma(a.v, b, c.v), ::fma(a.d, b, c.d)};
}
__device__ __forceinline__ Dual fma(const Dual& a, const Dual& b, double c) {
    return {::fma(a.v, b.v, c), ::fma(a.v, b.d, a.d * b.v)};
}
__device__ __forceinline__ Dual fma(const Dual& a, double b, double c) { return {::fma(a.v, b, c), a.d * b}; }
__device__ __forceinline__ Dual fma(double a, const Dual& b, double c) { return {::fma(a, b.v, c), a * b.d}; }
__device__ __forceinline__ Dual fma(double a, double b, const Dual& c) { return {::fma(a, b, c.v), c.d}; }
// The device arithmetic of device_math.cuh, lifted: d(x^-1/2) = -x^-3/2 dx / 2,
// d(1/x) = -dx / x^2, d(k x^-3/2) = -3/2 k x^-3/2 dx / x.
__device__ __forceinline__ Dual rsqrt_full(const Dual& x) {
    const double y = glisse::rsqrt_full(x.v);
    return {y, -0.5 * (y * (y * y)) * x.d};
}
__device__ __forceinline__ Dual rcp_full(const Dual& x) {
    const double y = glisse::rcp_full(x.v);
    return {y, -(y * y) * x.d};
}
__device__ __forceinline__ Dual rcp_40(const Dual& x) {
    const double y = glisse::rcp_40(x.v);
    return {y, -(y * y) * x.d};
}
__device__ __forceinline__ Dual k_rcube(const Dual& x, double k) {
    const double w = glisse::k_rcube(x.v, k);
    return {w, (-1.5 * w) * (x.d * glisse::rcp_full(x.v))};
}
}  // namespace ad
using ad::Dual;

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const Dual& x) { return x.v; }

// ---------------------------------------------------------------------------
// Stumpff functions for any scalar type.
// ---------------------------------------------------------------------------
// c2, c3 by their series, degree DEG.
template <int DEG, class T>
__device__ __forceinline__ void c23_series(const T& z, T& c2, T& c3) {
    constexpr double a[8] = {1.0 / 2.0, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0,
                             -1.0 / 479001600.0, 1.0 / 87178291200.0, -1.0 / 20922789888000.0};
    constexpr double b[8] = {1.0 / 6.0, -1.0 / 120.0, 1.0 / 5040.0, -1.0 / 362880.0, 1.0 / 39916800.0,
                             -1.0 / 6227020800.0, 1.0 / 1307674368000.0, -1.0 / 355687428096000.0};
    T p = fma(z, a[DEG], a[DEG - 1]), q = fma(z, b[DEG], b[DEG - 1]);
#pragma unroll
    for (int n = DEG - 2; n >= 0; --n) {
        p = fma(p, z, a[n]);
        q = fma(q, z, b[n]);
    }
    c2 = p;
    c3 = q;
}

// c4, c5 by their series, degree DEG.
template <int DEG, class T>
__device__ __forceinline__ void c45_series(const T& z, T& c4, T& c5) {
    constexpr double a[8] = {1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0, -1.0 / 3628800.0, 1.0 / 479001600.0,
                             -1.0 / 87178291200.0, 1.0 / 20922789888000.0, -1.0 / 6402373705728000.0};
    constexpr double b[8] = {1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0, 1.0 / 6227020800.0,
                             -1.0 / 1307674368000.0, 1.0 / 355687428096000.0, -1.0 / 121645100408832000.0};
    T p = fma(z, a[DEG], a[DEG - 1]), q = fma(z, b[DEG], b[DEG - 1]);
#pragma unroll
    for (int n = DEG - 2; n >= 0; --n) {
        p = fma(p, z, a[n]);
        q = fma(q, z, b[n]);
    }
    c4 = p;
    c5 = q;
}

// c0..c5 for any z: quarter z until |z| <= 0.1, series there, then the
// duplication formulas c0(4z) = 2 c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2 / 2,
// c3(4z) = (c3 + c1 c2) / 4; c4, c5 by series below |z| = 0.1, else
// c_{n+2} = (1/n! - c_n) / z.
template <class T>
__device__ inline void stumpff_all(const T& z0, T c[6]) {
    T z = z0;
    int k = 0;
    while (fabs(val(z)) > 0.1 && k < 80) {
        z = z * 0.25;
        ++k;
    }
    T c0, c1, c2, c3;
    c23_series<7>(z, c2, c3);
    c0 = fma(-z, c2, 1.0);
    c1 = fma(-z, c3, 1.0);
    for (; k > 0; --k) {
        const T n3 = 0.25 * fma(c1, c2, c3);
        const T n2 = 0.5 * (c1 * c1);
        const T n1 = c0 * c1;
        const T n0 = fma(2.0 * c0, c0, -1.0);
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    c[0] = c0;
    c[1] = c1;
    c[2] = c2;
    c[3] = c3;
    if (fabs(val(z0)) <= 0.1) {
        c45_series<7>(z0, c[4], c[5]);
    } else {
        c[4] = (0.5 - c[2]) / z0;
        c[5] = (1.0 / 6.0 - c[3]) / z0;
    }
}

// Where the derivative path evaluates the Stumpff series: |z| < kZSeries uses
// the series (degree 5: the first omitted terms of c2..c5 are below 3e-17
// relative at |z| = 0.1) and, below kZDeg3, degree 3 (below 1e-17 relative at
// |z| = 2e-3: ~1e-3 for the belts of 20-30 AU at dt = 0.5 yr).  The choice is
// made per lane from the lane's own z, so a recomputed step repeats it.
constexpr double kZSeries = 0.1;
constexpr double kZDeg3 = 2e-3;
__device__ __forceinline__ bool z_below(double z, double lim) { return lt_nonneg(fabs(z), lim); }

// G_0..G_3 from G_4, G_5 by the exact recurrence G_n = s^n / n! - beta G_{n+2}
// (c_n(z) = 1/n! - z c_{n+2}(z)); for |z| < 0.1 the correction beta G_{n+2} is
// at most a few percent of s^n / n!, so each G_n is good to an ulp or two.
template <class T>
__device__ __forceinline__ void g_from_g45(const T& s, const T& beta, T G[6]) {
    const T s2 = s * s;
    G[3] = fma(-beta, G[5], (s2 * s) * (1.0 / 6.0));
    G[2] = fma(-beta, G[4], 0.5 * s2);
    G[1] = fma(-beta, G[3], s);
    G[0] = fma(-beta, G[2], 1.0);
}

template <class T>
struct DriftScalarsT {
    T r0, u, beta, tau, dtau_dbeta, s;
    T G[6], Gb[4];  // G_0..G_5 and dG_n/dbeta, n = 0..3
    T R, f, g, fd, gd;
    T inv_r0, inv_R;    // 1/r0 and 1/R (MUFU seed + one correction: no divisions downstream)
    T mg2r, mg2R, irR;  // mu G2 / r0 (1 - f), mu G2 / R (1 - gd), 1 / (R r0), not rounded through 1 -
};
using DriftScalars = DriftScalarsT<double>;

// Drift scalars of one body at its current state, in two parts: drift_solve
// finds s (and tau, dtau/dbeta) and drift_finish evaluates the G-functions and
// f, g from them, so that a caller that stored s and tau can redo the second
// part alone.  drift_solve starts from the FP32 root of the fast path (five
// FP32 Newton steps, the last one within 2^-20 of s) and takes one FP64
// Halley step: from a start good to ~1e-7 the cubic step lands at rounding
// level.  Orbits outside the FP32 domain, or |z| > 0.1, use the general
// safeguarded solver.
__device__ inline bool drift_solve(double mu, double dt, const double st[6], DriftScalars& d) {
    const double x2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
    d.inv_r0 = rsqrt_full(x2);
    d.r0 = x2 * d.inv_r0;
    const double v2 = fma(st[3], st[3], fma(st[4], st[4], st[5] * st[5]));
    d.u = fma(st[0], st[3], fma(st[1], st[4], st[2] * st[5]));
    d.beta = fma(2.0 * mu, d.inv_r0, -v2);
    d.dtau_dbeta = 0.0;
    // FP32 start (the fast path's iteration), accepted only well inside its domain
    const int er = exp_bits(d.r0), ev = exp_bits(v2);
    bool ok = er > 1023 - 60 && er < 1023 + 60 && ev < 1023 + 120 && ev > 1023 - 200 && dt != 0.0;
    if (ok) {
        // FP32 copies by bit truncation (integer operations: no conversion on the FP64 pipe)
        const float r0f = d2f_bits(d.r0), uf = d2f_bits(d.u), bf = d2f_bits(d.beta), muf = d2f_bits(mu),
                    dtf = d2f_bits(dt);
        float sf = dtf / r0f, dsf = 0.f;
        for (int it = 0; it < 5; ++it) {
            const float zf = bf * sf * sf;
            const float c2 = fmaf(zf, fmaf(zf, fmaf(zf, -1.0f / 40320.0f, 1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
            const float c3 =
                fmaf(zf, fmaf(zf, fmaf(zf, -1.0f / 362880.0f, 1.0f / 5040.0f), -1.0f / 120.0f), 1.0f / 6.0f);
            const float G1 = sf * fmaf(-zf, c3, 1.0f), G2 = sf * sf * c2, G3 = sf * sf * sf * c3;
            const float F = fmaf(r0f, G1, fmaf(uf, G2, fmaf(muf, G3, -dtf)));
            const float Fp = fmaf(r0f, fmaf(-zf, c2, 1.0f), fmaf(uf, G1, muf * G2));
            dsf = -F / Fp;
            sf += dsf;
        }
        ok = isfinite(sf) && fabsf(dsf) <= 9.5367431640625e-7f * fabsf(sf) && fabsf(bf * sf * sf) <= 0.09f;
        if (ok) {
            double s = f2d_bits(sf);
            // one Halley step on F(s) = r0 G1 + u G2 + mu G3 - dt:
            // ds = -2 F F' / (2 F'^2 - F F''),  F' = r0 G0 + u G1 + mu G2,  F'' = u G0 + (mu - beta r0) G1
            double c2, c3;
            const double z = d.beta * s * s;
            if (z_below(z, kZDeg3))
                c23_poly<3>(z, c2, c3);
            else
                c23_poly<5>(z, c2, c3);
            const double s2 = s * s;
            const double G0 = fma(-z, c2, 1.0), G1 = s * fma(-z, c3, 1.0), G2 = s2 * c2, G3 = s2 * s * c3;
            const double F = fma(d.r0, G1, fma(d.u, G2, fma(mu, G3, -dt)));
            const double Fp = fma(d.r0, G0, fma(d.u, G1, mu * G2));
            const double Fpp = fma(d.u, G0, fma(-d.beta, d.r0, mu) * G1);
            const double den = fma(2.0 * Fp, Fp, -F * Fpp);
            s = fma(-2.0 * (F * Fp), rcp_full(den), s);
            ok = !nonfinite_bits(s) && z_below(d.beta * s * s, kZSeries);
            d.s = s;
            d.tau = dt;
        }
    }
    if (!ok) {
        double kper;
        if (!universal_solve(mu, dt, d.r0, d.u, d.beta, d.s, d.tau, kper)) return false;
        if (kper != 0.0) {
            const double period = 6.283185307179586476925286766559 * mu / (d.beta * sqrt(d.beta));
            d.dtau_dbeta = 1.5 * kper * period / d.beta;
        }
    }
    return true;
}

// Recover r0, u, beta and dtau/dbeta of a state whose s and tau were stored.
__device__ inline void drift_restore(double mu, double dt, const double st[6], double s, double tau,
                                     DriftScalars& d) {
    const double x2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
    d.inv_r0 = rsqrt_full(x2);
    d.r0 = x2 * d.inv_r0;
    const double v2 = fma(st[3], st[3], fma(st[4], st[4], st[5] * st[5]));
    d.u = fma(st[0], st[3], fma(st[1], st[4], st[2] * st[5]));
    d.beta = fma(2.0 * mu, d.inv_r0, -v2);
    d.s = s;
    d.tau = tau;
    d.dtau_dbeta = 0.0;
    if (tau != dt && d.beta > 0.0) {
        const double period = 6.283185307179586476925286766559 * mu / (d.beta * sqrt(d.beta));
        const double kper = rint((dt - tau) / period);
        d.dtau_dbeta = 1.5 * kper * period / d.beta;
    }
}

// True where G_0..G_3 come from G_4, G_5 by the recurrence (|z| < 0.1); the
// rest use the general Stumpff evaluation.
__device__ __forceinline__ bool g_small(const DriftScalars& d) { return z_below(d.beta * d.s * d.s, kZSeries); }

// G_0..G_5 at (s, beta).
template <class T>
__device__ inline void g_functions(DriftScalarsT<T>& d) {
    const T z = d.beta * d.s * d.s;
    if (z_below(val(z), kZSeries)) {
        T c4, c5;
        if (z_below(val(z), kZDeg3))
            c45_series<3>(z, c4, c5);
        else
            c45_series<5>(z, c4, c5);
        const T s2 = d.s * d.s;
        d.G[4] = (s2 * s2) * c4;
        d.G[5] = ((s2 * s2) * d.s) * c5;
        g_from_g45(d.s, d.beta, d.G);
    } else {
        T c[6];
        stumpff_all(z, c);
        d.G[0] = c[0];
        T sp = d.s;
        for (int n = 1; n < 6; ++n) {
            d.G[n] = sp * c[n];
            sp = sp * d.s;
        }
    }
}

// dG_n/dbeta = -(s G_{n+1} - n G_{n+2}) / 2 and f, g, fd, gd, given the G's and 1/R.
template <class T>
__device__ __forceinline__ void drift_fg(double mu, DriftScalarsT<T>& d) {
    const T hs = -0.5 * d.s;
    d.Gb[0] = hs * d.G[1];
    d.Gb[1] = fma(hs, d.G[2], 0.5 * d.G[3]);
    d.Gb[2] = fma(hs, d.G[3], d.G[4]);
    d.Gb[3] = fma(hs, d.G[4], 1.5 * d.G[5]);
    const T mg2 = mu * d.G[2];
    d.mg2r = mg2 * d.inv_r0;
    d.mg2R = mg2 * d.inv_R;
    d.irR = d.inv_R * d.inv_r0;
    d.f = fma(-mg2, d.inv_r0, 1.0);  // explicit: kernels that also use mg2r must round f alike
    d.g = fma(-mu, d.G[3], d.tau);
    d.fd = (-mu * d.G[1]) * d.irR;
    d.gd = fma(-mg2, d.inv_R, 1.0);
}

__device__ inline void drift_finish(double mu, DriftScalars& d) {
    g_functions(d);
    d.R = fma(d.r0, d.G[0], fma(d.u, d.G[1], mu * d.G[2]));
    d.inv_R = rcp_full(d.R);
    drift_fg(mu, d);
}

// drift_finish for a step whose G_4, G_5 and 1/R were stored by drift_finish:
// the same G's bit for bit (the recurrence where it applied, else the general
// evaluation again).  d.R is not set.
__device__ inline void drift_finish_stored(double mu, DriftScalars& d, double G4, double G5, double inv_R) {
    if (g_small(d)) {
        d.G[4] = G4;
        d.G[5] = G5;
        g_from_g45(d.s, d.beta, d.G);
    } else {
        g_functions(d);
    }
    d.inv_R = inv_R;
    drift_fg(mu, d);
}

// Drift scalars of one body at its current state.
__device__ inline bool drift_scalars(double mu, double dt, const double st[6], DriftScalars& d) {
    if (!drift_solve(mu, dt, st, d)) return false;
    drift_finish(mu, d);
    return true;
}

// The drift scalars as dual numbers along the state direction dx: the values
// are those of d (same arithmetic), the derivatives those of r0, u, beta (from
// their definitions), s (implicit differentiation, as in the tangent map),
// tau, and of everything computed from them.
__device__ inline DriftScalarsT<Dual> drift_lift(double mu, const double st[6], const double dx[6],
                                                 const DriftScalars& d) {
    DriftScalarsT<Dual> e;
    const double rdr = fma(st[0], dx[0], fma(st[1], dx[1], st[2] * dx[2]));
    const double dr0 = rdr * d.inv_r0;
    const double du = fma(dx[0], st[3], fma(dx[1], st[4], fma(dx[2], st[5], fma(st[0], dx[3], fma(st[1], dx[4],
                                                                                                   st[2] * dx[5])))));
    const double vdv = fma(st[3], dx[3], fma(st[4], dx[4], st[5] * dx[5]));
    const double dbeta = -2.0 * fma(mu * (d.inv_r0 * d.inv_r0), dr0, vdv);
    e.r0 = {d.r0, dr0};
    e.inv_r0 = {d.inv_r0, -dr0 * (d.inv_r0 * d.inv_r0)};
    e.u = {d.u, du};
    e.beta = {d.beta, dbeta};
    // tau = dt - k P(beta): dtau/dbeta = 1.5 k P / beta ~ beta^(-5/2)
    e.dtau_dbeta = {d.dtau_dbeta, d.dtau_dbeta != 0.0 ? -2.5 * d.dtau_dbeta * dbeta / d.beta : 0.0};
    e.tau = {d.tau, d.dtau_dbeta * dbeta};
    const double Tb = fma(d.r0, d.Gb[1], fma(d.u, d.Gb[2], mu * d.Gb[3]));
    const double ds = fma(-d.G[1], dr0, fma(-d.G[2], du, fma(-Tb, dbeta, e.tau.d))) * d.inv_R;
    e.s = {d.s, ds};
    g_functions(e);
    e.R = fma(e.r0, e.G[0], fma(e.u, e.G[1], mu * e.G[2]));
    e.inv_R = rcp_full(e.R);
    drift_fg(mu, e);
    return e;
}

// Tangent map of the drift: t <- M(st) t, with M from the scalars d at st.
template <class T>
__device__ inline void drift_tangent(double mu, const T st[6], const DriftScalarsT<T>& d, T t[6]) {
    const T *r = st, *v = st + 3;
    const T dr0 = fma(r[0], t[0], fma(r[1], t[1], r[2] * t[2])) * d.inv_r0;
    const T du = fma(t[0], v[0], fma(t[1], v[1], fma(t[2], v[2], fma(r[0], t[3], fma(r[1], t[4], r[2] * t[5])))));
    const T vtv = fma(v[0], t[3], fma(v[1], t[4], v[2] * t[5]));
    const T dbeta = -2.0 * fma(mu * (d.inv_r0 * d.inv_r0), dr0, vtv);
    const T dtau = d.dtau_dbeta * dbeta;
    const T Tb = fma(d.r0, d.Gb[1], fma(d.u, d.Gb[2], mu * d.Gb[3]));
    const T ds = fma(-d.G[1], dr0, fma(-d.G[2], du, fma(-Tb, dbeta, dtau))) * d.inv_R;
    const T dG0 = fma(-d.beta * d.G[1], ds, d.Gb[0] * dbeta);
    const T dG1 = fma(d.G[0], ds, d.Gb[1] * dbeta);
    const T dG2 = fma(d.G[1], ds, d.Gb[2] * dbeta);
    const T dG3 = fma(d.G[2], ds, d.Gb[3] * dbeta);
    // f = 1 - mu G2 / r0, g = tau - mu G3, fd = -mu G1 / (R r0), gd = 1 - mu G2 / R
    const T df = fma(d.mg2r, dr0, -mu * dG2) * d.inv_r0;
    const T dg = fma(-mu, dG3, dtau);
    const T dR = fma(dr0, d.G[0], fma(d.r0, dG0, fma(du, d.G[1], fma(d.u, dG1, mu * dG2))));
    const T dfd = fma(-mu * d.irR, dG1, -d.fd * fma(dR, d.inv_R, dr0 * d.inv_r0));
    const T dgd = fma(d.mg2R, dR, -mu * dG2) * d.inv_R;
    T o[6];
    for (int i = 0; i < 3; ++i) {
        o[i] = fma(df, r[i], fma(d.f, t[i], fma(dg, v[i], d.g * t[3 + i])));
        o[3 + i] = fma(dfd, r[i], fma(d.fd, t[i], fma(dgd, v[i], d.gd * t[3 + i])));
    }
    for (int i = 0; i < 6; ++i) t[i] = o[i];
}

// Adjoint of the drift: cotangent (lr1, lv1) at the end -> (lr, lv) at the start (in place).
// Reverse sweep through r1 = f r + g v, v1 = fd r + gd v with f = 1 - mu G2 / r0,
// g = tau - mu G3, fd = -mu G1 / (R r0), gd = 1 - mu G2 / R, R = r0 G0 + u G1 + mu G2,
// the G's through s(tau, r0, u, beta) (implicit differentiation) and beta, then
// r0 = |r|, u = r . v, beta = 2 mu / r0 - v . v.  Every accumulator starts from
// its first term (an add to 0.0 is not free under IEEE rules).
// With T = ad::Dual, the state carrying a tangent t as its derivative and the
// cotangent (lt, lx) as (value, derivative), the result is (M^T lt,
// (dM[t])^T lt + M^T lx): one reverse step of the map extended by its tangent
// (the second derivative of the map is symmetric, so d(M t)/dx^T lt = (dM[t])^T lt).
template <class T>
__device__ inline void drift_adjoint(double mu, const T st[6], const DriftScalarsT<T>& d, T l[6]) {
    const T *r = st, *v = st + 3;
    const T lf = fma(l[0], r[0], fma(l[1], r[1], l[2] * r[2]));
    const T lg = fma(l[0], v[0], fma(l[1], v[1], l[2] * v[2]));
    const T lfd = fma(l[3], r[0], fma(l[4], r[1], l[5] * r[2]));
    const T lgd = fma(l[3], v[0], fma(l[4], v[1], l[5] * v[2]));
    T lr[3], lv[3];
    for (int i = 0; i < 3; ++i) {
        lr[i] = fma(d.f, l[i], d.fd * l[3 + i]);
        lv[i] = fma(d.g, l[i], d.gd * l[3 + i]);
    }
    // through f, g, fd, gd
    const T a = lf * d.inv_r0;
    const T e = d.fd * lfd;
    T lG2 = -mu * fma(lgd, d.inv_R, a);
    const T lG3 = -mu * lg;
    T lG1 = (-mu * d.irR) * lfd;
    const T lR = d.inv_R * fma(d.mg2R, lgd, -e);
    T lr0 = fma(d.mg2r, a, -e * d.inv_r0);
    // through R
    lr0 = fma(d.G[0], lR, lr0);
    const T lG0 = d.r0 * lR;
    T lu = d.G[1] * lR;
    lG1 = fma(d.u, lR, lG1);
    lG2 = fma(mu, lR, lG2);
    // through the G's: s and beta
    const T ls = fma(-d.beta * d.G[1], lG0, fma(d.G[0], lG1, fma(d.G[1], lG2, d.G[2] * lG3)));
    T lbeta = fma(d.Gb[0], lG0, fma(d.Gb[1], lG1, fma(d.Gb[2], lG2, d.Gb[3] * lG3)));
    // s(tau, r0, u, beta): ds = (dtau - G1 dr0 - G2 du - Tb dbeta) / R
    const T Tb = fma(d.r0, d.Gb[1], fma(d.u, d.Gb[2], mu * d.Gb[3]));
    const T lsR = ls * d.inv_R;
    const T ltau = fma(ls, d.inv_R, lg);
    lr0 = fma(-d.G[1], lsR, lr0);
    lu = fma(-d.G[2], lsR, lu);
    lbeta = fma(-Tb, lsR, lbeta);
    lbeta = fma(d.dtau_dbeta, ltau, lbeta);
    // beta = 2 mu / r0 - v . v
    const T tb = 2.0 * lbeta;
    lr0 = fma(-tb, mu * (d.inv_r0 * d.inv_r0), lr0);
    // u = r . v ; r0 = |r|
    const T c = lr0 * d.inv_r0;
    for (int i = 0; i < 3; ++i) {
        l[i] = fma(lu, v[i], fma(c, r[i], lr[i]));
        l[3 + i] = fma(lu, r[i], fma(-tb, v[i], lv[i]));
    }
}

}  // namespace glisse
