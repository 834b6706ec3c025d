// kepler.cuh -- Kepler drift of one body for time dt about a central mass (FP64).
//
// Section 2.2 of the paper advances each particle along its two-body orbit
// by solving Kepler's equation for the change of mean anomaly.  Here the
// drift is written in universal variables (Stumpff / Danby G-functions),
// which covers bound, parabolic and hyperbolic orbits with one formula:
//
//   G_k(s) = s^k c_k(beta s^2),  beta = 2 mu / r0 - v0^2,  c_k(z) = sum_n (-z)^n / (2n+k)!
//   time equation  T(s) = r0 G1 + u G2 + mu G3 = dt,   u = r0 . v0
//   T'(s) = r(s) = r0 G0 + u G1 + mu G2,   T''(s) = u G0 + (mu - beta r0) G1
//   f - 1 = -mu G2 / r0,  g = dt - mu G3,  fdot = -mu G1 / (r r0),  gdot - 1 = -mu G2 / r
//
// drift_fast is the hot path.  It solves T(s) = dt in FP32 first (the FP32
// pipe is nearly free next to the FP64 pipe), takes one FP64 Halley step from
// that start (cubic convergence: a 1e-7 start lands below 1e-20), evaluates
// c2, c3 with a polynomial whose degree the warp picks from its largest |z|,
// and moves the G-functions to the corrected s with their addition formulas
// instead of re-evaluating them.  Lanes outside its domain report false and
// the caller runs drift_general for them only (the rest of the warp idles).
#pragma once
#include "device_math.cuh"

namespace glisse {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Stumpff c2, c3 as truncated Taylor polynomials in z (Horner form).
// Coefficients 1/(2n+2)! and 1/(2n+3)! with alternating signs.
// ---------------------------------------------------------------------------
template <int DEG>
__device__ __forceinline__ void c23_poly(double z, double& c2, double& c3) {
    constexpr double a[8] = {1.0 / 2.0, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0,
                             -1.0 / 479001600.0, 1.0 / 87178291200.0, -1.0 / 20922789888000.0};
    constexpr double b[8] = {1.0 / 6.0, -1.0 / 120.0, 1.0 / 5040.0, -1.0 / 362880.0, 1.0 / 39916800.0,
                             -1.0 / 6227020800.0, 1.0 / 1307674368000.0, -1.0 / 355687428096000.0};
    double p = a[DEG], q = b[DEG];
#pragma unroll
    for (int n = DEG - 1; n >= 0; --n) {
        p = fma(p, z, a[n]);
        q = fma(q, z, b[n]);
    }
    c2 = p;
    c3 = q;
}

// c0..c3 for any z: quarter z until |z| <= 0.1, series there, then the
// duplication formulas c0(4z) = 2 c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2 / 2,
// c3(4z) = (c3 + c1 c2) / 4.
__device__ inline void stumpff_any(double z, double& c0, double& c1, double& c2, double& c3) {
    int k = 0;
    while (fabs(z) > 0.1 && k < 80) {
        z *= 0.25;
        ++k;
    }
    c23_poly<7>(z, c2, c3);
    c0 = fma(-z, c2, 1.0);
    c1 = fma(-z, c3, 1.0);
    for (; k > 0; --k) {
        const double n3 = 0.25 * fma(c1, c2, c3);
        const double n2 = 0.5 * c1 * c1;
        const double n1 = c0 * c1;
        const double n0 = fma(2.0 * c0, c0, -1.0);
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
}

// ---------------------------------------------------------------------------
// General solver: any orbit, any dt.  Bound orbits first drop whole periods.
// Newton iteration on T(s) - dt with a bisection safeguard (bisect whenever
// Newton would leave the bracket or fails to halve the previous step).
// Returns false if it does not converge within the iteration budget.
// ---------------------------------------------------------------------------
// Solve T(s) = r0 G1 + u G2 + mu G3 = tau for s, where tau is dt minus whole
// periods for bound orbits (k periods removed; tau = dt - k P).  Newton with a
// bisection safeguard.  Returns false if it does not converge.
__device__ inline bool universal_solve(double mu, double dt, double r0, double u, double beta, double& s_out,
                                       double& tau_out, double& k_out) {
    double tau = dt, kper = 0.0;
    if (beta > 0.0) {
        const double n = beta * sqrt(beta) / mu;  // mean motion sqrt(mu alpha^3), alpha = beta / mu
        const double period = 6.283185307179586476925286766559 / n;
        kper = rint(dt / period);
        tau = dt - period * kper;
    }
    tau_out = tau;
    k_out = kper;
    if (tau == 0.0) {
        s_out = 0.0;
        return true;
    }
    const double sgn = tau > 0.0 ? 1.0 : -1.0;
    double c0, c1, c2, c3;
    // bracket: T(0) = 0 and T increases with s
    double lo = 0.0, hi = tau / r0;
    int grow = 0;
    for (;;) {
        stumpff_any(beta * hi * hi, c0, c1, c2, c3);
        const double T = r0 * hi * c1 + u * hi * hi * c2 + mu * hi * hi * hi * c3;
        if ((T - tau) * sgn >= 0.0) break;
        lo = hi;
        hi *= 2.0;
        if (++grow > 200) return false;
    }
    if (sgn < 0.0) {
        const double t = lo;
        lo = hi;
        hi = t;
    }
    double s = tau / r0;
    if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
    double dsold = hi - lo;
    for (int it = 0; it < 300; ++it) {
        stumpff_any(beta * s * s, c0, c1, c2, c3);
        const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
        const double F = r0 * G1 + u * G2 + mu * G3 - tau;
        const double Fp = r0 * c0 + u * G1 + mu * G2;
        if (F < 0.0) {
            if (s > lo) lo = s;
        } else {
            if (s < hi) hi = s;
        }
        double ds = -F / Fp;
        // a step below the tolerance is converged; test it before the safeguard,
        // since s + ds can round onto a bracket end and look like an escape
        if (fabs(ds) <= 1e-15 * fabs(s)) {
            s_out = s + ds;
            return true;
        }
        double sn = s + ds;
        if (!(sn > lo && sn < hi) || fabs(ds) > 0.5 * fabs(dsold)) {
            sn = 0.5 * (lo + hi);
            ds = sn - s;
        }
        dsold = ds;
        s = sn;
        if ((hi - lo) <= 1e-15 * fabs(s)) {
            s_out = s;
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// General solver: any orbit, any dt.  Bound orbits first drop whole periods.
// Returns false if the solve does not converge within the iteration budget.
// ---------------------------------------------------------------------------
__device__ inline bool drift_general(double mu, double dt, double& x, double& y, double& z, double& vx, double& vy,
                                     double& vz) {
    const double r0 = sqrt(x * x + y * y + z * z);
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double u = x * vx + y * vy + z * vz;
    if (!(r0 > 0.0) || !isfinite(r0) || !isfinite(v2)) return false;
    const double beta = 2.0 * mu / r0 - v2;
    double s, tau, kper;
    if (!universal_solve(mu, dt, r0, u, beta, s, tau, kper)) return false;
    if (tau == 0.0) return true;
    double c0, c1, c2, c3;
    stumpff_any(beta * s * s, c0, c1, c2, c3);
    const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
    const double r = r0 * c0 + u * G1 + mu * G2;
    const double fm1 = -mu * G2 / r0;
    const double g = tau - mu * G3;
    const double fd = -mu * G1 / (r * r0);
    const double gdm1 = -mu * G2 / r;
    const double x0 = x, y0 = y, z0 = z;
    x = fma(fm1, x0, fma(g, vx, x0));
    y = fma(fm1, y0, fma(g, vy, y0));
    z = fma(fm1, z0, fma(g, vz, z0));
    vx = fma(fd, x0, fma(gdm1, vx, vx));
    vy = fma(fd, y0, fma(gdm1, vy, vy));
    vz = fma(fd, z0, fma(gdm1, vz, vz));
    return true;
}

// ---------------------------------------------------------------------------
// The paper's solver (section 2.2): Newton's method on Kepler's equation with
// a fixed number of iterations from a starting guess, and deactivation of a
// particle whose solve has not converged to the quoted 1e-14.  Bound orbits
// with r0 alpha >= 1e-3 use the equation for x = E - E0 in difference form,
//   F(x) = x - ec sin x + es (1 - cos x) - dM,
//   ec = 1 - r0 alpha (= e cos E0),  es = u / (n a^2) (= e sin E0),  dM = n dt,
// with dM reduced to [-pi, pi] by whole periods, the start x0 = dM / (1 - ec)
// and plain Newton steps (no safeguard).  "Converged" means the last step has
// |dx| <= tol.  Other orbits (unbound or nearly radial), which the paper does
// not treat, use the converged universal-variable solver.  Library sin, cos,
// sqrt and division: this mode reproduces the paper's algorithm, it is not
// the tuned path.
// Returns 0 (drifted), 1 (not converged: state unchanged) or 2 (the
// universal-variable solver failed: state unchanged).
// ---------------------------------------------------------------------------
__device__ inline int drift_paper(double mu, double dt, int iters, double tol, double& x, double& y, double& z,
                                  double& vx, double& vy, double& vz) {
    const double r0 = sqrt(x * x + y * y + z * z);
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double u = x * vx + y * vy + z * vz;
    const double alpha = 2.0 / r0 - v2 / mu;
    if (!(alpha > 0.0 && r0 * alpha >= 1e-3)) {
        if (dt == 0.0) return 0;
        return drift_general(mu, dt, x, y, z, vx, vy, vz) ? 0 : 2;
    }
    constexpr double kTwoPi = 6.283185307179586476925286766559;
    const double a = 1.0 / alpha;
    const double n = sqrt(mu / (a * a * a));
    const double ec = 1.0 - r0 / a;
    const double es = u / (n * a * a);
    double dM = n * dt;
    dM = dM - floor(dM / kTwoPi + 0.5) * kTwoPi;
    double xe = dM / (1.0 - ec);
    double dx = 0.0;
    for (int it = 0; it < iters; ++it) {
        double sx, cx;
        sincos(xe, &sx, &cx);
        const double F = xe - ec * sx + es * (1.0 - cx) - dM;
        const double Fp = 1.0 - ec * cx + es * sx;
        dx = -F / Fp;
        xe = xe + dx;
    }
    if (!(fabs(dx) <= tol)) return 1;
    double sx, cx;
    sincos(xe, &sx, &cx);
    const double omc = 1.0 - cx;
    const double f = 1.0 - (a / r0) * omc;
    const double g = (dM - (xe - sx)) / n;
    const double r = a * (1.0 - ec * cx + es * sx);
    const double fd = -n * a * a * sx / (r * r0);
    const double gd = 1.0 - (a / r) * omc;
    const double x0 = x, y0 = y, z0 = z, vx0 = vx, vy0 = vy, vz0 = vz;
    x = f * x0 + g * vx0;
    y = f * y0 + g * vy0;
    z = f * z0 + g * vz0;
    vx = fd * x0 + gd * vx0;
    vy = fd * y0 + gd * vy0;
    vz = fd * z0 + gd * vz0;
    return 0;
}

// ---------------------------------------------------------------------------
// Fast path.  Must be called by all 32 lanes of a warp together.
//   part       : this lane's result is wanted (inactive lanes still execute)
//   r0, mur0   : |r| and mu/|r| of the current position; on success they are
//                replaced by the values at the drifted position (r(s) is known
//                from the solve, so the next step needs no square root)
// On success (return true) the state is advanced; on false nothing changes.
// ---------------------------------------------------------------------------
// polynomial tiers: largest |z| in the warp picks the degree of c2, c3
constexpr float kZ3 = 0.001953125f;  // 2^-9: degree 3 reaches 2^-56
constexpr float kZ5 = 0.03125f;      // 2^-5: degree 5
constexpr float kZ7 = 0.1f;          // degree 7 (fast-path limit)

// s0 is the FP32 root (24 significant bits), s2 = s0^2 exact and s3 = s0^3
// rounded once (float_powers).  The Halley step removes the start error of
// ~2^-24 |s|; its cubic convergence leaves far below 2^-60.
template <int DEG>
__device__ __forceinline__ void fast_tail(double mu, double dt, double beta, double& r0, double& mur0, double u,
                                          double q, double s0, double s2, double s3, float uf, float bf, double& x,
                                          double& y, double& z, double& vx, double& vy, double& vz, bool& ok) {
    const double zz = beta * s2;
    double c2, c3;
    c23_poly<DEG>(zz, c2, c3);
    const double G2 = s2 * c2;
    const double G3 = s3 * c3;
    const double G1 = fma(-beta, G3, s0);
    // r = T'(s) = r0 G0 + u G1 + mu G2 = r0 + q G2 + u G1  (q = mu - beta r0, G0 = 1 - beta G2)
    const double F = fma(r0, G1, fma(u, G2, fma(mu, G3, -dt)));
    const double r = fma(u, G1, fma(q, G2, r0));
    const double rinv = rcp_40(r);
    const double dN = -F * rinv;
    // Halley: dH = dN / (1 + dN T''/(2 T')) ~ dN (1 - k); k ~ 1e-8 needs only FP32
    const float G2f = d2f_bits(G2), G1f = d2f_bits(G1);
    const float G0f = fmaf(-bf, G2f, 1.0f);
    const float Fpp = fmaf(uf, G0f, d2f_bits(q) * G1f);  // T''(s) = u G0 + q G1
    const float dNf = d2f_bits(dN);
    const float kf = 0.5f * dNf * Fpp * d2f_bits(rinv);
    const double dH = fma(dN, -f2d_bits(kf), dN);
    const double s1 = s0 + dH;
    // G2(s+d) = G2 + d (G1 + d/2 G0),  G3(s+d) = G3 + d (G2 + d/2 G1)  (third order ~ d^3: negligible)
    const float hf = 0.5f * d2f_bits(dH);
    const double t2 = G1 + f2d_bits(hf * G0f);
    const double t3 = G2 + f2d_bits(hf * G1f);
    const double G2n = fma(dH, t2, G2);
    const double G3n = fma(dH, t3, G3);
    const double G1n = fma(-beta, G3n, s1);
    // domain checks (integer tests): r > 0 and the correction small against s
    const bool good = (__double2hiint(r) > 0) && (exp_bits(dH) + 14 <= exp_bits(s0) || dH == 0.0);
    ok = ok && good;
    const double fm1 = -mur0 * G2n;
    const double g = fma(-mu, G3n, dt);
    const double x1 = fma(fm1, x, fma(g, vx, x));
    const double y1 = fma(fm1, y, fma(g, vy, y));
    const double z1 = fma(fm1, z, fma(g, vz, z));
    // |r| and mu/|r| at the new position from the position itself: the next
    // step starts from them, and values carried from r(s) instead would
    // random-walk away from |x| (amplified in beta = 2 mu/r - v^2, which
    // cancels strongly near the pericentre of an eccentric orbit)
    const double x2 = fma(x1, x1, fma(y1, y1, z1 * z1));
    const double rinv1 = rsqrt_full(x2);
    const double fd = -(mur0 * rinv1) * G1n;
    const double mur1 = mu * rinv1;
    const double gdm1 = -mur1 * G2n;
    if (ok) {
        const double x0 = x, y0 = y, z0 = z;
        x = x1;
        y = y1;
        z = z1;
        vx = fma(fd, x0, fma(gdm1, vx, vx));
        vy = fma(fd, y0, fma(gdm1, vy, vy));
        vz = fma(fd, z0, fma(gdm1, vz, vz));
        r0 = x2 * rinv1;
        mur0 = mur1;
    }
}

// Returns true when the lane's drift was done here; false when the caller must
// use drift_general (or when part == false).
__device__ __forceinline__ bool drift_fast(double mu, float muf, double dt, float dtf, bool part, double& r0,
                                           double& mur0, double& x, double& y, double& z, double& vx, double& vy,
                                           double& vz) {
    const double u = fma(x, vx, fma(y, vy, z * vz));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double beta = fma(2.0, mur0, -v2);

    // ---- FP32 solve of T(s) = dt ------------------------------------------------
    const float r0f = d2f_bits(r0), uf = d2f_bits(u), bf = d2f_bits(beta);
    // domain: r0 and |v|^2 well inside the float range (integer exponent tests)
    const int er = exp_bits(r0), ev = exp_bits(v2);
    bool ok = part && er > 1023 - 60 && er < 1023 + 60 && ev < 1023 + 120 && ev > 1023 - 200;
    float s = __fdividef(dtf, r0f);
    float zf = 0.f, dsf = 0.f;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
        zf = bf * s * s;
        const float c2 = fmaf(zf, fmaf(zf, fmaf(zf, -1.0f / 40320.0f, 1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
        const float c3 = fmaf(zf, fmaf(zf, fmaf(zf, -1.0f / 362880.0f, 1.0f / 5040.0f), -1.0f / 120.0f), 1.0f / 6.0f);
        const float s2f = s * s;
        const float G1 = s * fmaf(-zf, c3, 1.0f);
        const float G2 = s2f * c2;
        const float G3 = s2f * s * c3;
        const float F = fmaf(r0f, G1, fmaf(uf, G2, fmaf(muf, G3, -dtf)));
        const float Fp = fmaf(r0f, fmaf(-zf, c2, 1.0f), fmaf(uf, G1, muf * G2));
        dsf = -__fdividef(F, Fp);
        s += dsf;
    }
    zf = bf * s * s;
    // accept the FP32 root only if its last Newton step was below 2^-20 |s|: the
    // Halley step then leaves ~(2^-20)^3 and the neglected third-order terms of
    // the G-function updates are as small; other lanes use the general solver
    ok = ok && (fabsf(zf) <= kZ7) && (fabsf(dsf) <= 9.5367431640625e-7f * fabsf(s) + 1e-30f) && isfinite(s);
    // ---- warp-uniform polynomial degree ------------------------------------------
    const unsigned zb = ok ? __float_as_uint(fabsf(zf)) : 0u;
    const unsigned zmax = __reduce_max_sync(kFullMask, zb);
    // s0 = the FP32 root; s0^2 exact and s0^3 rounded once, in integer arithmetic
    const double s0 = f2d_bits(s);
    double s2, s3;
    ok = float_powers(s, s2, s3) && ok;
    const double q = fma(-beta, r0, mu);
    if (zmax <= __float_as_uint(kZ3)) {
        fast_tail<3>(mu, dt, beta, r0, mur0, u, q, s0, s2, s3, uf, bf, x, y, z, vx, vy, vz, ok);
    } else if (zmax <= __float_as_uint(kZ5)) {
        fast_tail<5>(mu, dt, beta, r0, mur0, u, q, s0, s2, s3, uf, bf, x, y, z, vx, vy, vz, ok);
    } else {
        fast_tail<7>(mu, dt, beta, r0, mur0, u, q, s0, s2, s3, uf, bf, x, y, z, vx, vy, vz, ok);
    }
    return ok;
}

// |r| and 1/|r| of a position (used where no previous drift provides them).
__device__ __forceinline__ void radius_of(double x, double y, double z, double& r, double& rinv) {
    const double r2 = fma(x, x, fma(y, y, z * z));
    rinv = rsqrt_full(r2);
    r = r2 * rinv;
}

// ---------------------------------------------------------------------------
// Derivatives of the drift (tangent and adjoint maps).
//
// With G_n(s, beta) = s^n c_n(beta s^2):  dG_n/ds = G_{n-1} (dG_0/ds = -beta G_1)
// and dG_n/dbeta = -(s G_{n+1} - n G_{n+2}) / 2 (from the series term by term).
// s solves T(s) = r0 G1 + u G2 + mu G3 = tau with tau = dt - k P(beta),
// P = 2 pi mu beta^(-3/2), so by implicit differentiation
//   ds = (dtau - G1 dr0 - G2 du - T_beta dbeta) / R,   R = T'(s),
//   T_beta = r0 G1_beta + u G2_beta + mu G3_beta,   dtau = 1.5 k P dbeta / beta,
// and r0 = |r|, u = r . v, beta = 2 mu / r0 - v . v.
// ---------------------------------------------------------------------------
// c0..c5 for any z (c4, c5 by series below |z| = 0.1, else c_{n+2} = (1/n! - c_n) / z).
__device__ inline void stumpff_all(double z, double c[6]) {
    stumpff_any(z, c[0], c[1], c[2], c[3]);
    if (fabs(z) <= 0.1) {
        // c4 = sum (-z)^n / (2n+4)!, c5 = sum (-z)^n / (2n+5)!, n = 0..7
        const double a4[8] = {1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0, -1.0 / 3628800.0, 1.0 / 479001600.0,
                              -1.0 / 87178291200.0, 1.0 / 20922789888000.0, -1.0 / 6402373705728000.0};
        const double a5[8] = {1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0, 1.0 / 6227020800.0,
                              -1.0 / 1307674368000.0, 1.0 / 355687428096000.0, -1.0 / 121645100408832000.0};
        double p = a4[7], q = a5[7];
        for (int n = 6; n >= 0; --n) {
            p = fma(p, z, a4[n]);
            q = fma(q, z, a5[n]);
        }
        c[4] = p;
        c[5] = q;
    } else {
        c[4] = (0.5 - c[2]) / z;
        c[5] = (1.0 / 6.0 - c[3]) / z;
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

// c4 and c5 by their series, degree DEG.
template <int DEG>
__device__ __forceinline__ void c45_poly(double z, double& c4, double& c5) {
    constexpr double a[6] = {1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0, -1.0 / 3628800.0, 1.0 / 479001600.0,
                             -1.0 / 87178291200.0};
    constexpr double b[6] = {1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0, 1.0 / 6227020800.0,
                             -1.0 / 1307674368000.0};
    double p = a[DEG], q = b[DEG];
#pragma unroll
    for (int n = DEG - 1; n >= 0; --n) {
        p = fma(p, z, a[n]);
        q = fma(q, z, b[n]);
    }
    c4 = p;
    c5 = q;
}

// G_0..G_3 from G_4, G_5 by the exact recurrence G_n = s^n / n! - beta G_{n+2}
// (c_n(z) = 1/n! - z c_{n+2}(z)); for |z| < 0.1 the correction beta G_{n+2} is
// at most a few percent of s^n / n!, so each G_n is good to an ulp or two.
__device__ __forceinline__ void g_from_g45(double s, double beta, double G[6]) {
    const double s2 = s * s;
    G[3] = fma(-beta, G[5], s2 * s * (1.0 / 6.0));
    G[2] = fma(-beta, G[4], 0.5 * s2);
    G[1] = fma(-beta, G[3], s);
    G[0] = fma(-beta, G[2], 1.0);
}

struct DriftScalars {
    double r0, u, beta, tau, dtau_dbeta, s;
    double G[6], Gb[4];  // G_0..G_5 and dG_n/dbeta, n = 0..3
    double R, f, g, fd, gd;
    double inv_r0, inv_R;  // 1/r0 and 1/R (MUFU seed + one correction: no divisions downstream)
    double mg2r, mg2R, irR;  // mu G2 / r0 (= 1 - f), mu G2 / R (= 1 - gd), 1 / (R r0), unrounded by the 1 -
};

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
__device__ inline void g_functions(DriftScalars& d) {
    const double z = d.beta * d.s * d.s;
    if (z_below(z, kZSeries)) {
        double c4, c5;
        if (z_below(z, kZDeg3))
            c45_poly<3>(z, c4, c5);
        else
            c45_poly<5>(z, c4, c5);
        const double s2 = d.s * d.s;
        d.G[4] = (s2 * s2) * c4;
        d.G[5] = (s2 * s2) * d.s * c5;
        g_from_g45(d.s, d.beta, d.G);
    } else {
        double c[6];
        stumpff_all(z, c);
        double sp = 1.0;
        for (int n = 0; n < 6; ++n) {
            d.G[n] = sp * c[n];
            sp *= d.s;
        }
    }
}

// dG_n/dbeta = -(s G_{n+1} - n G_{n+2}) / 2 and f, g, fd, gd, given the G's and 1/R.
__device__ __forceinline__ void drift_fg(double mu, DriftScalars& d) {
    const double hs = -0.5 * d.s;
    d.Gb[0] = hs * d.G[1];
    d.Gb[1] = fma(hs, d.G[2], 0.5 * d.G[3]);
    d.Gb[2] = fma(hs, d.G[3], d.G[4]);
    d.Gb[3] = fma(hs, d.G[4], 1.5 * d.G[5]);
    const double mg2 = mu * d.G[2];
    d.mg2r = mg2 * d.inv_r0;
    d.mg2R = mg2 * d.inv_R;
    d.irR = d.inv_R * d.inv_r0;
    d.f = 1.0 - d.mg2r;
    d.g = fma(-mu, d.G[3], d.tau);
    d.fd = (-mu * d.G[1]) * d.irR;
    d.gd = 1.0 - d.mg2R;
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

__device__ inline void drift_tangent(double mu, const double st[6], const DriftScalars& d, double t[6]) {
    const double *r = st, *v = st + 3;
    const double dr0 = fma(r[0], t[0], fma(r[1], t[1], r[2] * t[2])) * d.inv_r0;
    const double du = fma(t[0], v[0], fma(t[1], v[1], fma(t[2], v[2], fma(r[0], t[3], fma(r[1], t[4], r[2] * t[5])))));
    const double vtv = fma(v[0], t[3], fma(v[1], t[4], v[2] * t[5]));
    const double dbeta = -2.0 * fma(mu * (d.inv_r0 * d.inv_r0), dr0, vtv);
    const double dtau = d.dtau_dbeta * dbeta;
    const double Tb = fma(d.r0, d.Gb[1], fma(d.u, d.Gb[2], mu * d.Gb[3]));
    const double ds = fma(-d.G[1], dr0, fma(-d.G[2], du, fma(-Tb, dbeta, dtau))) * d.inv_R;
    const double dG0 = fma(-d.beta * d.G[1], ds, d.Gb[0] * dbeta);
    const double dG1 = fma(d.G[0], ds, d.Gb[1] * dbeta);
    const double dG2 = fma(d.G[1], ds, d.Gb[2] * dbeta);
    const double dG3 = fma(d.G[2], ds, d.Gb[3] * dbeta);
    // f = 1 - mu G2 / r0, g = tau - mu G3, fd = -mu G1 / (R r0), gd = 1 - mu G2 / R
    const double df = fma(d.mg2r, dr0, -mu * dG2) * d.inv_r0;
    const double dg = fma(-mu, dG3, dtau);
    const double dR = fma(dr0, d.G[0], fma(d.r0, dG0, fma(du, d.G[1], fma(d.u, dG1, mu * dG2))));
    const double dfd = fma(-mu * d.irR, dG1, -d.fd * fma(dR, d.inv_R, dr0 * d.inv_r0));
    const double dgd = fma(d.mg2R, dR, -mu * dG2) * d.inv_R;
    double o[6];
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
__device__ inline void drift_adjoint(double mu, const double st[6], const DriftScalars& d, double l[6]) {
    const double *r = st, *v = st + 3;
    const double lf = fma(l[0], r[0], fma(l[1], r[1], l[2] * r[2]));
    const double lg = fma(l[0], v[0], fma(l[1], v[1], l[2] * v[2]));
    const double lfd = fma(l[3], r[0], fma(l[4], r[1], l[5] * r[2]));
    const double lgd = fma(l[3], v[0], fma(l[4], v[1], l[5] * v[2]));
    double lr[3], lv[3];
    for (int i = 0; i < 3; ++i) {
        lr[i] = fma(d.f, l[i], d.fd * l[3 + i]);
        lv[i] = fma(d.g, l[i], d.gd * l[3 + i]);
    }
    // through f, g, fd, gd
    const double a = lf * d.inv_r0;
    const double e = d.fd * lfd;
    double lG2 = -mu * fma(lgd, d.inv_R, a);
    const double lG3 = -mu * lg;
    double lG1 = (-mu * d.irR) * lfd;
    const double lR = d.inv_R * fma(d.mg2R, lgd, -e);
    double lr0 = fma(d.mg2r, a, -e * d.inv_r0);
    // through R
    lr0 = fma(d.G[0], lR, lr0);
    const double lG0 = d.r0 * lR;
    double lu = d.G[1] * lR;
    lG1 = fma(d.u, lR, lG1);
    lG2 = fma(mu, lR, lG2);
    // through the G's: s and beta
    const double ls = fma(-d.beta * d.G[1], lG0, fma(d.G[0], lG1, fma(d.G[1], lG2, d.G[2] * lG3)));
    double lbeta = fma(d.Gb[0], lG0, fma(d.Gb[1], lG1, fma(d.Gb[2], lG2, d.Gb[3] * lG3)));
    // s(tau, r0, u, beta): ds = (dtau - G1 dr0 - G2 du - Tb dbeta) / R
    const double Tb = fma(d.r0, d.Gb[1], fma(d.u, d.Gb[2], mu * d.Gb[3]));
    const double lsR = ls * d.inv_R;
    const double ltau = lg + lsR;
    lr0 = fma(-d.G[1], lsR, lr0);
    lu = fma(-d.G[2], lsR, lu);
    lbeta = fma(-Tb, lsR, lbeta);
    lbeta = fma(d.dtau_dbeta, ltau, lbeta);
    // beta = 2 mu / r0 - v . v
    const double tb = 2.0 * lbeta;
    lr0 = fma(-tb, mu * (d.inv_r0 * d.inv_r0), lr0);
    // u = r . v ; r0 = |r|
    const double c = lr0 * d.inv_r0;
    for (int i = 0; i < 3; ++i) {
        l[i] = fma(lu, v[i], fma(c, r[i], lr[i]));
        l[3 + i] = fma(lu, r[i], fma(-tb, v[i], lv[i]));
    }
}

}  // namespace glisse
