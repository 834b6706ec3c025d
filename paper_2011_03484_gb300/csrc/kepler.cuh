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
// bisection safeguard.  Returns false if it does not converge.  Multiply-adds
// are explicit fmas, so every kernel that inlines this rounds the same way.
__device__ inline bool universal_solve(double mu, double dt, double r0, double u, double beta, double& s_out,
                                       double& tau_out, double& k_out) {
    double tau = dt, kper = 0.0;
    if (beta > 0.0) {
        const double n = beta * sqrt(beta) / mu;  // mean motion sqrt(mu alpha^3), alpha = beta / mu
        const double period = 6.283185307179586476925286766559 / n;
        kper = rint(dt / period);
        tau = fma(-period, kper, dt);
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
        const double h2 = hi * hi;
        const double T = fma(r0 * hi, c1, fma(u * h2, c2, (mu * h2) * (hi * c3)));
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
        const double G1 = s * c1, G2 = (s * s) * c2, G3 = (s * s) * (s * c3);
        const double F = fma(r0, G1, fma(u, G2, fma(mu, G3, -tau)));
        const double Fp = fma(r0, c0, fma(u, G1, mu * G2));
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
    // every multiply-add written as an fma: the result must not depend on how a
    // compiler fuses the expression in each kernel that inlines this
    const double r0 = sqrt(fma(x, x, fma(y, y, z * z)));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double u = fma(x, vx, fma(y, vy, z * vz));
    if (!(r0 > 0.0) || !isfinite(r0) || !isfinite(v2)) return false;
    const double beta = (2.0 * mu) / r0 - v2;
    double s, tau, kper;
    if (!universal_solve(mu, dt, r0, u, beta, s, tau, kper)) return false;
    if (tau == 0.0) return true;
    double c0, c1, c2, c3;
    stumpff_any(beta * s * s, c0, c1, c2, c3);
    const double G1 = s * c1, G2 = (s * s) * c2, G3 = (s * s) * (s * c3);
    const double r = fma(r0, c0, fma(u, G1, mu * G2));
    const double fm1 = -mu * G2 / r0;
    const double g = fma(-mu, G3, tau);
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
    const double r0 = sqrt(fma(x, x, fma(y, y, z * z)));
    const double v2 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double u = fma(x, vx, fma(y, vy, z * vz));
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
    dM = fma(-floor(dM / kTwoPi + 0.5), kTwoPi, dM);
    double xe = dM / (1.0 - ec);
    double dx = 0.0;
    for (int it = 0; it < iters; ++it) {
        double sx, cx;
        sincos(xe, &sx, &cx);
        const double F = fma(es, 1.0 - cx, fma(-ec, sx, xe)) - dM;
        const double Fp = fma(es, sx, fma(-ec, cx, 1.0));
        dx = -F / Fp;
        xe = xe + dx;
    }
    if (!(fabs(dx) <= tol)) return 1;
    double sx, cx;
    sincos(xe, &sx, &cx);
    const double omc = 1.0 - cx;
    const double f = fma(-(a / r0), omc, 1.0);
    const double g = (dM - (xe - sx)) / n;
    const double r = a * fma(es, sx, fma(-ec, cx, 1.0));
    const double fd = -n * a * a * sx / (r * r0);
    const double gd = fma(-(a / r), omc, 1.0);
    const double x0 = x, y0 = y, z0 = z, vx0 = vx, vy0 = vy, vz0 = vz;
    x = fma(f, x0, g * vx0);
    y = fma(f, y0, g * vy0);
    z = fma(f, z0, g * vz0);
    vx = fma(fd, x0, gd * vx0);
    vy = fma(fd, y0, gd * vy0);
    vz = fma(fd, z0, gd * vz0);
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

}  // namespace glisse
