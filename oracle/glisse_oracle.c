/*
 * glisse_oracle.c -- plain, slow, scalar FP64 CPU oracle of the GLISSE
 * test-particle map (Zhang & Gladman, arXiv 2011.03484).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the package smoke check and the
 * CPU-baseline leg of the benchmark can compare the CUDA path against an
 * independent statement of the method.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * No FMA contraction, IEEE round-to-nearest double throughout.  Units are
 * AU, yr, M_sun with G = 4 pi^2.
 *
 * What it computes (paper section 2.2, "Implementation"):
 *   - Eq. 1-2: the particle Hamiltonian split H = H_Kepler + H_int with
 *     H_Kepler/m = v^2/2 - G m0/|r| (heliocentric = Jacobi index 1 for a
 *     massless particle) and H_int the direct planet terms plus the indirect
 *     term.
 *   - the five-item kick / elements / drift / Cartesian / kick step list of
 *     section 2.2: a half kick from H_int, a Kepler drift for dt, a half kick.
 *   - the kick acceleration printed after the step list of section 2.2:
 *       dv/dt = -sum_j G m_j r_j/|r_j|^3 - sum_j G m_j (r - r_j)/|r - r_j|^3,
 *     whose first sum is the common term h0 defined in section 2.2.
 *   - the planets follow the standard Wisdom-Holman MVS map in Jacobi
 *     coordinates (section 2.2; the Jacobi definitions are the commented
 *     equations after Eq. 2): eta_i = sum_{j<=i} m_j, r'_i = r_i - R_{i-1},
 *     R_i = sum_{j<=i} m_j r_j / eta_i, Kepler part p'^2/2m' - G m_i m0/|r'_i|.
 *   - removal (section 2.2, close-encounter paragraph): a particle is
 *     deactivated when it comes within R_crit,j of planet j, with
 *     R_crit,j = k * a_j (m_j / 3 m0)^(1/3) (Hill radius) or a fixed distance;
 *     its state is kept as it was at the encounter.  An escape radius r_max
 *     is added (the tiny 1024-particle workload removes particles that reach
 *     r > 1000 AU); the paper itself never states one.
 *
 * Readings of points the paper leaves open are listed at each function.
 */
#ifndef ORC_OPCOUNT /* opcount.cpp compiles the real-valued map alone, as C++ */
#include <complex.h>
#endif
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_G (4.0 * ORC_PI * ORC_PI)

/* status codes shared by the oracle's own functions */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_EKEPLER -2
#define ORC_ENONFINITE -3

/* removal reasons recorded per particle */
#define RSN_ALIVE 0
#define RSN_ESCAPE -1
#define RSN_KEPLER -2
#define RSN_NONFINITE -3

double orc_G(void) { return ORC_G; }

/* ------------------------------------------------------------------------ */
/* Stumpff functions c_k(z) = sum_{n>=0} (-z)^n / (2n+k)!, k = 0..3.         */
/* Textbook definition (Stumpff; Danby ch. 6).  Series for |z| < 1, closed  */
/* trigonometric / hyperbolic forms elsewhere.                              */
/* ------------------------------------------------------------------------ */
static void stumpff(double z, double c[4])
{
    if (fabs(z) < 1.0) {
        for (int k = 0; k < 4; ++k) {
            /* term_n = (-z)^n / (2n+k)! */
            double fact = 1.0;
            for (int i = 2; i <= k; ++i) fact *= (double)i;
            double term = 1.0 / fact;
            double sum = term;
            for (int n = 1; n < 40; ++n) {
                term *= -z / ((double)(2 * n + k - 1) * (double)(2 * n + k));
                sum += term;
                if (fabs(term) < 1e-20 * fabs(sum)) break;
            }
            c[k] = sum;
        }
    } else if (z > 0.0) {
        double w = sqrt(z);
        c[0] = cos(w);
        c[1] = sin(w) / w;
        c[2] = (1.0 - cos(w)) / z;
        c[3] = (w - sin(w)) / (z * w);
    } else {
        double w = sqrt(-z);
        c[0] = cosh(w);
        c[1] = sinh(w) / w;
        c[2] = (cosh(w) - 1.0) / (-z);
        c[3] = (sinh(w) - w) / (-z * w);
    }
}

/* ------------------------------------------------------------------------ */
/* Kepler drift: advance (r, v) for time dt on the two-body orbit with       */
/* gravitational parameter mu.  Section 2.2 describes it as solving          */
/* Kepler's equation for the change of mean anomaly                          */
/*     dM = sqrt(G m0 / a^3) dt = E(t) - E(t0) - e (sin E(t) - sin E(t0)),   */
/* then converting elements back to Cartesian.  Reading: the equivalent      */
/* Gauss f and g form in x = E(t) - E(t0) is used for bound orbits;          */
/* unbound or nearly radial orbits use the universal-variable form.  Both    */
/* are exact two-body propagations; Newton iteration with a bisection        */
/* safeguard runs to convergence (the paper's fixed five iterations are a    */
/* performance choice of its GPU code, section 2.2).                        */
/* ------------------------------------------------------------------------ */

/* counts Newton iterations of the last drift (diagnostic only) */
static _Thread_local int g_last_iters;

static int drift_dE(double mu, double dt, double* st, double r0, double u, double alpha)
{
    double a = 1.0 / alpha;
    double n = sqrt(mu / (a * a * a));
    double ec = 1.0 - r0 / a;      /* e cos E0 */
    double es = u / (n * a * a);   /* e sin E0 */
    double e = sqrt(ec * ec + es * es);
    double dM = n * dt;
    /* whole orbits change nothing: reduce dM to [-pi, pi] */
    double k = floor(dM / (2.0 * ORC_PI) + 0.5);
    dM = dM - k * (2.0 * ORC_PI);
    /* F(x) = x - ec sin x + es (1 - cos x) - dM is increasing (F' = r/a > 0)
     * and F(x) - (x - dM) = e sin E0 - e sin(E0 + x) lies in [-2e, 2e]. */
    double lo = dM - 2.0 * e - 1e-14, hi = dM + 2.0 * e + 1e-14;
    double x = dM / (1.0 - ec);
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    int it;
    int conv = 0;
    double dxold = hi - lo;
    for (it = 0; it < 200; ++it) {
        double s = sin(x), c = cos(x);
        double F = x - ec * s + es * (1.0 - c) - dM;
        double Fp = 1.0 - ec * c + es * s;
        if (F < 0.0) { if (x > lo) lo = x; }
        else { if (x < hi) hi = x; }
        double dx = -F / Fp;
        /* a Newton step below the tolerance is the converged answer (checked before
         * the safeguard: x + dx may round onto a bracket end) */
        if (fabs(dx) <= 1e-15) { x += dx; conv = 1; break; }
        double xn = x + dx;
        /* safeguard: bisect when Newton leaves the bracket or does not halve the last step */
        if (!(xn > lo && xn < hi) || fabs(dx) > 0.5 * fabs(dxold)) { xn = 0.5 * (lo + hi); dx = xn - x; }
        dxold = dx;
        x = xn;
        if (hi - lo <= 1e-15) { conv = 1; break; }
    }
    g_last_iters = it + 1;
    if (!conv) return ORC_EKEPLER;
    double s = sin(x), c = cos(x);
    double omc = 1.0 - c;
    double f = 1.0 - (a / r0) * omc;
    double g = (dM - (x - s)) / n;
    double r = a * (1.0 - ec * c + es * s);
    double fd = -n * a * a * s / (r * r0);
    double gd = 1.0 - (a / r) * omc;
    double x0 = st[0], y0 = st[1], z0 = st[2], vx = st[3], vy = st[4], vz = st[5];
    st[0] = f * x0 + g * vx;
    st[1] = f * y0 + g * vy;
    st[2] = f * z0 + g * vz;
    st[3] = fd * x0 + gd * vx;
    st[4] = fd * y0 + gd * vy;
    st[5] = fd * z0 + gd * vz;
    return ORC_OK;
}

/* Universal variables (Danby, "Fundamentals of Celestial Mechanics", sec.
 * 6.9; G-functions G_k(s) = s^k c_k(beta s^2), beta = 2 mu / r0 - v0^2):
 *   time:  r0 G1 + u G2 + mu G3 = dt,   u = r0 . v0
 *   r(s) = r0 G0 + u G1 + mu G2  (= dt'(s) > 0)
 *   f = 1 - mu G2 / r0, g = dt - mu G3, fdot = -mu G1 / (r r0), gdot = 1 - mu G2 / r. */
static int drift_univ(double mu, double dt, double* st, double r0, double u, double alpha)
{
    double beta = mu * alpha;
    if (alpha > 0.0) {
        double n = sqrt(mu * alpha * alpha * alpha);
        double P = 2.0 * ORC_PI / n;
        double k = floor(dt / P + 0.5);
        dt = dt - k * P;
    }
    if (dt == 0.0) { g_last_iters = 0; return ORC_OK; }
    double sgn = dt > 0.0 ? 1.0 : -1.0;
    double c[4];
    /* bracket the root: F(0) = -dt, F increasing */
    double lo = 0.0, hi = dt / r0;
    int grow = 0;
    for (;;) {
        stumpff(beta * hi * hi, c);
        double G1 = hi * c[1], G2 = hi * hi * c[2], G3 = hi * hi * hi * c[3];
        double F = r0 * G1 + u * G2 + mu * G3 - dt;
        if (F * sgn >= 0.0) break;
        lo = hi;
        hi *= 2.0;
        if (++grow > 200) return ORC_EKEPLER;
    }
    if (sgn < 0.0) { double t = lo; lo = hi; hi = t; } /* keep lo < hi */
    double s = dt / r0;
    if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
    int it, conv = 0;
    double dsold = hi - lo;
    for (it = 0; it < 300; ++it) {
        stumpff(beta * s * s, c);
        double G0 = c[0], G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
        double F = r0 * G1 + u * G2 + mu * G3 - dt;
        double Fp = r0 * G0 + u * G1 + mu * G2;
        if (F < 0.0) { if (s > lo) lo = s; }
        else { if (s < hi) hi = s; }
        double ds = -F / Fp;
        /* a Newton step below the tolerance is the converged answer (checked before
         * the safeguard: s + ds may round onto a bracket end) */
        if (fabs(ds) <= 1e-15 * fabs(s)) { s += ds; conv = 1; break; }
        double sn = s + ds;
        /* safeguard: bisect when Newton leaves the bracket or does not halve the last step */
        if (!(sn > lo && sn < hi) || fabs(ds) > 0.5 * fabs(dsold)) { sn = 0.5 * (lo + hi); ds = sn - s; }
        dsold = ds;
        s = sn;
        if (hi - lo <= 1e-15 * fabs(s)) { conv = 1; break; }
    }
    g_last_iters = it + 1;
    if (!conv) return ORC_EKEPLER;
    stumpff(beta * s * s, c);
    double G0 = c[0], G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
    double r = r0 * G0 + u * G1 + mu * G2;
    double f = 1.0 - mu * G2 / r0;
    double g = dt - mu * G3;
    double fd = -mu * G1 / (r * r0);
    double gd = 1.0 - mu * G2 / r;
    double x0 = st[0], y0 = st[1], z0 = st[2], vx = st[3], vy = st[4], vz = st[5];
    st[0] = f * x0 + g * vx;
    st[1] = f * y0 + g * vy;
    st[2] = f * z0 + g * vz;
    st[3] = fd * x0 + gd * vx;
    st[4] = fd * y0 + gd * vy;
    st[5] = fd * z0 + gd * vz;
    return ORC_OK;
}

/* Public: drift st[6] = (x,y,z,vx,vy,vz) by dt about mu.  Returns 0, or
 * ORC_EKEPLER when the solve did not converge, ORC_ENONFINITE on bad input. */
int orc_kepler_drift(double mu, double dt, double* st)
{
    for (int i = 0; i < 6; ++i) if (!isfinite(st[i])) return ORC_ENONFINITE;
    double r0 = sqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2]);
    if (!(r0 > 0.0)) return ORC_ENONFINITE;
    double v2 = st[3] * st[3] + st[4] * st[4] + st[5] * st[5];
    double u = st[0] * st[3] + st[1] * st[4] + st[2] * st[5];
    double alpha = 2.0 / r0 - v2 / mu;
    if (dt == 0.0) { g_last_iters = 0; return ORC_OK; } /* zero time: identity */
    /* bound and not nearly radial near pericentre: eccentric-anomaly form */
    if (alpha > 0.0 && r0 * alpha >= 1e-3) return drift_dE(mu, dt, st, r0, u, alpha);
    return drift_univ(mu, dt, st, r0, u, alpha);
}

int orc_last_iters(void) { return g_last_iters; }

/* ------------------------------------------------------------------------ */
/* The paper's own solver (section 2.2): Newton's method on Kepler's         */
/* equation with a fixed, user-set number of iterations (five by default),   */
/* started from a "judicious" guess; a particle whose solve has not reached  */
/* the 1e-14 convergence the paper quotes is deactivated.                    */
/* Readings: the equation is taken in the difference form of drift_dE,       */
/*     F(x) = x - ec sin x + es (1 - cos x) - dM,                            */
/* the guess is x0 = dM / (1 - ec) (dM reduced to [-pi, pi]), every         */
/* iteration is a plain Newton step x <- x - F(x)/F'(x) with no safeguard,   */
/* and "converged" means the last step satisfies |dx| <= tol (absolute, in   */
/* radians).  Orbits outside the eccentric-anomaly branch (unbound or nearly */
/* radial) are not covered by the paper and use the converged universal-     */
/* variable drift.  *last_dx receives |dx| of the last step (0 when the      */
/* universal branch ran).                                                    */
/* ------------------------------------------------------------------------ */
static int drift_dE_fixed(double mu, double dt, double* st, double r0, double u, double alpha, int iters,
                          double tol, double* last_dx)
{
    double a = 1.0 / alpha;
    double n = sqrt(mu / (a * a * a));
    double ec = 1.0 - r0 / a;
    double es = u / (n * a * a);
    double dM = n * dt;
    double k = floor(dM / (2.0 * ORC_PI) + 0.5);
    dM = dM - k * (2.0 * ORC_PI);
    double x = dM / (1.0 - ec);
    double dx = 0.0;
    for (int it = 0; it < iters; ++it) {
        double s = sin(x), c = cos(x);
        double F = x - ec * s + es * (1.0 - c) - dM;
        double Fp = 1.0 - ec * c + es * s;
        dx = -F / Fp;
        x = x + dx;
    }
    g_last_iters = iters;
    *last_dx = fabs(dx);
    if (!(fabs(dx) <= tol)) return ORC_EKEPLER;
    double s = sin(x), c = cos(x);
    double omc = 1.0 - c;
    double f = 1.0 - (a / r0) * omc;
    double g = (dM - (x - s)) / n;
    double r = a * (1.0 - ec * c + es * s);
    double fd = -n * a * a * s / (r * r0);
    double gd = 1.0 - (a / r) * omc;
    double x0 = st[0], y0 = st[1], z0 = st[2], vx = st[3], vy = st[4], vz = st[5];
    st[0] = f * x0 + g * vx;
    st[1] = f * y0 + g * vy;
    st[2] = f * z0 + g * vz;
    st[3] = fd * x0 + gd * vx;
    st[4] = fd * y0 + gd * vy;
    st[5] = fd * z0 + gd * vz;
    return ORC_OK;
}

/* Public: drift with the paper's fixed-iteration solve (see above).  Returns
 * 0, ORC_EKEPLER when the last Newton step exceeds tol (st unchanged), or
 * ORC_ENONFINITE on bad input. */
int orc_kepler_drift_fixed(double mu, double dt, double* st, int iters, double tol, double* last_dx)
{
    *last_dx = 0.0;
    if (iters < 1) return ORC_EINVAL;
    for (int i = 0; i < 6; ++i) if (!isfinite(st[i])) return ORC_ENONFINITE;
    double r0 = sqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2]);
    if (!(r0 > 0.0)) return ORC_ENONFINITE;
    double v2 = st[3] * st[3] + st[4] * st[4] + st[5] * st[5];
    double u = st[0] * st[3] + st[1] * st[4] + st[2] * st[5];
    double alpha = 2.0 / r0 - v2 / mu;
    if (alpha > 0.0 && r0 * alpha >= 1e-3) return drift_dE_fixed(mu, dt, st, r0, u, alpha, iters, tol, last_dx);
    if (dt == 0.0) return ORC_OK;
    return drift_univ(mu, dt, st, r0, u, alpha);
}

/* ------------------------------------------------------------------------ */
/* Planets: Wisdom-Holman MVS in Jacobi coordinates (section 2.2).            */
/* Index convention: planets 1..np (array index 0..np-1), star 0.            */
/*   eta_i = m0 + sum_{j<=i} m_j                                             */
/*   helio -> Jacobi:  r'_i = r_i - R_{i-1},  R_{i-1} = sum_{j<i} m_j r_j / eta_{i-1}
 *   Jacobi -> helio:  r_i = r'_i + sum_{k<i} (m_k / eta_k) r'_k             */
/* (velocities transform the same way).                                     */
/* H_Kepler = sum_i [ p'_i^2 / 2m'_i - G m0 m_i / |r'_i| ],  m'_i = m_i eta_{i-1}/eta_i,
 *   so each r'_i drifts on a Kepler orbit with mu_i = G m0 eta_i / eta_{i-1}.
 * H_int = sum_i G m0 m_i (1/|r'_i| - 1/|r_i|) - sum_{i<j} G m_i m_j / |r_i - r_j|.
 * Kick (reading, derived by the chain rule through r(r')):
 *   dv'_k/dt = -(eta_k/eta_{k-1}) [ -G m0 r'_k/|r'_k|^3 + ghat_k + S_k/eta_k ]
 *   ghat_i = G m0 r_i/|r_i|^3 + sum_{j != i} G m_j (r_i - r_j)/|r_i - r_j|^3
 *   S_k = sum_{i>k} m_i ghat_i.                                             */
/* ------------------------------------------------------------------------ */
#define ORC_MAXP 64

typedef struct {
    int np;
    double m0;
    double m[ORC_MAXP];
    double eta[ORC_MAXP + 1]; /* eta[0] = m0, eta[i] = m0 + m_1..m_i (planet i = index i-1) */
    double q[ORC_MAXP][3];    /* Jacobi positions  */
    double w[ORC_MAXP][3];    /* Jacobi velocities */
} orc_psys;

static void jac_to_helio(const orc_psys* P, double (*src)[3], double (*dst)[3])
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < P->np; ++i) {
        for (int d = 0; d < 3; ++d) dst[i][d] = src[i][d] + acc[d];
        double fr = P->m[i] / P->eta[i + 1];
        for (int d = 0; d < 3; ++d) acc[d] += fr * src[i][d];
    }
}

static void helio_to_jac(const orc_psys* P, const double (*src)[3], double (*dst)[3])
{
    double msum[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < P->np; ++i) {
        for (int d = 0; d < 3; ++d) dst[i][d] = src[i][d] - msum[d] / P->eta[i];
        for (int d = 0; d < 3; ++d) msum[d] += P->m[i] * src[i][d];
    }
}

static void planet_kick(orc_psys* P, double tau)
{
    int np = P->np;
    double r[ORC_MAXP][3], gh[ORC_MAXP][3];
    jac_to_helio(P, P->q, r);
    double Gm0 = ORC_G * P->m0;
    for (int i = 0; i < np; ++i) {
        double ri2 = r[i][0] * r[i][0] + r[i][1] * r[i][1] + r[i][2] * r[i][2];
        double ri3 = ri2 * sqrt(ri2);
        for (int d = 0; d < 3; ++d) gh[i][d] = Gm0 * r[i][d] / ri3;
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            double dx = r[i][0] - r[j][0], dy = r[i][1] - r[j][1], dz = r[i][2] - r[j][2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double d3 = d2 * sqrt(d2);
            double Gmj = ORC_G * P->m[j];
            gh[i][0] += Gmj * dx / d3;
            gh[i][1] += Gmj * dy / d3;
            gh[i][2] += Gmj * dz / d3;
        }
    }
    double S[3] = {0.0, 0.0, 0.0}; /* sum over i > k of m_i ghat_i */
    for (int k = np - 1; k >= 0; --k) {
        double q2 = P->q[k][0] * P->q[k][0] + P->q[k][1] * P->q[k][1] + P->q[k][2] * P->q[k][2];
        double q3 = q2 * sqrt(q2);
        double ratio = P->eta[k + 1] / P->eta[k];
        for (int d = 0; d < 3; ++d) {
            double grad = -Gm0 * P->q[k][d] / q3 + gh[k][d] + S[d] / P->eta[k + 1];
            P->w[k][d] -= tau * ratio * grad;
        }
        for (int d = 0; d < 3; ++d) S[d] += P->m[k] * gh[k][d];
    }
}

static int planet_drift(orc_psys* P, double dt)
{
    for (int i = 0; i < P->np; ++i) {
        double mu = ORC_G * P->m0 * P->eta[i + 1] / P->eta[i];
        double st[6] = {P->q[i][0], P->q[i][1], P->q[i][2], P->w[i][0], P->w[i][1], P->w[i][2]};
        int rc = orc_kepler_drift(mu, dt, st);
        if (rc) return rc;
        for (int d = 0; d < 3; ++d) { P->q[i][d] = st[d]; P->w[i][d] = st[3 + d]; }
    }
    return ORC_OK;
}

static void psys_init(orc_psys* P, double m0, int np, const double* pl /* [np][7] m,x,y,z,vx,vy,vz */)
{
    P->np = np;
    P->m0 = m0;
    P->eta[0] = m0;
    double r[ORC_MAXP][3], v[ORC_MAXP][3];
    for (int i = 0; i < np; ++i) {
        P->m[i] = pl[7 * i];
        P->eta[i + 1] = P->eta[i] + P->m[i];
        for (int d = 0; d < 3; ++d) { r[i][d] = pl[7 * i + 1 + d]; v[i][d] = pl[7 * i + 4 + d]; }
    }
    helio_to_jac(P, (const double (*)[3])r, P->q);
    helio_to_jac(P, (const double (*)[3])v, P->w);
}

static void psys_export(const orc_psys* P, double* pl)
{
    double r[ORC_MAXP][3], v[ORC_MAXP][3];
    jac_to_helio(P, (double (*)[3])P->q, r);
    jac_to_helio(P, (double (*)[3])P->w, v);
    for (int i = 0; i < P->np; ++i) {
        pl[7 * i] = P->m[i];
        for (int d = 0; d < 3; ++d) { pl[7 * i + 1 + d] = r[i][d]; pl[7 * i + 4 + d] = v[i][d]; }
    }
}

/* Total energy of star + planets in the barycentric frame (Jacobi kinetic
 * energy plus the full potential); used only as a self-test of the map. */
static double psys_energy(const orc_psys* P)
{
    double r[ORC_MAXP][3];
    jac_to_helio(P, (double (*)[3])P->q, r);
    double T = 0.0, V = 0.0;
    for (int i = 0; i < P->np; ++i) {
        double mp = P->m[i] * P->eta[i] / P->eta[i + 1];
        double w2 = P->w[i][0] * P->w[i][0] + P->w[i][1] * P->w[i][1] + P->w[i][2] * P->w[i][2];
        T += 0.5 * mp * w2;
        double ri = sqrt(r[i][0] * r[i][0] + r[i][1] * r[i][1] + r[i][2] * r[i][2]);
        V -= ORC_G * P->m0 * P->m[i] / ri;
        for (int j = i + 1; j < P->np; ++j) {
            double dx = r[i][0] - r[j][0], dy = r[i][1] - r[j][1], dz = r[i][2] - r[j][2];
            V -= ORC_G * P->m[i] * P->m[j] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    }
    return T + V;
}

/* Advance the planets nsteps steps of kick(dt/2) drift(dt) kick(dt/2).
 *   pl:        [np][7] heliocentric m,x,y,z,vx,vy,vz; in/out
 *   log_pos:   [nsteps+1][np][3] heliocentric positions at t_0..t_n, or NULL
 *   energy:    [nsteps+1] total energy at t_0..t_n, or NULL
 * Returns 0 or a negative status. */
int orc_planet_wh(double m0, int np, double* pl, double dt, int64_t nsteps, double* log_pos, double* energy)
{
    if (np < 0 || np > ORC_MAXP || nsteps < 0) return ORC_EINVAL;
    orc_psys P;
    psys_init(&P, m0, np, pl);
    double r[ORC_MAXP][3];
    if (log_pos) {
        jac_to_helio(&P, P.q, r);
        for (int i = 0; i < np; ++i) for (int d = 0; d < 3; ++d) log_pos[3 * i + d] = r[i][d];
    }
    if (energy) energy[0] = psys_energy(&P);
    for (int64_t k = 0; k < nsteps; ++k) {
        planet_kick(&P, 0.5 * dt);
        int rc = planet_drift(&P, dt);
        if (rc) return rc;
        planet_kick(&P, 0.5 * dt);
        if (log_pos) {
            jac_to_helio(&P, P.q, r);
            double* o = log_pos + (size_t)(k + 1) * 3 * np;
            for (int i = 0; i < np; ++i) for (int d = 0; d < 3; ++d) o[3 * i + d] = r[i][d];
        }
        if (energy) energy[k + 1] = psys_energy(&P);
    }
    psys_export(&P, pl);
    return ORC_OK;
}

/* Critical encounter radius of each planet (section 2.2).  mode 0:
 * R = value * a_j (m_j / (3 m0))^(1/3) where a_j is the planet's initial
 * osculating heliocentric semi-major axis with mu = G (m0 + m_j) (reading:
 * the paper writes a_p without saying which).  mode 1: R = value (a fixed
 * distance for every planet).  Returns ORC_EINVAL for an unbound planet. */
int orc_rcrit(double m0, int np, const double* pl, int mode, double value, double* rcrit)
{
    for (int i = 0; i < np; ++i) {
        if (mode == 1) { rcrit[i] = value; continue; }
        const double* p = pl + 7 * i;
        double r = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
        double v2 = p[4] * p[4] + p[5] * p[5] + p[6] * p[6];
        double mu = ORC_G * (m0 + p[0]);
        double inva = 2.0 / r - v2 / mu;
        if (!(inva > 0.0)) return ORC_EINVAL;
        rcrit[i] = value * (1.0 / inva) * cbrt(p[0] / (3.0 * m0));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Particles: the map of section 2.2 applied to one particle at a time.      */
/* Per step k -> k+1 (planet positions P_k from the log):                    */
/*   1. kick(dt/2) with the acceleration at t_k                              */
/*   2. Kepler drift of dt about mu = G m0                                   */
/*   3. removal tests at t_{k+1} on the drifted position (reading: the paper */
/*      makes the test as part of the acceleration, i.e. at each kick time)  */
/*   4. kick(dt/2) with the acceleration at t_{k+1}                          */
/* A particle whose test fires keeps the state of step 3 (after the drift,   */
/* before the closing kick), removal_step = k+1 (global index), reason =     */
/* planet index 1..np (lowest index wins), or -1 for escape (encounter wins  */
/* over escape).  A failed Kepler solve keeps the state it had just before  */
/* the drift (after the opening kick), reason -2; a non-finite drift result  */
/* keeps the same state, reason -3 (reading: the paper only says such        */
/* particles are deactivated).  The test at t_0 is made when test_first.     */
/* margin[p] records min over all tests of |metric - 1| (metric = d^2 / R^2  */
/* or r^2 / rmax^2); closest[p] records min over tests of d_j^2 / R_j^2.     */
/* ------------------------------------------------------------------------ */
static void particle_accel(int np, const double* Gm, const double* pos /* [np][3] */, const double* r, double* a)
{
    /* h0 = - sum_j G m_j r_j / |r_j|^3 (section 2.2) */
    double h0[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
        const double* rj = pos + 3 * j;
        double rj2 = rj[0] * rj[0] + rj[1] * rj[1] + rj[2] * rj[2];
        double rj3 = rj2 * sqrt(rj2);
        for (int d = 0; d < 3; ++d) h0[d] -= Gm[j] * rj[d] / rj3;
    }
    double dir[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
        const double* rj = pos + 3 * j;
        double dx = r[0] - rj[0], dy = r[1] - rj[1], dz = r[2] - rj[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        double d3 = d2 * sqrt(d2);
        dir[0] -= Gm[j] * dx / d3;
        dir[1] -= Gm[j] * dy / d3;
        dir[2] -= Gm[j] * dz / d3;
    }
    for (int d = 0; d < 3; ++d) a[d] = h0[d] + dir[d];
}

/* returns reason code (0 = no removal) and updates margin / closest */
static int particle_test(int np, const double* pos, const double* rc2, double rmax2, const double* r, double* margin, double* closest)
{
    int hit = 0;
    for (int j = 0; j < np; ++j) {
        const double* rj = pos + 3 * j;
        double dx = r[0] - rj[0], dy = r[1] - rj[1], dz = r[2] - rj[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (rc2[j] > 0.0) {
            double m = d2 / rc2[j];
            double gap = fabs(m - 1.0);
            if (gap < *margin) *margin = gap;
            if (m < *closest) *closest = m;
            if (d2 < rc2[j] && hit == 0) hit = j + 1;
        }
    }
    if (rmax2 > 0.0) {
        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double m = r2 / rmax2;
        double gap = fabs(m - 1.0);
        if (gap < *margin) *margin = gap;
        if (hit == 0 && r2 > rmax2) hit = RSN_ESCAPE;
    }
    return hit;
}

/* Advance npart particles by nsteps steps.
 *   m0, np, pmass[np]: star and planet masses
 *   log_pos: [nsteps+1][np][3] heliocentric planet positions at t_0..t_n
 *   rcrit[np]: encounter radii (0 disables a planet's test); rmax <= 0 disables escape
 *   state: [npart][6] heliocentric x,y,z,vx,vy,vz, in/out
 *   removal_step: [npart] in/out, -1 while alive (particles already removed are skipped)
 *   reason: [npart] in/out
 *   margin, closest: [npart] in/out running minima (initialise to +inf)
 *   step0: global step index of log_pos[0]
 *   test_first: test at t_0 before the first step
 *   nthreads: OpenMP threads (<= 0: library default)
 */
int orc_particles_ex(double m0, int np, const double* pmass, const double* log_pos, int64_t nsteps, double dt,
                     const double* rcrit, double rmax, double* state, int64_t npart, int64_t* removal_step,
                     int32_t* reason, double* margin, double* closest, int64_t step0, int test_first, int nthreads,
                     int kepler_iters, double kepler_tol, double* kepler_dx)
{
    if (np < 0 || np > ORC_MAXP || nsteps < 0 || npart < 0 || kepler_iters < 0) return ORC_EINVAL;
    double Gm[ORC_MAXP], rc2[ORC_MAXP];
    for (int j = 0; j < np; ++j) { Gm[j] = ORC_G * pmass[j]; rc2[j] = rcrit[j] * rcrit[j]; }
    double rmax2 = rmax > 0.0 ? rmax * rmax : 0.0;
    double mu = ORC_G * m0;
    size_t stride = (size_t)3 * np;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int64_t p = 0; p < npart; ++p) {
        if (removal_step[p] >= 0) continue;
        double st[6];
        memcpy(st, state + 6 * p, sizeof st);
        double mg = margin[p], cl = closest[p];
        double kdx = kepler_dx ? kepler_dx[p] : 0.0;
        int64_t rstep = -1;
        int rsn = 0;
        if (test_first) {
            int h = particle_test(np, log_pos, rc2, rmax2, st, &mg, &cl);
            if (h) { rstep = step0; rsn = h; }
        }
        for (int64_t k = 0; k < nsteps && rstep < 0; ++k) {
            const double* P0 = log_pos + (size_t)k * stride;
            const double* P1 = P0 + stride;
            double a[3];
            double saved[6];
            particle_accel(np, Gm, P0, st, a);
            for (int d = 0; d < 3; ++d) st[3 + d] += 0.5 * dt * a[d];
            memcpy(saved, st, sizeof st);
            int rc;
            if (kepler_iters > 0) {
                double ldx;
                rc = orc_kepler_drift_fixed(mu, dt, st, kepler_iters, kepler_tol, &ldx);
                if (ldx > kdx) kdx = ldx;
            } else {
                rc = orc_kepler_drift(mu, dt, st);
            }
            int bad = 0;
            for (int d = 0; d < 6; ++d) if (!isfinite(st[d])) bad = 1;
            if (rc == ORC_EKEPLER || rc == ORC_ENONFINITE || bad) {
                memcpy(st, saved, sizeof st);
                rstep = step0 + k + 1;
                rsn = (rc == ORC_EKEPLER) ? RSN_KEPLER : RSN_NONFINITE;
                break;
            }
            int h = particle_test(np, P1, rc2, rmax2, st, &mg, &cl);
            if (h) { rstep = step0 + k + 1; rsn = h; break; }
            particle_accel(np, Gm, P1, st, a);
            for (int d = 0; d < 3; ++d) st[3 + d] += 0.5 * dt * a[d];
        }
        memcpy(state + 6 * p, st, sizeof st);
        removal_step[p] = rstep;
        reason[p] = rsn;
        margin[p] = mg;
        closest[p] = cl;
        if (kepler_dx) kepler_dx[p] = kdx;
    }
    return ORC_OK;
}

int orc_particles(double m0, int np, const double* pmass, const double* log_pos, int64_t nsteps, double dt,
                  const double* rcrit, double rmax, double* state, int64_t npart, int64_t* removal_step,
                  int32_t* reason, double* margin, double* closest, int64_t step0, int test_first, int nthreads)
{
    return orc_particles_ex(m0, np, pmass, log_pos, nsteps, dt, rcrit, rmax, state, npart, removal_step, reason,
                            margin, closest, step0, test_first, nthreads, 0, 0.0, NULL);
}

/* Convenience: planets and particles together for nsteps from a heliocentric
 * start, exactly as a user of the library would run them. */
int orc_run_ex(double m0, int np, double* pl, double dt, int64_t nsteps, const double* rcrit, double rmax,
               double* state, int64_t npart, int64_t* removal_step, int32_t* reason, double* margin,
               double* closest, int test_first, int nthreads, int kepler_iters, double kepler_tol,
               double* kepler_dx)
{
    double* log = (double*)malloc(sizeof(double) * (size_t)(nsteps + 1) * 3 * (np > 0 ? np : 1));
    if (!log) return ORC_EINVAL;
    double pm[ORC_MAXP];
    for (int j = 0; j < np; ++j) pm[j] = pl[7 * j];
    int rc = orc_planet_wh(m0, np, pl, dt, nsteps, log, NULL);
    if (rc == 0)
        rc = orc_particles_ex(m0, np, pm, log, nsteps, dt, rcrit, rmax, state, npart, removal_step, reason,
                              margin, closest, 0, test_first, nthreads, kepler_iters, kepler_tol, kepler_dx);
    free(log);
    return rc;
}

int orc_run(double m0, int np, double* pl, double dt, int64_t nsteps, const double* rcrit, double rmax,
            double* state, int64_t npart, int64_t* removal_step, int32_t* reason, double* margin, double* closest,
            int test_first, int nthreads)
{
    return orc_run_ex(m0, np, pl, dt, nsteps, rcrit, rmax, state, npart, removal_step, reason, margin, closest,
                      test_first, nthreads, 0, 0.0, NULL);
}

/* ------------------------------------------------------------------------ */
/* Orbital elements and the resonant argument (section 3: the runs log       */
/* osculating elements at a fixed interval, and a particle is counted as     */
/* librating in the p:q resonance with a planet when                         */
/*     phi = p lambda - q lambda_N - (p - q) varpi                           */
/* never comes within 10 degrees of 0, or never within 10 degrees of 180,    */
/* over the logged samples; lambda = varpi + M is the mean longitude and     */
/* varpi = Omega + omega the longitude of pericentre).                      */
/* Readings: elements are those of the two-body orbit about mu in the frame  */
/* asked for; the heliocentric frame uses mu = G m0 for particles and        */
/* G (m0 + m_j) for planet j, the barycentric frame (the frame of the        */
/* paper's 3:1 study) subtracts the barycentre of star and planets and uses  */
/* mu = G (m0 + sum m_j) for every body.  Angles are in [0, 2 pi); for       */
/* e = 0 the pericentre is put at the node, for i = 0 the node on the x      */
/* axis.  Only bound samples (e < 1) of the particle and planet count.      */
/* ------------------------------------------------------------------------ */
static double wrap_2pi(double x)
{
    double y = fmod(x, 2.0 * ORC_PI);
    return y < 0.0 ? y + 2.0 * ORC_PI : y;
}

/* el = a, e, i, Omega, omega, M (hyperbolic orbits: M = e sinh F - F, not wrapped) */
int orc_elements(double mu, const double* st, double* el)
{
    double x = st[0], y = st[1], z = st[2], vx = st[3], vy = st[4], vz = st[5];
    double r = sqrt(x * x + y * y + z * z);
    if (!(r > 0.0) || !(mu > 0.0)) return ORC_EINVAL;
    double v2 = vx * vx + vy * vy + vz * vz;
    double rv = x * vx + y * vy + z * vz;
    /* angular momentum h = r x v */
    double hx = y * vz - z * vy, hy = z * vx - x * vz, hz = x * vy - y * vx;
    double h = sqrt(hx * hx + hy * hy + hz * hz);
    if (!(h > 0.0)) return ORC_EINVAL;
    /* eccentricity vector ((v^2 - mu/r) r - (r.v) v) / mu */
    double c = v2 - mu / r;
    double ex = (c * x - rv * vx) / mu, ey = (c * y - rv * vy) / mu, ez = (c * z - rv * vz) / mu;
    double e = sqrt(ex * ex + ey * ey + ez * ez);
    double a = 1.0 / (2.0 / r - v2 / mu);
    double hxy = sqrt(hx * hx + hy * hy);
    double inc = atan2(hxy, hz);
    /* ascending node along z x h = (-hy, hx, 0) */
    double Om = hxy > 0.0 ? atan2(hx, -hy) : 0.0;
    /* in-plane basis: P towards the node, Q = h_hat x P */
    double Px = cos(Om), Py = sin(Om);
    double Qx = -hz * Py / h, Qy = hz * Px / h, Qz = (hx * Py - hy * Px) / h;
    double u = atan2(x * Qx + y * Qy + z * Qz, x * Px + y * Py); /* argument of latitude */
    double om = e > 0.0 ? atan2(ex * Qx + ey * Qy + ez * Qz, ex * Px + ey * Py) : 0.0;
    double f = u - om; /* true anomaly */
    double M;
    if (e < 1.0) {
        double E = atan2(sqrt(1.0 - e * e) * sin(f), e + cos(f));
        M = wrap_2pi(E - e * sin(E));
    } else if (e > 1.0) {
        double F = 2.0 * atanh(sqrt((e - 1.0) / (e + 1.0)) * tan(0.5 * f));
        M = e * sinh(F) - F;
    } else {
        double D = tan(0.5 * f);
        M = D + D * D * D / 3.0;
    }
    el[0] = a;
    el[1] = e;
    el[2] = inc;
    el[3] = wrap_2pi(Om);
    el[4] = wrap_2pi(om);
    el[5] = M;
    return ORC_OK;
}

/* Heliocentric state of the barycentre of star and planets: sum m_j s_j / (m0 + sum m_j). */
void orc_barycentre(double m0, int np, const double* pm, const double* pl, double* R)
{
    double mt = m0;
    for (int j = 0; j < np; ++j) mt += pm[j];
    for (int d = 0; d < 6; ++d) {
        double acc = 0.0;
        for (int j = 0; j < np; ++j) acc += pm[j] * pl[6 * j + d];
        R[d] = acc / mt;
    }
}

/* One sample: elements of every particle with live[p] != 0 (NaN rows otherwise) in the
 * given frame (0 heliocentric, 1 barycentric); with res_planet >= 0 also the resonant
 * argument phi[p] (NaN when not used) and the running flags near0 / near180 / count.
 *   pl: [np][6] heliocentric planet states at the sample time; pm: [np] masses. */
int orc_sample(double m0, int np, const double* pm, const double* pl, int frame, int res_planet, int res_p,
               int res_q, double avoid, const double* state, const uint8_t* live, int64_t npart, double* elem,
               double* phi, uint8_t* near0, uint8_t* near180, int32_t* count)
{
    if (np < 0 || np > ORC_MAXP || res_planet >= np || (frame != 0 && frame != 1)) return ORC_EINVAL;
    double R[6] = {0, 0, 0, 0, 0, 0};
    double mt = m0;
    for (int j = 0; j < np; ++j) mt += pm[j];
    if (frame == 1) orc_barycentre(m0, np, pm, pl, R);
    double mu_p = ORC_G * (frame == 1 ? mt : m0);
    double lamN = 0.0;
    int resok = 0;
    if (res_planet >= 0) {
        double sN[6], elN[6];
        for (int d = 0; d < 6; ++d) sN[d] = pl[6 * res_planet + d] - R[d];
        double muN = ORC_G * (frame == 1 ? mt : m0 + pm[res_planet]);
        if (orc_elements(muN, sN, elN) == ORC_OK && elN[1] < 1.0) {
            lamN = elN[3] + elN[4] + elN[5];
            resok = 1;
        }
    }
    for (int64_t p = 0; p < npart; ++p) {
        double* o = elem + 6 * p;
        if (phi) phi[p] = NAN;
        if (!live[p]) {
            for (int d = 0; d < 6; ++d) o[d] = NAN;
            continue;
        }
        double s[6];
        for (int d = 0; d < 6; ++d) s[d] = state[6 * p + d] - R[d];
        if (orc_elements(mu_p, s, o) != ORC_OK) {
            for (int d = 0; d < 6; ++d) o[d] = NAN;
            continue;
        }
        if (res_planet >= 0 && resok && o[1] < 1.0) {
            double varpi = o[3] + o[4];
            double lam = varpi + o[5];
            double ph = wrap_2pi(res_p * lam - res_q * lamN - (res_p - res_q) * varpi);
            double d0 = ph < ORC_PI ? ph : 2.0 * ORC_PI - ph;
            double d180 = fabs(ph - ORC_PI);
            if (phi) phi[p] = ph;
            if (d0 < avoid) near0[p] = 1;
            if (d180 < avoid) near180[p] = 1;
            count[p] += 1;
        }
    }
    return ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifndef ORC_OPCOUNT
/* ------------------------------------------------------------------------ */
/* Tangent map by complex-step differentiation (reading for the derivative   */
/* of the map; the paper has no tangent map).  The particle map above is     */
/* repeated in complex arithmetic on state + i h dir, h = 1e-20: every step  */
/* is an analytic function of the state, so Im(result) / h is the exact     */
/* directional derivative J dir up to rounding (no difference quotient, no   */
/* cancellation).  Control flow (branches, convergence, removal tests)       */
/* follows the real parts.  Each Newton solve runs to convergence on the    */
/* real part and then takes two plain complex Newton steps, which carry the  */
/* imaginary part to the root of the perturbed equation.                    */
/* ------------------------------------------------------------------------ */
typedef double complex cplx;

static void stumpff_c(cplx z, cplx c[4])
{
    if (cabs(z) < 1.0) {
        for (int k = 0; k < 4; ++k) {
            double fact = 1.0;
            for (int i = 2; i <= k; ++i) fact *= (double)i;
            cplx term = 1.0 / fact;
            cplx sum = term;
            for (int n = 1; n < 40; ++n) {
                term *= -z / ((double)(2 * n + k - 1) * (double)(2 * n + k));
                sum += term;
                if (cabs(term) < 1e-20 * cabs(sum)) break;
            }
            c[k] = sum;
        }
    } else if (creal(z) > 0.0) {
        cplx w = csqrt(z);
        c[0] = ccos(w);
        c[1] = csin(w) / w;
        c[2] = (1.0 - ccos(w)) / z;
        c[3] = (w - csin(w)) / (z * w);
    } else {
        cplx w = csqrt(-z);
        c[0] = ccosh(w);
        c[1] = csinh(w) / w;
        c[2] = (ccosh(w) - 1.0) / (-z);
        c[3] = (csinh(w) - w) / (-z * w);
    }
}

static void apply_fg_c(cplx* st, cplx f, cplx g, cplx fd, cplx gd)
{
    cplx x0 = st[0], y0 = st[1], z0 = st[2], vx = st[3], vy = st[4], vz = st[5];
    st[0] = f * x0 + g * vx;
    st[1] = f * y0 + g * vy;
    st[2] = f * z0 + g * vz;
    st[3] = fd * x0 + gd * vx;
    st[4] = fd * y0 + gd * vy;
    st[5] = fd * z0 + gd * vz;
}

static int drift_dE_c(double mu, double dt, cplx* st, cplx r0, cplx u, cplx alpha)
{
    cplx a = 1.0 / alpha;
    cplx n = csqrt(mu / (a * a * a));
    cplx ec = 1.0 - r0 / a;
    cplx es = u / (n * a * a);
    double e = sqrt(creal(ec) * creal(ec) + creal(es) * creal(es));
    cplx dM = n * dt;
    double k = floor(creal(dM) / (2.0 * ORC_PI) + 0.5);
    dM = dM - k * (2.0 * ORC_PI);
    double lo = creal(dM) - 2.0 * e - 1e-14, hi = creal(dM) + 2.0 * e + 1e-14;
    cplx x = dM / (1.0 - ec);
    if (!(creal(x) > lo && creal(x) < hi)) x = 0.5 * (lo + hi);
    double dxold = hi - lo;
    int conv = 0;
    for (int it = 0; it < 200 && !conv; ++it) {
        cplx F = x - ec * csin(x) + es * (1.0 - ccos(x)) - dM;
        cplx Fp = 1.0 - ec * ccos(x) + es * csin(x);
        if (creal(F) < 0.0) { if (creal(x) > lo) lo = creal(x); }
        else { if (creal(x) < hi) hi = creal(x); }
        cplx dx = -F / Fp;
        if (fabs(creal(dx)) <= 1e-15) { x += dx; conv = 1; break; }
        double xn = creal(x) + creal(dx);
        if (!(xn > lo && xn < hi) || fabs(creal(dx)) > 0.5 * fabs(dxold)) dx = 0.5 * (lo + hi) - creal(x);
        dxold = creal(dx);
        x += dx;
        if (hi - lo <= 1e-15) conv = 1;
    }
    if (!conv) return ORC_EKEPLER;
    for (int it = 0; it < 2; ++it) {
        cplx F = x - ec * csin(x) + es * (1.0 - ccos(x)) - dM;
        cplx Fp = 1.0 - ec * ccos(x) + es * csin(x);
        x -= F / Fp;
    }
    cplx sx = csin(x), cx = ccos(x);
    cplx omc = 1.0 - cx;
    cplx f = 1.0 - (a / r0) * omc;
    cplx g = (dM - (x - sx)) / n;
    cplx r = a * (1.0 - ec * cx + es * sx);
    cplx fd = -n * a * a * sx / (r * r0);
    cplx gd = 1.0 - (a / r) * omc;
    apply_fg_c(st, f, g, fd, gd);
    return ORC_OK;
}

static int drift_univ_c(double mu, double dt0, cplx* st, cplx r0, cplx u, cplx alpha)
{
    cplx beta = mu * alpha;
    cplx dt = dt0;
    if (creal(alpha) > 0.0) {
        cplx n = csqrt(mu * alpha * alpha * alpha);
        cplx P = 2.0 * ORC_PI / n;
        double k = floor(dt0 / creal(P) + 0.5);
        dt = dt0 - k * P;
    }
    if (creal(dt) == 0.0) return ORC_OK;
    double sgn = creal(dt) > 0.0 ? 1.0 : -1.0;
    cplx c[4];
    double lo = 0.0, hi = creal(dt / r0);
    int grow = 0;
    for (;;) {
        stumpff_c(beta * hi * hi, c);
        cplx T = r0 * hi * c[1] + u * hi * hi * c[2] + mu * hi * hi * hi * c[3];
        if (creal(T - dt) * sgn >= 0.0) break;
        lo = hi;
        hi *= 2.0;
        if (++grow > 200) return ORC_EKEPLER;
    }
    if (sgn < 0.0) { double t = lo; lo = hi; hi = t; }
    cplx s = dt / r0;
    if (!(creal(s) > lo && creal(s) < hi)) s = 0.5 * (lo + hi);
    double dsold = hi - lo;
    int conv = 0;
    for (int it = 0; it < 300 && !conv; ++it) {
        stumpff_c(beta * s * s, c);
        cplx F = r0 * s * c[1] + u * s * s * c[2] + mu * s * s * s * c[3] - dt;
        cplx Fp = r0 * c[0] + u * s * c[1] + mu * s * s * c[2];
        if (creal(F) < 0.0) { if (creal(s) > lo) lo = creal(s); }
        else { if (creal(s) < hi) hi = creal(s); }
        cplx ds = -F / Fp;
        if (fabs(creal(ds)) <= 1e-15 * fabs(creal(s))) { s += ds; conv = 1; break; }
        double sn = creal(s) + creal(ds);
        if (!(sn > lo && sn < hi) || fabs(creal(ds)) > 0.5 * fabs(dsold)) ds = 0.5 * (lo + hi) - creal(s);
        dsold = creal(ds);
        s += ds;
        if (hi - lo <= 1e-15 * fabs(creal(s))) conv = 1;
    }
    if (!conv) return ORC_EKEPLER;
    for (int it = 0; it < 2; ++it) {
        stumpff_c(beta * s * s, c);
        cplx F = r0 * s * c[1] + u * s * s * c[2] + mu * s * s * s * c[3] - dt;
        cplx Fp = r0 * c[0] + u * s * c[1] + mu * s * s * c[2];
        s -= F / Fp;
    }
    stumpff_c(beta * s * s, c);
    cplx G1 = s * c[1], G2 = s * s * c[2], G3 = s * s * s * c[3];
    cplx r = r0 * c[0] + u * G1 + mu * G2;
    apply_fg_c(st, 1.0 - mu * G2 / r0, dt - mu * G3, -mu * G1 / (r * r0), 1.0 - mu * G2 / r);
    return ORC_OK;
}

static int kepler_drift_c(double mu, double dt, cplx* st)
{
    cplx r0 = csqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2]);
    cplx v2 = st[3] * st[3] + st[4] * st[4] + st[5] * st[5];
    cplx u = st[0] * st[3] + st[1] * st[4] + st[2] * st[5];
    cplx alpha = 2.0 / r0 - v2 / mu;
    if (dt == 0.0) return ORC_OK;
    if (creal(alpha) > 0.0 && creal(r0 * alpha) >= 1e-3) return drift_dE_c(mu, dt, st, r0, u, alpha);
    return drift_univ_c(mu, dt, st, r0, u, alpha);
}

static void particle_accel_c(int np, const double* Gm, const double* pos, const cplx* r, cplx* a)
{
    double h0[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
        const double* rj = pos + 3 * j;
        double rj2 = rj[0] * rj[0] + rj[1] * rj[1] + rj[2] * rj[2];
        double rj3 = rj2 * sqrt(rj2);
        for (int d = 0; d < 3; ++d) h0[d] -= Gm[j] * rj[d] / rj3;
    }
    cplx dir[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
        const double* rj = pos + 3 * j;
        cplx dx = r[0] - rj[0], dy = r[1] - rj[1], dz = r[2] - rj[2];
        cplx d2 = dx * dx + dy * dy + dz * dz;
        cplx d3 = d2 * csqrt(d2);
        dir[0] -= Gm[j] * dx / d3;
        dir[1] -= Gm[j] * dy / d3;
        dir[2] -= Gm[j] * dz / d3;
    }
    for (int d = 0; d < 3; ++d) a[d] = h0[d] + dir[d];
}

/* Tangent map of orc_particles: for each particle, state0 + i h dir through
 * nsteps steps (planet log as in orc_particles, removal tests on the real
 * part).  Outputs the final state (real part), J dir (imaginary part / h),
 * removal step and reason.  A removed particle's derivative is that of its
 * frozen state. */
int orc_particles_jvp(double m0, int np, const double* pmass, const double* log_pos, int64_t nsteps, double dt,
                      const double* rcrit, double rmax, const double* state0, const double* dir, int64_t npart,
                      double* state1, double* jvp, int64_t* removal_step, int32_t* reason, int test_first,
                      int nthreads)
{
    if (np < 0 || np > ORC_MAXP || nsteps < 0 || npart < 0) return ORC_EINVAL;
    const double h = 1e-20;
    double Gm[ORC_MAXP], rc2[ORC_MAXP];
    for (int j = 0; j < np; ++j) { Gm[j] = ORC_G * pmass[j]; rc2[j] = rcrit[j] * rcrit[j]; }
    double rmax2 = rmax > 0.0 ? rmax * rmax : 0.0;
    double mu = ORC_G * m0;
    size_t stride = (size_t)3 * np;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
    for (int64_t p = 0; p < npart; ++p) {
        cplx st[6];
        for (int d = 0; d < 6; ++d) st[d] = state0[6 * p + d] + I * (h * dir[6 * p + d]);
        double mg = INFINITY, cl = INFINITY;
        int64_t rstep = -1;
        int rsn = 0;
        double re[6];
        if (test_first) {
            for (int d = 0; d < 6; ++d) re[d] = creal(st[d]);
            int hh = particle_test(np, log_pos, rc2, rmax2, re, &mg, &cl);
            if (hh) { rstep = 0; rsn = hh; }
        }
        for (int64_t k = 0; k < nsteps && rstep < 0; ++k) {
            const double* P0 = log_pos + (size_t)k * stride;
            const double* P1 = P0 + stride;
            cplx a[3];
            particle_accel_c(np, Gm, P0, st, a);
            for (int d = 0; d < 3; ++d) st[3 + d] += 0.5 * dt * a[d];
            cplx saved[6];
            memcpy(saved, st, sizeof st);
            int rc = kepler_drift_c(mu, dt, st);
            int bad = 0;
            for (int d = 0; d < 6; ++d) if (!isfinite(creal(st[d]))) bad = 1;
            if (rc || bad) {
                memcpy(st, saved, sizeof st);
                rstep = k + 1;
                rsn = rc == ORC_EKEPLER ? RSN_KEPLER : RSN_NONFINITE;
                break;
            }
            for (int d = 0; d < 6; ++d) re[d] = creal(st[d]);
            int hh = particle_test(np, P1, rc2, rmax2, re, &mg, &cl);
            if (hh) { rstep = k + 1; rsn = hh; break; }
            particle_accel_c(np, Gm, P1, st, a);
            for (int d = 0; d < 3; ++d) st[3 + d] += 0.5 * dt * a[d];
        }
        for (int d = 0; d < 6; ++d) {
            state1[6 * p + d] = creal(st[d]);
            jvp[6 * p + d] = cimag(st[d]) / h;
        }
        removal_step[p] = rstep;
        reason[p] = rsn;
    }
    return ORC_OK;
}
#endif /* ORC_OPCOUNT */
