// ephemeris.cu -- the planets: set-up and the chunked Wisdom-Holman map (section 2.2).
//
// The paper integrates the planets with the standard mixed-variable
// symplectic (Wisdom-Holman) map in Jacobi coordinates, a chunk of steps
// ahead of the particles, and ships the heliocentric positions plus the
// common indirect term h0 = -sum_j G m_j r_j / |r_j|^3 for every step.
// Here that runs on the GPU in one block of two warps on a side stream, one
// chunk ahead of the particle kernel: warp 0 steps the planets (its lanes are
// planet rows x 4 columns, so each pair interaction is computed once, in
// parallel lanes), warp 1 -- on another SM partition -- turns every step's
// synchronised state into the log records, h0 and the heliocentric history.
//
// Jacobi coordinates (commented equations after Eq. 2 of the paper), planets
// i = 1..N_p (lane i-1), star 0:
//   eta_i = m0 + m_1 + ... + m_i
//   r'_i = r_i - sum_{k<i} m_k r_k / eta_{i-1}        (helio -> Jacobi)
//   r_i  = r'_i + sum_{k<i} (m_k / eta_k) r'_k         (Jacobi -> helio)
// Kepler part of H: sum_i p'_i^2 / 2m'_i - G m0 m_i / |r'_i| with
//   m'_i = m_i eta_{i-1} / eta_i, i.e. a Kepler drift with mu_i = G m0 eta_i / eta_{i-1}.
// Interaction part: H_int = sum_i G m0 m_i (1/|r'_i| - 1/|r_i|) - sum_{i<j} G m_i m_j / |r_i - r_j|.
// Its kick, by the chain rule through r(r'):
//   dv'_k/dt = -(eta_k / eta_{k-1}) [ -G m0 r'_k / |r'_k|^3 + ghat_k + S_k / eta_k ]
//   ghat_i = G m0 r_i / |r_i|^3 + sum_{j != i} G m_j (r_i - r_j) / |r_i - r_j|^3
//   S_k = sum_{i > k} m_i ghat_i
#include "glisse_internal.h"
#include "kepler.cuh"

namespace glisse {

// Scans over the first n lanes (n <= 32, warp-uniform).  Lanes >= n must hold 0.
// exclusive prefix: sum over lanes k < lane
__device__ __forceinline__ double warp_excl_prefix(double v, int lane, int n) {
    double incl = v;
    for (int o = 1; o < n; o <<= 1) {
        const double t = __shfl_up_sync(kFullMask, incl, o);
        if (lane >= o) incl += t;
    }
    return incl - v;
}

// exclusive suffix: sum over lanes k > lane (k < n)
__device__ __forceinline__ double warp_excl_suffix(double v, int lane, int n) {
    double incl = v;
    for (int o = 1; o < n; o <<= 1) {
        const double t = __shfl_down_sync(kFullMask, incl, o);
        if (lane + o < n) incl += t;
    }
    return incl - v;
}

// total over lanes < n, valid in lane 0
__device__ __forceinline__ double warp_total0(double v, int lane, int n) {
    return warp_excl_suffix(v, lane, n) + v;
}

// ---------------------------------------------------------------------------
// Set-up: constants, Jacobi state, encounter radii.  One warp.
//   planets : [np][7] heliocentric m, x, y, z, vx, vy, vz (device copy)
//   jac     : out [2][np][3]: Jacobi positions then Jacobi velocities
//   status  : out 0, or GLISSE_E_INVAL (unbound planet, or not ordered by a)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) eph_setup_kernel(const double* __restrict__ planets, int np, double m0, double G,
                                                         int enc_mode, double enc_value, PlanetConsts* pc,
                                                         double* jac, int* status) {
    const int lane = threadIdx.x;
    const bool on = lane < np;
    const double m = on ? planets[7 * lane] : 0.0;
    double r[3], v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r[d] = on ? planets[7 * lane + 1 + d] : 0.0;
        v[d] = on ? planets[7 * lane + 4 + d] : 0.0;
    }
    // eta_i for this lane's planet (inclusive) and eta_{i-1}
    const double eta_prev = m0 + warp_excl_prefix(m, lane, 32);
    const double eta_i = eta_prev + m;
    double q[3], w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double mr = warp_excl_prefix(m * r[d], lane, 32);
        const double mv = warp_excl_prefix(m * v[d], lane, 32);
        q[d] = r[d] - mr / eta_prev;
        w[d] = v[d] - mv / eta_prev;
    }
    // initial osculating heliocentric semi-major axis with mu = G (m0 + m_j)
    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double inva = 2.0 / rn - v2 / (G * (m0 + m));
    const bool bound = inva > 0.0;
    const double a = 1.0 / inva;
    const double rcrit = (enc_mode == GLISSE_ENC_FIXED) ? enc_value : enc_value * a * cbrt(m / (3.0 * m0));
    // ordering by increasing a
    const double a_prev = __shfl_up_sync(kFullMask, a, 1);
    const bool order_ok = (lane == 0) || !(a <= a_prev);
    const unsigned bad = __ballot_sync(kFullMask, on && (!bound || !order_ok || !isfinite(rcrit)));
    if (on) {
        pc->m[lane] = m;
        pc->eta[lane + 1] = eta_i;
        pc->mu_jac[lane] = G * m0 * eta_i / eta_prev;
        pc->gm[lane] = G * m;
        pc->rcrit[lane] = rcrit;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            jac[3 * lane + d] = q[d];
            jac[3 * np + 3 * lane + d] = w[d];
        }
    }
    if (lane == 0) {
        pc->np = np;
        pc->m0 = m0;
        pc->G = G;
        pc->mu0 = G * m0;
        pc->eta[0] = m0;
        *status = bad ? GLISSE_E_INVAL : 0;
    }
}

// ---------------------------------------------------------------------------
// The chunked Wisdom-Holman step of the planets.
//
// A GPU FP64 instruction of a warp costs the same whatever its active lanes,
// and one warp steps the planets serially, so the time of a step is the
// number of FP64 instructions on its critical path.  Two things shorten it:
//   * warp 0 holds planet i in the four lanes 4i .. 4i + 3 (replicated), and
//     lane 4i + c also handles the interaction with planet j = c (and
//     c + 4 for 5 to 8 planets): the N_p^2 pair terms, the positions' Jacobi
//     prefix sums and the suffix sums of the kick are each one lane-parallel
//     term plus a two-stage butterfly within the row;
//   * what only the log needs -- h0, the heliocentric velocities, the stores
//     and the progress count -- runs on warp 1 from a double-buffered
//     shared-memory hand-off, ordered by named barriers.
// Each step is open half kick, Kepler drift of every Jacobi body, positions,
// kick terms, closing half kick, identically at every step, so the planet
// sequence does not depend on where chunks begin.
// ---------------------------------------------------------------------------
constexpr int kEphThreads = 64;  // warp 0: dynamics, warp 1: log records
constexpr int kEphCols = 4;      // lanes per planet row in warp 0

// named barriers of the hand-off ring: FULL slot b = 1 + b, EMPTY slot b = 3 + b
__device__ __forceinline__ void eph_bar_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kEphThreads) : "memory");
}
__device__ __forceinline__ void eph_bar_arrive(int id) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "n"(kEphThreads) : "memory");
}

struct EphRing {
    double r[2][kMaxPlanets][3];  // heliocentric positions of the emitted step
    double w[2][kMaxPlanets][3];  // synchronised Jacobi velocities
};

// Sum over the four lanes of a planet row (every lane of the row gets the same bits).
__device__ __forceinline__ double row_sum(double v) {
    v += __shfl_xor_sync(kFullMask, v, 1);
    v += __shfl_xor_sync(kFullMask, v, 2);
    return v;
}

// Warp 0: positions r from the Jacobi positions q of every row (r_i = q_i + sum_{k<i} m_k/eta_k q_k).
template <int H>
__device__ __forceinline__ void eph_positions(const double (&moe)[2], const bool (&below)[2], const double q[3],
                                              double r[3], int col) {
    double p[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int src = kEphCols * (col + kEphCols * h);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double qj = __shfl_sync(kFullMask, q[d], src);
            p[d] = fma(below[h] ? moe[h] : 0.0, qj, p[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) r[d] = q[d] + row_sum(p[d]);
}

// Warp 0: Jacobi acceleration of the row's planet at heliocentric positions r.
//   ghat_i = G m0 r_i / |r_i|^3 + sum_{j != i} G m_j (r_i - r_j) / |r_i - r_j|^3  (lane-parallel over j)
//   S_k    = sum_{i > k} m_i ghat_i                                             (lane-parallel over i)
//   acc_k  = -(eta_k / eta_{k-1}) [ghat_k + S_k / eta_k - G m0 q_k / |q_k|^3]
template <int H>
__device__ __forceinline__ void eph_accel(const PlanetConsts& pc, bool on, int row, int col, const double (&kj)[2],
                                          const bool (&valid)[2], const double (&mi)[2], const bool (&above)[2],
                                          double inv_eta, double ratio, const double q[3], double qr,
                                          const double r[3], double acc[3]) {
    double t[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int j = col + kEphCols * h;
        const int src = kEphCols * j;
        const bool self = j == row;
        double dv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double rj = __shfl_sync(kFullMask, r[d], src);
            dv[d] = r[d] - (self ? 0.0 : rj);
        }
        const double d2 = fma(dv[0], dv[0], fma(dv[1], dv[1], dv[2] * dv[2]));
        const double sc = k_rcube(valid[h] ? d2 : 1.0, kj[h]);
#pragma unroll
        for (int d = 0; d < 3; ++d) t[d] = fma(sc, dv[d], t[d]);
    }
    double gh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gh[d] = row_sum(t[d]);
    double sv[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int src = kEphCols * (col + kEphCols * h);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double gi = __shfl_sync(kFullMask, gh[d], src);
            sv[d] = fma(above[h] ? mi[h] : 0.0, gi, sv[d]);
        }
    }
    // |q|^2 from the radius the drift leaves (or radius_of at a chunk's start: the same expression)
    const double iq3 = k_rcube(on ? qr * qr : 1.0, pc.mu0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double S = row_sum(sv[d]);
        const double grad = fma(S, inv_eta, fma(-iq3, q[d], gh[d]));
        acc[d] = on ? -ratio * grad : 0.0;
    }
}

// Warp 0 of the block: nsteps steps from the Jacobi state `jac` (in place), each step's
// synchronised state handed to warp 1.  status: GLISSE_E_KEPLER if a planet's drift fails.
template <int H>
__device__ __forceinline__ void eph_dynamics(const PlanetConsts& pc, double* jac, double dt, int nsteps, EphRing& ring,
                                             int* status) {
    const int np = pc.np;
    const int lane = threadIdx.x & 31;
    const int row = lane / kEphCols, col = lane % kEphCols;
    const bool on = row < np;
    double q[3], w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        q[d] = on ? jac[3 * row + d] : (d == 0 ? 1.0 + row : 0.0);
        w[d] = on ? jac[3 * np + 3 * row + d] : 0.0;
    }
    const double inv_eta = on ? 1.0 / pc.eta[row + 1] : 1.0;
    const double ratio = on ? pc.eta[row + 1] / pc.eta[row] : 1.0;
    const double mu = on ? pc.mu_jac[row] : pc.mu0;
    const float muf = d2f_bits(mu), dtf = d2f_bits(dt);
    const double hdt = 0.5 * dt;
    // per column j = col + 4h: m_j / eta_j for the positions (j < row), the kick's G-coefficient
    // (G m0 on the diagonal, G m_j off it), m_j for the suffix sums (j > row)
    double moe[2], kj[2], mi[2];
    bool below[2], valid[2], above[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = col + kEphCols * h;
        const bool jon = h < H && j < np;
        moe[h] = jon ? pc.m[j] / pc.eta[j + 1] : 0.0;
        below[h] = jon && on && j < row;
        valid[h] = jon && on;
        kj[h] = valid[h] ? (j == row ? pc.mu0 : pc.gm[j]) : 0.0;
        mi[h] = jon ? pc.m[j] : 0.0;
        above[h] = jon && on && j > row;
    }
    double r[3], acc[3];
    // |q| and mu/|q| of the Jacobi position: here from the position, then carried from each
    // drift (which forms them from the new position with the same expression)
    double qr, qmur;
    radius_of(q[0], q[1], q[2], qr, qmur);
    qmur *= mu;
    eph_positions<H>(moe, below, q, r, col);
    eph_accel<H>(pc, on, row, col, kj, valid, mi, above, inv_eta, ratio, q, qr, r, acc);
    if (on && col == 0)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ring.r[0][row][d] = r[d];
            ring.w[0][row][d] = w[d];
        }
    eph_bar_arrive(1);
    bool failed = false;
    for (int k = 0; k < nsteps; ++k) {
        // opening half kick, Kepler drift of each Jacobi body
#pragma unroll
        for (int d = 0; d < 3; ++d) w[d] = fma(hdt, acc[d], w[d]);
        const bool done = drift_fast(mu, muf, dt, dtf, on, qr, qmur, q[0], q[1], q[2], w[0], w[1], w[2]);
        if (on && !done) {
            if (!drift_general(mu, dt, q[0], q[1], q[2], w[0], w[1], w[2])) failed = true;
            radius_of(q[0], q[1], q[2], qr, qmur);
            qmur *= mu;
        }
        eph_positions<H>(moe, below, q, r, col);
        eph_accel<H>(pc, on, row, col, kj, valid, mi, above, inv_eta, ratio, q, qr, r, acc);
        // closing half kick: synchronised state at t_{k+1}
#pragma unroll
        for (int d = 0; d < 3; ++d) w[d] = fma(hdt, acc[d], w[d]);
        const int e = k + 1, b = e & 1;
        if (e >= 2) eph_bar_sync(3 + b);  // warp 1 is done with emitted step e - 2
        if (on && col == 0)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ring.r[b][row][d] = r[d];
                ring.w[b][row][d] = w[d];
            }
        eph_bar_arrive(1 + b);
    }
    // wait for warp 1 to finish the last emitted steps
    for (int e = nsteps > 0 ? nsteps - 1 : 0; e <= nsteps; ++e) eph_bar_sync(3 + (e & 1));
    if (on && col == 0)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            jac[3 * row + d] = q[d];
            jac[3 * np + 3 * row + d] = w[d];
        }
    if (__any_sync(kFullMask, failed) && lane == 0) *status = GLISSE_E_KEPLER;
}

// Warp 1 of the block: for each emitted step e = 0..nsteps, log record e (positions + h0,
// broadcast layout) and the synchronised heliocentric states hist[e][np][6].
// progress (optional, host-mapped): after every kProgressEvery-th step and the last, the
// number of steps whose log entries are written, published with a system-scope fence so
// that the host may launch work on them while this runs.
__device__ __forceinline__ void eph_emit(const PlanetConsts& pc, int nsteps, const EphRing& ring,
                                         double* __restrict__ log, double* __restrict__ hist, int* progress) {
    const int np = pc.np;
    const int lane = threadIdx.x & 31;
    const bool on = lane < np;
    const int S = log_stride(np);
    const double gm = on ? pc.gm[lane] : 0.0;
    const double m_over_eta = on ? pc.m[lane] / pc.eta[lane + 1] : 0.0;
    for (int e = 0; e <= nsteps; ++e) {
        const int b = e & 1;
        eph_bar_sync(1 + b);
        double r[3], w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r[d] = on ? ring.r[b][lane][d] : 0.0;
            w[d] = on ? ring.w[b][lane][d] : 0.0;
        }
        eph_bar_arrive(3 + b);  // the ring slot may be refilled
        // h0 = -sum_j G m_j r_j / |r_j|^3
        const double r2 = on ? fma(r[0], r[0], fma(r[1], r[1], r[2] * r[2])) : 1.0;
        const double own = k_rcube(r2, gm);
        double h0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) h0[d] = -warp_total0(own * r[d], lane, np);
        double* L = log + (size_t)e * S;
        if (on) {
            L[kRec * lane + 0] = r[0];
            L[kRec * lane + 1] = r[1];
            L[kRec * lane + 2] = r[2];
            L[kRec * lane + 3] = 0.0;
        }
        if (lane == 0) {
            L[kRec * np + 0] = h0[0];
            L[kRec * np + 1] = h0[1];
            L[kRec * np + 2] = h0[2];
            L[kRec * np + 3] = 0.0;
        }
        if (hist) {  // the same pointer on every lane: the warp takes this branch together
            double* Hs = hist + (size_t)e * 6 * np;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double vh = w[d] + warp_excl_prefix(m_over_eta * w[d], lane, np);
                if (on) {
                    Hs[6 * lane + d] = r[d];
                    Hs[6 * lane + 3 + d] = vh;
                }
            }
        }
        if (progress && e > 0 && ((e % kProgressEvery) == 0 || e == nsteps)) {
            __threadfence_system();  // every lane's log entries before the count
            __syncwarp();
            if (lane == 0) *reinterpret_cast<volatile int*>(progress) = e;
        }
    }
}

__device__ __forceinline__ void eph_advance(const PlanetConsts& pc, double* jac, double dt, int nsteps,
                                            double* __restrict__ log, double* __restrict__ hist, int* status,
                                            int* progress = nullptr) {
    __shared__ EphRing ring;
    if (threadIdx.x < 32) {
        if (pc.np > kEphCols)
            eph_dynamics<2>(pc, jac, dt, nsteps, ring, status);
        else
            eph_dynamics<1>(pc, jac, dt, nsteps, ring, status);
    } else {
        eph_emit(pc, nsteps, ring, log, hist, progress);
    }
}

__global__ void __launch_bounds__(kEphThreads) eph_chunk_kernel(const PlanetConsts* __restrict__ pcp, double* jac,
                                                                  double dt, int nsteps, double* __restrict__ log,
                                                                  double* __restrict__ hist, int* status,
                                                                  int* progress) {
    eph_advance(*pcp, jac, dt, nsteps, log, hist, status, progress);
}

// Many independent systems: block b advances system b.
//   jac  : [n_sys][2][kMaxPlanets][3] Jacobi states (per-system stride 6 kMaxPlanets)
//   log  : system b's log at log + log_off[b] (stride 4 (np_b + 1) doubles per step)
//   dt   : [n_sys] steps
__global__ void __launch_bounds__(kEphThreads) eph_batch_kernel(const PlanetConsts* __restrict__ pcs, double* jac,
                                                                  const double* __restrict__ dt, int nsteps,
                                                                  double* __restrict__ log,
                                                                  const int64_t* __restrict__ log_off, int* status) {
    const int b = blockIdx.x;
    eph_advance(pcs[b], jac + (size_t)b * 6 * kMaxPlanets, dt[b], nsteps, log + log_off[b], nullptr, status);
}

// ---------------------------------------------------------------------------
// External positions -> log layout with h0.  One thread per step.
//   pos : [n+1][np][3] heliocentric positions
// ---------------------------------------------------------------------------
__global__ void eph_external_kernel(const PlanetConsts* __restrict__ pcp, const double* __restrict__ pos, int64_t n1,
                                    double* __restrict__ log) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n1) return;
    const int np = pcp->np;
    const int S = log_stride(np);
    double hx = 0.0, hy = 0.0, hz = 0.0;
    for (int j = 0; j < np; ++j) {
        const double x = pos[(k * np + j) * 3 + 0], y = pos[(k * np + j) * 3 + 1], z = pos[(k * np + j) * 3 + 2];
        const double r2 = fma(x, x, fma(y, y, z * z));
        const double s = k_rcube(r2, pcp->gm[j]);
        hx = fma(-s, x, hx);
        hy = fma(-s, y, hy);
        hz = fma(-s, z, hz);
        log[k * S + kRec * j + 0] = x;
        log[k * S + kRec * j + 1] = y;
        log[k * S + kRec * j + 2] = z;
        log[k * S + kRec * j + 3] = 0.0;
    }
    log[k * S + kRec * np + 0] = hx;
    log[k * S + kRec * np + 1] = hy;
    log[k * S + kRec * np + 2] = hz;
    log[k * S + kRec * np + 3] = 0.0;
}

// host launchers ----------------------------------------------------------------
cudaError_t launch_eph_setup(const double* planets, int np, double m0, double G, int enc_mode, double enc_value,
                             PlanetConsts* pc, double* jac, int* status, cudaStream_t s) {
    eph_setup_kernel<<<1, 32, 0, s>>>(planets, np, m0, G, enc_mode, enc_value, pc, jac, status);
    return cudaGetLastError();
}

// The ephemeris is one serial block of two warps.  Sharing an SM partition
// with particle warps would slow it by the number of warps it shares the FP64
// pipe with, so its block asks for the largest dynamic shared-memory
// allocation a block may have: no other block fits on that SM while it runs
// (the memory is unused).  The particle grids are sized for the other SMs.
// In steady state the planets run a chunk ahead and the reservation changes
// nothing measurable (the step time agreed to 0.01% without it); it matters
// in the first chunk of a context, where the particles follow the planets a
// few steps behind and a slowed ephemeris would hold them back.
cudaError_t launch_eph_chunk(const PlanetConsts* pc, double* jac, double dt, int nsteps, double* log, double* hist,
                             int* status, cudaStream_t s, int* progress) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, eph_chunk_kernel);
    // all of a block's shared memory: the kernel's own hand-off ring plus the rest as dynamic
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (e == cudaSuccess && dyn < 0) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eph_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    eph_chunk_kernel<<<1, kEphThreads, (size_t)dyn, s>>>(pc, jac, dt, nsteps, log, hist, status, progress);
    return cudaGetLastError();
}

cudaError_t launch_eph_batch(const PlanetConsts* pcs, int n_sys, double* jac, const double* dt, int nsteps,
                             double* log, const int64_t* log_off, int* status, cudaStream_t s) {
    if (n_sys <= 0) return cudaSuccess;
    eph_batch_kernel<<<n_sys, kEphThreads, 0, s>>>(pcs, jac, dt, nsteps, log, log_off, status);
    return cudaGetLastError();
}

cudaError_t launch_eph_external(const PlanetConsts* pc, const double* pos, int64_t n1, double* log, cudaStream_t s) {
    const int bs = 128;
    const int64_t grid = (n1 + bs - 1) / bs;
    eph_external_kernel<<<(unsigned)grid, bs, 0, s>>>(pc, pos, n1, log);
    return cudaGetLastError();
}

}  // namespace glisse
