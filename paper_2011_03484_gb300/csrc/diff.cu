// diff.cu -- tangent (forward-mode) and adjoint (reverse-mode) maps of the
// particle map, for gradients of final states with respect to initial states.
//
// The map of one step is K(t_{k+1}, dt/2) o D(dt) o K(t_k, dt/2) with
//   kick  K(tau): v += tau a(r),  a(r) = h0 - sum_j G m_j d_j / |d_j|^3, d_j = r - r_j
//   drift D(dt):  the two-body flow, derivatives in drift_tangent / drift_adjoint (drift_diff.cuh).
// The kick's Jacobian is dv'/dr = tau A(r) with the symmetric tidal matrix
//   tau A w = -sum_j s_j (w - 3 d_j (d_j . w) / |d_j|^2),  s_j = tau G m_j / |d_j|^3,
// so the tangent adds tau A dr to dv and the adjoint adds tau A lv to lr.
// Planet positions are data (no derivative with respect to the planets).
//
// Forward: one thread per particle carries the state and up to kMaxTangents
// tangent vectors through n steps and stores the synchronised state every K
// steps.  Inside a K-step segment the closing half kick of a step and the
// opening half kick of the next use the same planet positions and are one
// kick of dt (their Jacobians, tau A(r) at the same r, merge the same way);
// at a segment boundary and at the end they stay half kicks.  Backward: for each K-step segment from
// the last, the thread recomputes the segment from its checkpoint, keeping the
// pre-drift state, the post-drift position, the solved universal anomaly s,
// the reduced time tau, G_4, G_5 and 1/R of every step in a scratch buffer,
// then runs the adjoint kicks and drifts backwards through it (the other
// G-functions follow from G_4, G_5 by their recurrence: no second solve and no
// second series).
// Tape mode (checkpoint_every = 0) keeps that record for every step of the
// run, written by the forward pass itself: the backward pass is the reverse
// sweep alone, at 112 + 16 N_p B per particle-step of device memory (176 B with
// four planets: 115 GB for 65536 particles over 10^4 steps, which HBM holds).
// The record also keeps the closing kick's s_j and 1/|d_j|^2, so the sweep
// does not evaluate the kick's reciprocals again.
// A removed particle's output is its frozen state; its derivatives are those
// of that frozen state (the steps after removal contribute nothing).
//
// Tangent growth g = log(|J t0| / |t0|): its gradient with respect to the
// initial state needs the second derivative of the map contracted with t0.
// diff_backward_growth_kernel gets it in one reverse sweep of the map extended
// by its tangent (checkpoints of the state and of t), running each kick's and
// drift's adjoint in dual numbers (state (x, t), cotangent (lt, lx));
// diff_growth_kernel gets the part at fixed t0 in forward mode, one thread per
// particle and state coordinate (used in tape mode, and as a cross-check).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "glisse_internal.h"
#include "nvtx_range.h"
#include "drift_diff.cuh"

namespace glisse {
cudaError_t launch_eph_setup(const double*, int, double, double, int, double, PlanetConsts*, double*, int*,
                             cudaStream_t);
cudaError_t launch_eph_chunk(const PlanetConsts*, double*, double, int, double*, double*, int*, cudaStream_t,
                             int* progress = nullptr);

constexpr int kMaxTangents = 6;
constexpr int kScratchRows = 14;  // pre-drift state (6), post-drift position (3), s, tau, G_4, G_5, 1/R
// Rows of one step's record: the kScratchRows of the drift, then the closing kick's
// s_j = tau G m_j / |d_j|^3 and 1/|d_j|^2 (40-bit) for each planet j, which the forward
// pass (or the recompute) forms anyway, so the reverse sweep reads them instead of
// evaluating two reciprocals per planet again.
__host__ __device__ constexpr int record_rows(int np) { return kScratchRows + 2 * np; }
constexpr int kDiffBlock = 128;

struct DiffArgs {
    const double* log;      // [nsteps + 1] planet log steps
    int64_t n;              // particles
    int64_t nsteps;
    int32_t K;              // checkpoint interval
    int32_t ntan;           // tangent vectors (0..kMaxTangents)
    int32_t tape;           // 1: scratch holds every step, written by the forward pass
    int32_t rec_rows;       // rows of one step's record in scratch: record_rows(NP), or
                            // record_rows(NP) + 9 when the tape also keeps tangent 0
    int32_t tan_row;        // first of tangent 0's 9 rows in a record (0: not kept)
    const double* state0;   // [n][6]
    double* state1;         // [n][6]
    const double* tan0;     // [ntan][n][6]
    double* tan1;           // [ntan][n][6]
    double* log_growth;     // [n] log(|J t0| / |t0|) of tangent 0, or null
    int64_t* rstep;         // [n] removal step (-1 live)
    int32_t* reason;        // [n]
    double* ckpt;           // [ceil(nsteps / K)][6][n]
    double* scratch;        // [K][rec_rows][n]
    const double* grad1;    // [n][6]
    double* grad0;          // [n][6]
    // growth indicator of tangent 0 (glisse_diff_backward_growth)
    double* ckpt_t;         // [ceil(nsteps / K)][6][n] tangent 0 at each checkpoint (written by forward)
    const double* gradg;    // [n] cotangent of the growth log(|J t0| / |t0|), or null
    const double* tanN;     // [n][6] J t0 from the forward pass
    double* gradt0;         // [n][6] out: gradient with respect to t0
};

// v += tau a(r) for the log step L; returns the lowest planet index whose encounter test fires.
// rec (optional): a step record (stride ld), which receives s_j and 1/|d_j|^2 of this kick.
template <int NP>
__device__ __forceinline__ int kick_state(double st[6], const double* __restrict__ L, double tau,
                                          const double (&tgm)[kMaxPlanets], const double (&rc2)[kMaxPlanets],
                                          double* rec = nullptr, int64_t ld = 0) {
    const double h0x = L[kRec * NP], h0y = L[kRec * NP + 1], h0z = L[kRec * NP + 2];
    st[3] = fma(tau, h0x, st[3]);
    st[4] = fma(tau, h0y, st[4]);
    st[5] = fma(tau, h0z, st[5]);
    int hit = 0;
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        const double dx = st[0] - L[kRec * j], dy = st[1] - L[kRec * j + 1], dz = st[2] - L[kRec * j + 2];
        const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
        hit = lt_nonneg(d2, rc2[j]) ? (j + 1) : hit;
        const double s = k_rcube(d2, tgm[j]);
        if (rec) {
            rec[(kScratchRows + j) * ld] = s;
            rec[(kScratchRows + NP + j) * ld] = rcp_40(d2);
        }
        st[3] = fma(-s, dx, st[3]);
        st[4] = fma(-s, dy, st[4]);
        st[5] = fma(-s, dz, st[5]);
    }
    return hit;
}

// out += tau A(r) w  (tgm = tau G m_j), A(r) = sum_j -G m_j (I - 3 d d^T / |d|^2) / |d|^3.
// A is symmetric, so the same routine serves the tangent and the adjoint map.
// 1/|d|^2 takes the 40-bit reciprocal: it scales a term that is itself
// ~tau G m_j / |d|^3 (1e-4 or less) of the step's Jacobian.
// Generic over the scalar type: with ad::Dual components (r, dr) and (w, dw) it
// also gives d(tau A(r) w) = tau A(r) dw + tau (dA(r)[dr]) w.
// Planets in kick_state's order (last first), as kick_tangents sums them.
template <int NP, class T>
__device__ __forceinline__ void kick_jac(const T r[3], const double* __restrict__ L,
                                         const double (&tgm)[kMaxPlanets], const T w[3], T out[3]) {
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        const T dx = r[0] - L[kRec * j], dy = r[1] - L[kRec * j + 1], dz = r[2] - L[kRec * j + 2];
        const T d2 = fma(dx, dx, fma(dy, dy, dz * dz));
        const T s = k_rcube(d2, tgm[j]);
        const T c = (3.0 * fma(dx, w[0], fma(dy, w[1], dz * w[2]))) * rcp_40(d2);
        out[0] = fma(-s, fma(-c, dx, w[0]), out[0]);
        out[1] = fma(-s, fma(-c, dy, w[1]), out[1]);
        out[2] = fma(-s, fma(-c, dz, w[2]), out[2]);
    }
}

// kick_state and the tangent's kick_jac in one pass over the planets, sharing the
// separation, |d|^2 and s_j: the velocity v and the tangent's velocity part tv get
// exactly what kick_state and kick_jac give them (same expressions, same order);
// w is the tangent's position part.  Returns what kick_state returns.
template <int NP>
__device__ __forceinline__ int kick_tangent(const double r[3], double v[3], const double w[3], double tv[3],
                                            const double* __restrict__ L, double tau,
                                            const double (&tgm)[kMaxPlanets], const double (&rc2)[kMaxPlanets],
                                            double* rec = nullptr, int64_t ld = 0) {
    const double h0x = L[kRec * NP], h0y = L[kRec * NP + 1], h0z = L[kRec * NP + 2];
    v[0] = fma(tau, h0x, v[0]);
    v[1] = fma(tau, h0y, v[1]);
    v[2] = fma(tau, h0z, v[2]);
    int hit = 0;
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        const double dx = r[0] - L[kRec * j], dy = r[1] - L[kRec * j + 1], dz = r[2] - L[kRec * j + 2];
        const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
        hit = lt_nonneg(d2, rc2[j]) ? (j + 1) : hit;
        const double s = k_rcube(d2, tgm[j]);
        const double inv = rcp_40(d2);
        if (rec) {
            rec[(kScratchRows + j) * ld] = s;
            rec[(kScratchRows + NP + j) * ld] = inv;
        }
        v[0] = fma(-s, dx, v[0]);
        v[1] = fma(-s, dy, v[1]);
        v[2] = fma(-s, dz, v[2]);
        const double c = (3.0 * fma(dx, w[0], fma(dy, w[1], dz * w[2]))) * inv;
        tv[0] = fma(-s, fma(-c, dx, w[0]), tv[0]);
        tv[1] = fma(-s, fma(-c, dy, w[1]), tv[1]);
        tv[2] = fma(-s, fma(-c, dz, w[2]), tv[2]);
    }
    return hit;
}

// kick_jac at the closing kick of a recorded step: s_j and 1/|d_j|^2 come from the
// record (rec: its kick rows, stride ld), the same values kick_jac would form.
template <int NP>
__device__ __forceinline__ void kick_jac_rec(const double r[3], const double* __restrict__ L,
                                             const double* __restrict__ rec, int64_t ld, const double w[3],
                                             double out[3]) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const double dx = r[0] - L[kRec * j], dy = r[1] - L[kRec * j + 1], dz = r[2] - L[kRec * j + 2];
        const double s = rec[j * ld];
        const double c = (3.0 * fma(dx, w[0], fma(dy, w[1], dz * w[2]))) * rec[(NP + j) * ld];
        out[0] = fma(-s, fma(-c, dx, w[0]), out[0]);
        out[1] = fma(-s, fma(-c, dy, w[1]), out[1]);
        out[2] = fma(-s, fma(-c, dz, w[2]), out[2]);
    }
}

// Steps [k_lo, k_hi) of the forward pass for particle i (stopping at a removal): state
// st, tangents t[0..T), removal step / reason, `opened` (the step's opening kick was merged
// into the previous closing kick).  Checkpoints at every multiple of K and the tape
// record of each step are written as the steps pass, so any split of [0, nsteps) into
// consecutive calls does the same arithmetic.
template <int NP, int T, int TA>
__device__ __forceinline__ void forward_steps(const DiffArgs& a, const ParticleConsts& pc, int64_t i, double (&st)[6],
                                              double (&t)[TA][6], int64_t& rstep, int& reason, bool& opened,
                                              int64_t k_lo, int64_t k_hi) {
    const int S = log_stride(NP);
    const bool has_rmax = __double_as_longlong(pc.rmax) != 0;
    for (int64_t k = k_lo; k < k_hi && rstep < 0; ++k) {
        if (k % a.K == 0) {
            double* cp = a.ckpt + (k / a.K) * 6 * a.n;
            for (int c = 0; c < 6; ++c) cp[c * a.n + i] = st[c];
            if (T > 0 && a.ckpt_t) {
                double* ct = a.ckpt_t + (k / a.K) * 6 * a.n;
                for (int c = 0; c < 6; ++c) ct[c * a.n + i] = t[0][c];
            }
        }
        const double* L0 = a.log + k * S;
        const double* L1 = L0 + S;
        // opening half kick (A is evaluated at r, which the kick leaves unchanged)
        if (!opened) {
            if constexpr (T == 1) {
                kick_tangent<NP>(st, st + 3, t[0], t[0] + 3, L0, pc.half_dt, pc.tgm_half, pc.rc2);
            } else {
#pragma unroll
                for (int q = 0; q < T; ++q) kick_jac<NP>(st, L0, pc.tgm_half, t[q], t[q] + 3);
                kick_state<NP>(st, L0, pc.half_dt, pc.tgm_half, pc.rc2);
            }
        }
        double pre[6];
        for (int c = 0; c < 6; ++c) pre[c] = st[c];
        double* tp = a.tape ? a.scratch + k * a.rec_rows * a.n + i : nullptr;
        if (tp)
            for (int c = 0; c < 6; ++c) tp[c * a.n] = pre[c];
        // the tape of the growth gradient's sweep also keeps tangent 0 (before the drift)
        if constexpr (T >= 1)
            if (tp && a.tan_row > 0)
                for (int c = 0; c < 6; ++c) tp[(a.tan_row + c) * a.n] = t[0][c];
        DriftScalars d;
        if (!drift_scalars(pc.mu, pc.dt, pre, d)) {
            rstep = k + 1;
            reason = GLISSE_REMOVED_KEPLER;
            break;
        }
        for (int c = 0; c < 3; ++c) {
            st[c] = fma(d.f, pre[c], d.g * pre[3 + c]);
            st[3 + c] = fma(d.fd, pre[c], d.gd * pre[3 + c]);
        }
        if (tp) {
            for (int c = 0; c < 3; ++c) tp[(6 + c) * a.n] = st[c];
            tp[9 * a.n] = d.s;
            tp[10 * a.n] = d.tau;
            tp[11 * a.n] = d.G[4];
            tp[12 * a.n] = d.G[5];
            tp[13 * a.n] = d.inv_R;
        }
        bool bad = false;
        for (int c = 0; c < 6; ++c) bad |= nonfinite_bits(st[c]);
        if (bad) {
            for (int c = 0; c < 6; ++c) st[c] = pre[c];
            rstep = k + 1;
            reason = GLISSE_REMOVED_NONFINITE;
            break;
        }
#pragma unroll
        for (int q = 0; q < T; ++q) drift_tangent(pc.mu, pre, d, t[q]);
        if constexpr (T >= 1)
            if (tp && a.tan_row > 0)
                for (int c = 0; c < 3; ++c) tp[(a.tan_row + 6 + c) * a.n] = t[0][c];
        // tests at t_{k+1}, then the closing kick (merged with the next opening one
        // inside a segment)
        const bool merge = (k + 1 < a.nsteps) && ((k + 1) % a.K != 0);
        const double tau = merge ? pc.dt : pc.half_dt;
        const double(&tgm)[kMaxPlanets] = merge ? pc.tgm_full : pc.tgm_half;
        const double r2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
        int hit = (has_rmax && lt_nonneg(pc.rmax2, r2)) ? GLISSE_REMOVED_ESCAPE : 0;
        double nst[6], ntv[3];
        for (int c = 0; c < 6; ++c) nst[c] = st[c];
        int enc;
        if constexpr (T == 1) {
            for (int c = 0; c < 3; ++c) ntv[c] = t[0][3 + c];
            enc = kick_tangent<NP>(st, nst + 3, t[0], ntv, L1, tau, tgm, pc.rc2, tp, a.n);
        } else {
            enc = kick_state<NP>(nst, L1, tau, tgm, pc.rc2, tp, a.n);
        }
        hit = enc ? enc : hit;
        if (hit) {
            rstep = k + 1;
            reason = hit;
            break;
        }
        if constexpr (T == 1) {
            for (int c = 0; c < 3; ++c) t[0][3 + c] = ntv[c];
        } else {
#pragma unroll
            for (int q = 0; q < T; ++q) kick_jac<NP>(st, L1, tgm, t[q], t[q] + 3);
        }
        for (int c = 0; c < 6; ++c) st[c] = nst[c];
        opened = merge;
    }
}

// The removal test at t_0 (before the first step).
template <int NP>
__device__ __forceinline__ void forward_test_first(const DiffArgs& a, const ParticleConsts& pc, const double (&st)[6],
                                                   int64_t& rstep, int& reason) {
    const bool has_rmax = __double_as_longlong(pc.rmax) != 0;
    double tmp[6];
    for (int c = 0; c < 6; ++c) tmp[c] = st[c];
    const int hit = kick_state<NP>(tmp, a.log, 0.0, pc.tgm_half, pc.rc2);
    const double r2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
    const int esc = (has_rmax && lt_nonneg(pc.rmax2, r2)) ? GLISSE_REMOVED_ESCAPE : 0;
    if (hit || esc) {
        rstep = 0;
        reason = hit ? hit : esc;
    }
}

// |t0|^2 and |J t0|^2 with explicit fma, exactly as the growth-gradient kernel forms them.
template <int TA>
__device__ __forceinline__ double norm2(const double (&t)[TA][6]) {
    double n = 0.0;
    for (int c = 0; c < 6; ++c) n = fma(t[0][c], t[0][c], n);
    return n;
}

// TMAX: compile-time tangent capacity (0, 1 or kMaxTangents) so that the
// tangent vectors stay in registers; tangents a.ntan..TMAX-1 are zero.
template <int NP, int TMAX>
__global__ void __launch_bounds__(kDiffBlock, TMAX == 0 ? 7 : (TMAX == 1 ? 4 : 1)) diff_forward_kernel(const DiffArgs a, const ParticleConsts pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    constexpr int T = TMAX;
    constexpr int TA = TMAX > 0 ? TMAX : 1;
    double st[6], t[TA][6];
    for (int c = 0; c < 6; ++c) st[c] = a.state0[6 * i + c];
#pragma unroll
    for (int k = 0; k < TA; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) t[k][c] = (k < a.ntan) ? a.tan0[((int64_t)k * a.n + i) * 6 + c] : 0.0;
    const double n0 = norm2<TA>(t);
    int64_t rstep = -1;
    int reason = 0;
    forward_test_first<NP>(a, pc, st, rstep, reason);
    bool opened = false;
    forward_steps<NP, T, TA>(a, pc, i, st, t, rstep, reason, opened, 0, a.nsteps);
    for (int c = 0; c < 6; ++c) a.state1[6 * i + c] = st[c];
#pragma unroll
    for (int q = 0; q < T; ++q)
        if (q < a.ntan)
            for (int c = 0; c < 6; ++c) a.tan1[((int64_t)q * a.n + i) * 6 + c] = t[q][c];
    if (a.log_growth) {
        const double n1 = norm2<TA>(t);
        a.log_growth[i] = (a.ntan > 0 && n0 > 0.0) ? 0.5 * log(n1 / n0) : 0.0;
    }
    a.rstep[i] = rstep;
    a.reason[i] = reason;
}

// Gradient of the tangent-growth indicator g = log(|J t0| / |t0|) with respect
// to the initial state, the seed t0 held fixed: thread (i, c) carries particle
// i's state x, the first-order tangent dx along coordinate c of the initial
// state, and the growth tangent t as dual numbers (t, dt) with
// dt = d(J t0)/dx0 [e_c], through the same steps, kick merging and removals as
// the forward pass.  Then dg/dx0_c = (J t0) . dt / |J t0|^2.
// a.grad0[6 i + c] <- dg/dx0_c; a.log_growth[i] <- g (from the c = 0 thread).
template <int NP>
__global__ void __launch_bounds__(kDiffBlock) diff_growth_kernel(const DiffArgs a, const ParticleConsts pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= a.n) return;
    const int S = log_stride(NP);
    double st[6], dx[6];
    Dual t[6];
    for (int k = 0; k < 6; ++k) {
        st[k] = a.state0[6 * i + k];
        dx[k] = (k == c) ? 1.0 : 0.0;
        t[k] = {a.tan0[6 * i + k], 0.0};
    }
    double n0 = 0.0;
    for (int k = 0; k < 6; ++k) n0 = fma(t[k].v, t[k].v, n0);
    bool removed = false;
    const bool has_rmax = __double_as_longlong(pc.rmax) != 0;
    {
        double tmp[6];
        for (int k = 0; k < 6; ++k) tmp[k] = st[k];
        const int hit = kick_state<NP>(tmp, a.log, 0.0, pc.tgm_half, pc.rc2);
        const double r2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
        removed = hit != 0 || (has_rmax && lt_nonneg(pc.rmax2, r2));
    }
    bool opened = false;
    for (int64_t k = 0; k < a.nsteps && !removed; ++k) {
        const double* L0 = a.log + k * S;
        const double* L1 = L0 + S;
        if (!opened) {
            const Dual rd[3] = {{st[0], dx[0]}, {st[1], dx[1]}, {st[2], dx[2]}};
            kick_jac<NP>(rd, L0, pc.tgm_half, t, t + 3);
            kick_jac<NP>(st, L0, pc.tgm_half, dx, dx + 3);
            kick_state<NP>(st, L0, pc.half_dt, pc.tgm_half, pc.rc2);
        }
        double pre[6], pdx[6];
        for (int q = 0; q < 6; ++q) {
            pre[q] = st[q];
            pdx[q] = dx[q];
        }
        DriftScalars d;
        if (!drift_scalars(pc.mu, pc.dt, pre, d)) {
            removed = true;
            break;
        }
        for (int q = 0; q < 3; ++q) {
            st[q] = fma(d.f, pre[q], d.g * pre[3 + q]);
            st[3 + q] = fma(d.fd, pre[q], d.gd * pre[3 + q]);
        }
        bool bad = false;
        for (int q = 0; q < 6; ++q) bad |= nonfinite_bits(st[q]);
        if (bad) {
            for (int q = 0; q < 6; ++q) st[q] = pre[q];
            removed = true;
            break;
        }
        drift_tangent(pc.mu, pre, d, dx);
        {
            const DriftScalarsT<Dual> e = drift_lift(pc.mu, pre, pdx, d);
            Dual pd[6];
            for (int q = 0; q < 6; ++q) pd[q] = {pre[q], pdx[q]};
            drift_tangent(pc.mu, pd, e, t);
        }
        const bool merge = (k + 1 < a.nsteps) && ((k + 1) % a.K != 0);
        const double tau = merge ? pc.dt : pc.half_dt;
        const double(&tgm)[kMaxPlanets] = merge ? pc.tgm_full : pc.tgm_half;
        const double r2 = fma(st[0], st[0], fma(st[1], st[1], st[2] * st[2]));
        double nst[6];
        for (int q = 0; q < 6; ++q) nst[q] = st[q];
        const int enc = kick_state<NP>(nst, L1, tau, tgm, pc.rc2);
        if (enc != 0 || (has_rmax && lt_nonneg(pc.rmax2, r2))) {
            removed = true;
            break;
        }
        const Dual rd[3] = {{st[0], dx[0]}, {st[1], dx[1]}, {st[2], dx[2]}};
        kick_jac<NP>(rd, L1, tgm, t, t + 3);
        kick_jac<NP>(st, L1, tgm, dx, dx + 3);
        for (int q = 0; q < 6; ++q) st[q] = nst[q];
        opened = merge;
    }
    double n1 = 0.0, p1 = 0.0;
    for (int k = 0; k < 6; ++k) {
        n1 = fma(t[k].v, t[k].v, n1);
        p1 = fma(t[k].v, t[k].d, p1);
    }
    a.grad0[6 * i + c] = n1 > 0.0 ? p1 / n1 : 0.0;
    if (c == 0 && a.log_growth) a.log_growth[i] = (n0 > 0.0 && n1 > 0.0) ? 0.5 * log(n1 / n0) : 0.0;
}

// The backward pass over one checkpoint segment [k0, k1) of particle i (k1 <= kend, its
// removal step or nsteps): recompute the segment from checkpoint cseg into the scratch
// (checkpoint mode; tape mode has the record already), then the adjoint sweep over the
// steps [s_lo, s_hi) of the segment, last step first.  l: cotangent of the state at s_hi
// in, at s_lo out.  The plain launch sweeps whole segments; the task launch cuts the one
// segment of tape mode into sub-chunks.
template <int NP>
__device__ __forceinline__ void backward_piece(const DiffArgs& a, const ParticleConsts& pc, int64_t i,
                                               double (&l)[6], int64_t cseg, int64_t k0, int64_t k1,
                                               int64_t s_lo, int64_t s_hi, int64_t kend, bool cut_after_drift,
                                               bool cut_before_drift) {
    const int S = log_stride(NP);
    double st[6];
    const double* cp = a.ckpt + cseg * 6 * a.n;
    for (int c = 0; c < 6; ++c) st[c] = cp[c * a.n + i];
    // recompute the segment: pre-drift state (6) and post-drift position (3) per step
    // (in tape mode the forward pass wrote them already)
    const int64_t krec = a.tape ? k0 : k1;  // steps to recompute: none in tape mode
    for (int64_t k = k0; k < krec; ++k) {
        const double* L0 = a.log + k * S;
        if (k == k0) kick_state<NP>(st, L0, pc.half_dt, pc.tgm_half, pc.rc2);  // else merged below
        double* sc = a.scratch + (k - k0) * a.rec_rows * a.n + i;
        for (int c = 0; c < 6; ++c) sc[c * a.n] = st[c];
        if (k == kend - 1 && cut_before_drift) break;
        DriftScalars d;
        drift_scalars(pc.mu, pc.dt, st, d);
        sc[9 * a.n] = d.s;
        sc[10 * a.n] = d.tau;
        sc[11 * a.n] = d.G[4];
        sc[12 * a.n] = d.G[5];
        sc[13 * a.n] = d.inv_R;
        double pre[6];
        for (int c = 0; c < 6; ++c) pre[c] = st[c];
        for (int c = 0; c < 3; ++c) {
            st[c] = fma(d.f, pre[c], d.g * pre[3 + c]);
            st[3 + c] = fma(d.fd, pre[c], d.gd * pre[3 + c]);
        }
        for (int c = 0; c < 3; ++c) sc[(6 + c) * a.n] = st[c];
        // closing kick of step k merged with the opening kick of step k + 1 (as in the forward
        // pass); at the segment's end the closing half kick, recorded only
        if (k + 1 < krec) {
            kick_state<NP>(st, a.log + (k + 1) * S, pc.dt, pc.tgm_full, pc.rc2, sc, a.n);
        } else {
            double tmp[6];
            for (int c = 0; c < 6; ++c) tmp[c] = st[c];
            kick_state<NP>(tmp, a.log + (k + 1) * S, pc.half_dt, pc.tgm_half, pc.rc2, sc, a.n);
        }
    }
    // adjoint sweep, last step first
    for (int64_t k = s_hi - 1; k >= s_lo; --k) {
        const double* sc = a.scratch + (k - k0) * a.rec_rows * a.n + i;
        double pre[6], post[3];
        for (int c = 0; c < 6; ++c) pre[c] = sc[c * a.n];
        for (int c = 0; c < 3; ++c) post[c] = sc[(6 + c) * a.n];
        const bool last = (k == kend - 1);
        if (!(last && (cut_after_drift || cut_before_drift))) {
            // closing kick at t_{k+1}: lr += tau A(post) lv, tau = dt inside the segment
            // (merged with the opening kick of step k + 1), dt/2 at its end; its s_j and
            // 1/|d_j|^2 are in the step's record
            kick_jac_rec<NP>(post, a.log + (k + 1) * S, sc + kScratchRows * a.n, a.n, l + 3, l);
        }
        if (!(last && cut_before_drift)) {
            DriftScalars d;
            drift_restore(pc.mu, pc.dt, pre, sc[9 * a.n], sc[10 * a.n], d);
            drift_finish_stored(pc.mu, d, sc[11 * a.n], sc[12 * a.n], sc[13 * a.n]);
            drift_adjoint(pc.mu, pre, d, l);
        }
        // opening half kick at t_k (only at the segment start; inside, it is part of
        // the previous step's merged closing kick): lr += (dt/2) A(pre) lv
        if (k == k0) kick_jac<NP>(pre, a.log + k * S, pc.tgm_half, l + 3, l);
    }
}

template <int NP>
__global__ void __launch_bounds__(kDiffBlock, 4) diff_backward_kernel(const DiffArgs a, const ParticleConsts pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double l[6];
    for (int c = 0; c < 6; ++c) l[c] = a.grad1[6 * i + c];
    const int64_t rstep = a.rstep[i];
    const int reason = a.reason[i];
    const int64_t kend = rstep >= 0 ? rstep : a.nsteps;  // steps the particle took (last one maybe partial)
    // the last step of a removed particle stops after the drift (encounter / escape)
    // or before it (Kepler failure / non-finite)
    const bool cut_after_drift = rstep > 0 && reason != GLISSE_REMOVED_KEPLER && reason != GLISSE_REMOVED_NONFINITE;
    const bool cut_before_drift = rstep > 0 && !cut_after_drift;
    if (kend > 0) {
        const int64_t nseg = (kend + a.K - 1) / a.K;
        for (int64_t cseg = nseg - 1; cseg >= 0; --cseg) {
            const int64_t k0 = cseg * a.K;
            const int64_t k1 = min(k0 + (int64_t)a.K, kend);
            backward_piece<NP>(a, pc, i, l, cseg, k0, k1, k0, k1, kend, cut_after_drift, cut_before_drift);
        }
    }
    for (int c = 0; c < 6; ++c) a.grad0[6 * i + c] = l[c];
}

// Task launch of the backward pass (the particle map's task launch, applied to the
// sweep): every warp of the plain launch does the same work, so it lasts as long as the
// SM partition holding the most warps (65536 particles: 2048 warps over 608 partitions,
// 3 or 4 each).  Here a fixed grid of warps takes (32-particle group, sub-chunk) tasks
// in order from a counter, the last sub-chunk of the run first; a sub-chunk is a
// checkpoint segment, or kTapeSub steps of the one segment of tape mode.  The cotangent
// passes between a group's tasks through grad0 (exact doubles), and a task waits,
// bounded, for the group's previous one: the result equals the plain launch bit for bit.
constexpr int kTapeSub = 64;
constexpr int kDiffWaitPolls = 1 << 25;

struct DiffTaskArgs {
    int64_t sub;                       // steps per sub-chunk
    int32_t n_groups;                  // ceil(n / 32)
    int32_t n_sub;                     // sub-chunks of the run
    unsigned long long* task_counter;  // zero before the launch
    int32_t* group_done;               // [n_groups] sub-chunks finished, zero before the launch
    int* status;                       // GLISSE_E_TIMEOUT if a wait gives up
    int32_t wait_polls;                // polls before a wait gives up; 0: the default (seconds)
};

__device__ __forceinline__ int diff_ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void diff_st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int NP>
__global__ void __launch_bounds__(kDiffBlock, 4) diff_backward_tasks_kernel(const DiffArgs a, const ParticleConsts pc,
                                                                            const DiffTaskArgs ta) {
    const int lane = threadIdx.x & 31;
    const int64_t n_tasks = (int64_t)ta.n_groups * ta.n_sub;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ta.task_counter, 1ull);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if ((int64_t)t >= n_tasks) break;
        const int64_t g = (int64_t)t % ta.n_groups;
        const int r = (int)((int64_t)t / ta.n_groups);  // 0: the last sub-chunk of the run
        if (r > 0) {
            int ok = 1;
            if (lane == 0) {
                const int limit = ta.wait_polls > 0 ? ta.wait_polls : kDiffWaitPolls;
                int polls = 0;
                while (diff_ld_acquire(ta.group_done + g) < r && ++polls < limit) __nanosleep(64);
                ok = polls < limit;
            }
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(ta.status, GLISSE_E_TIMEOUT);
                break;
            }
        }
        __syncwarp();
        const int64_t i = g * 32 + lane;
        if (i < a.n) {
            double l[6];
            // the first task reads the cotangent given, later ones the one their group left
            // (written by another warp's task: read through L2)
            for (int c = 0; c < 6; ++c) l[c] = r == 0 ? a.grad1[6 * i + c] : __ldcg(a.grad0 + 6 * i + c);
            const int64_t rstep = a.rstep[i];
            const int reason = a.reason[i];
            const int64_t kend = rstep >= 0 ? rstep : a.nsteps;
            const bool cut_after_drift =
                rstep > 0 && reason != GLISSE_REMOVED_KEPLER && reason != GLISSE_REMOVED_NONFINITE;
            const bool cut_before_drift = rstep > 0 && !cut_after_drift;
            const int64_t c_idx = ta.n_sub - 1 - r;
            const int64_t lo = c_idx * ta.sub;
            const int64_t hi = min(lo + ta.sub, kend);
            if (hi > lo) {
                if (a.tape)
                    backward_piece<NP>(a, pc, i, l, 0, 0, kend, lo, hi, kend, cut_after_drift, cut_before_drift);
                else
                    backward_piece<NP>(a, pc, i, l, c_idx, lo, hi, lo, hi, kend, cut_after_drift, cut_before_drift);
            }
            for (int c = 0; c < 6; ++c) __stcg(a.grad0 + 6 * i + c, l[c]);
        }
        // every lane's stores before the group's counter moves on (release at device scope)
        __threadfence();
        __syncwarp();
        if (lane == 0) diff_st_release(ta.group_done + g, r + 1);
    }
}

// Task launch of the forward pass (no tangent or one): tasks (32-particle group, sub-chunk
// of kFwdSub steps) forward in time, the first sub-chunk first.  Between a group's tasks the
// state, tangent, removal step and reason pass through state1 / tan1 / rstep / reason (read
// through L2), |t0|^2 through log_growth; checkpoints and the tape are written as the steps
// pass.  The arithmetic is forward_steps', so the outputs equal the plain launch's bit for bit.
constexpr int kFwdSub = 64;

template <int NP, int TMAX>
__global__ void __launch_bounds__(kDiffBlock, 4) diff_forward_tasks_kernel(const DiffArgs a, const ParticleConsts pc,
                                                                           const DiffTaskArgs ta) {
    constexpr int T = TMAX;
    constexpr int TA = TMAX > 0 ? TMAX : 1;
    const int lane = threadIdx.x & 31;
    const int64_t n_tasks = (int64_t)ta.n_groups * ta.n_sub;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ta.task_counter, 1ull);
        tk = __shfl_sync(0xFFFFFFFFu, tk, 0);
        if ((int64_t)tk >= n_tasks) break;
        const int64_t g = (int64_t)tk % ta.n_groups;
        const int sidx = (int)((int64_t)tk / ta.n_groups);
        if (sidx > 0) {
            int ok = 1;
            if (lane == 0) {
                const int limit = ta.wait_polls > 0 ? ta.wait_polls : kDiffWaitPolls;
                int polls = 0;
                while (diff_ld_acquire(ta.group_done + g) < sidx && ++polls < limit) __nanosleep(64);
                ok = polls < limit;
            }
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(ta.status, GLISSE_E_TIMEOUT);
                break;
            }
        }
        __syncwarp();
        const int64_t i = g * 32 + lane;
        if (i < a.n) {
            double st[6], t[TA][6];
            int64_t rstep = -1;
            int reason = 0;
            if (sidx == 0) {
                for (int c = 0; c < 6; ++c) st[c] = a.state0[6 * i + c];
#pragma unroll
                for (int q = 0; q < TA; ++q)
#pragma unroll
                    for (int c = 0; c < 6; ++c) t[q][c] = (q < a.ntan) ? a.tan0[((int64_t)q * a.n + i) * 6 + c] : 0.0;
                if (a.log_growth) a.log_growth[i] = norm2<TA>(t);  // |t0|^2, until the last task
                forward_test_first<NP>(a, pc, st, rstep, reason);
            } else {
                for (int c = 0; c < 6; ++c) st[c] = __ldcg(a.state1 + 6 * i + c);
#pragma unroll
                for (int q = 0; q < TA; ++q)
#pragma unroll
                    for (int c = 0; c < 6; ++c)
                        t[q][c] = (q < a.ntan) ? __ldcg(a.tan1 + ((int64_t)q * a.n + i) * 6 + c) : 0.0;
                rstep = (int64_t)__ldcg(reinterpret_cast<const long long*>(a.rstep + i));
                reason = __ldcg(a.reason + i);
            }
            const int64_t lo = (int64_t)sidx * ta.sub;
            const int64_t hi = min(lo + ta.sub, a.nsteps);
            // inside a checkpoint segment the previous step's closing kick opened this one
            bool opened = lo > 0 && lo < a.nsteps && lo % a.K != 0;
            forward_steps<NP, T, TA>(a, pc, i, st, t, rstep, reason, opened, lo, hi);
            for (int c = 0; c < 6; ++c) __stcg(a.state1 + 6 * i + c, st[c]);
#pragma unroll
            for (int q = 0; q < T; ++q)
                if (q < a.ntan)
                    for (int c = 0; c < 6; ++c) __stcg(a.tan1 + ((int64_t)q * a.n + i) * 6 + c, t[q][c]);
            __stcg(reinterpret_cast<long long*>(a.rstep + i), (long long)rstep);
            __stcg(a.reason + i, reason);
            if (sidx + 1 == ta.n_sub && a.log_growth) {
                const double n0 = __ldcg(a.log_growth + i);
                const double n1 = norm2<TA>(t);
                a.log_growth[i] = (a.ntan > 0 && n0 > 0.0) ? 0.5 * log(n1 / n0) : 0.0;
            }
        }
        // every lane's stores before the group's counter moves on (release at device scope)
        __threadfence();
        __syncwarp();
        if (lane == 0) diff_st_release(ta.group_done + g, sidx + 1);
    }
}

// Scratch rows of the extended recompute: the kScratchRows of the plain one,
// then tangent 0 before the drift (6) and its position part after the drift (3).
constexpr int kScratchRowsG = kScratchRows + 9;

// One reverse sweep of the map extended by its tangent, z = (x, t) with
// t_{k+1} = M_k(x_k) t_k, for the cotangent (lx, lt) = (grad_state1,
// grad_growth (J t0) / |J t0|^2) at the end.  Each piece (kick, drift) runs its
// adjoint in dual numbers: state (x, t), cotangent (lt, lx) -> (M^T lt,
// (dM[t])^T lt + M^T lx); see drift_adjoint.  Segments are recomputed from the
// state and tangent checkpoints, as the plain backward pass does, or, with
// GLISSE_DIFF_TAPE_TANGENT, read from the forward call's record of every step.
// a.grad0 <- lx at t_0 (= J^T grad_state1 + grad_growth dg/dstate0 at fixed t0);
// a.gradt0 <- lt at t_0 minus grad_growth t0 / |t0|^2 (= dg/dt0 times grad_growth).
template <int NP>
__global__ void __launch_bounds__(kDiffBlock, 2) diff_backward_growth_kernel(const DiffArgs a, const ParticleConsts pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int S = log_stride(NP);
    const double gg = a.gradg ? a.gradg[i] : 0.0;
    double nn = 0.0;
    for (int c = 0; c < 6; ++c) nn = fma(a.tanN[6 * i + c], a.tanN[6 * i + c], nn);
    const double w = nn > 0.0 ? gg / nn : 0.0;
    Dual l[6];
    for (int c = 0; c < 6; ++c) l[c] = {w * a.tanN[6 * i + c], a.grad1 ? a.grad1[6 * i + c] : 0.0};
    const int64_t rstep = a.rstep[i];
    const int reason = a.reason[i];
    const int64_t kend = rstep >= 0 ? rstep : a.nsteps;
    const bool cut_after_drift = rstep > 0 && reason != GLISSE_REMOVED_KEPLER && reason != GLISSE_REMOVED_NONFINITE;
    const bool cut_before_drift = rstep > 0 && !cut_after_drift;
    // records: the tape (tangent 0 kept beside the state's rows) or the segment's recompute
    const int64_t rows = a.tape ? a.rec_rows : kScratchRowsG;
    const int trow = a.tape ? a.tan_row : kScratchRows;
    if (kend > 0) {
        const int64_t nseg = (kend + a.K - 1) / a.K;
        for (int64_t cseg = nseg - 1; cseg >= 0; --cseg) {
            const int64_t k0 = cseg * a.K;
            const int64_t k1 = min(k0 + (int64_t)a.K, kend);
            const int64_t krec = a.tape ? k0 : k1;  // steps to recompute: none with a tape
            double st[6], t[6];
            const double* cp = a.ckpt + cseg * 6 * a.n;
            const double* ct = a.ckpt_t + cseg * 6 * a.n;
            for (int c = 0; c < 6; ++c) {
                st[c] = cp[c * a.n + i];
                t[c] = ct[c * a.n + i];
            }
            for (int64_t k = k0; k < krec; ++k) {
                const double* L0 = a.log + k * S;
                if (k == k0) {
                    kick_jac<NP>(st, L0, pc.tgm_half, t, t + 3);
                    kick_state<NP>(st, L0, pc.half_dt, pc.tgm_half, pc.rc2);
                }
                double* sc = a.scratch + (k - k0) * rows * a.n + i;
                for (int c = 0; c < 6; ++c) {
                    sc[c * a.n] = st[c];
                    sc[(trow + c) * a.n] = t[c];
                }
                if (k == kend - 1 && cut_before_drift) break;
                DriftScalars d;
                drift_scalars(pc.mu, pc.dt, st, d);
                sc[9 * a.n] = d.s;
                sc[10 * a.n] = d.tau;
                sc[11 * a.n] = d.G[4];
                sc[12 * a.n] = d.G[5];
                sc[13 * a.n] = d.inv_R;
                double pre[6];
                for (int c = 0; c < 6; ++c) pre[c] = st[c];
                for (int c = 0; c < 3; ++c) {
                    st[c] = fma(d.f, pre[c], d.g * pre[3 + c]);
                    st[3 + c] = fma(d.fd, pre[c], d.gd * pre[3 + c]);
                }
                drift_tangent(pc.mu, pre, d, t);
                for (int c = 0; c < 3; ++c) {
                    sc[(6 + c) * a.n] = st[c];
                    sc[(trow + 6 + c) * a.n] = t[c];
                }
                if (k + 1 < k1) {
                    kick_jac<NP>(st, a.log + (k + 1) * S, pc.tgm_full, t, t + 3);
                    kick_state<NP>(st, a.log + (k + 1) * S, pc.dt, pc.tgm_full, pc.rc2);
                }
            }
            for (int64_t k = k1 - 1; k >= k0; --k) {
                const double* sc = a.scratch + (k - k0) * rows * a.n + i;
                double pre[6];
                Dual pd[6], qd[3];
                for (int c = 0; c < 6; ++c) {
                    pre[c] = sc[c * a.n];
                    pd[c] = {pre[c], sc[(trow + c) * a.n]};
                }
                for (int c = 0; c < 3; ++c) qd[c] = {sc[(6 + c) * a.n], sc[(trow + 6 + c) * a.n]};
                const bool last = (k == kend - 1);
                if (!(last && (cut_after_drift || cut_before_drift)))
                    kick_jac<NP>(qd, a.log + (k + 1) * S, (k + 1 < k1) ? pc.tgm_full : pc.tgm_half, l + 3, l);
                if (!(last && cut_before_drift)) {
                    DriftScalars d;
                    drift_restore(pc.mu, pc.dt, pre, sc[9 * a.n], sc[10 * a.n], d);
                    drift_finish_stored(pc.mu, d, sc[11 * a.n], sc[12 * a.n], sc[13 * a.n]);
                    const double tp[6] = {pd[0].d, pd[1].d, pd[2].d, pd[3].d, pd[4].d, pd[5].d};
                    const DriftScalarsT<Dual> e = drift_lift(pc.mu, pre, tp, d);
                    drift_adjoint(pc.mu, pd, e, l);
                }
                if (k == k0) kick_jac<NP>(pd, a.log + k * S, pc.tgm_half, l + 3, l);
            }
        }
    }
    double n0 = 0.0, t0[6];
    for (int c = 0; c < 6; ++c) {
        t0[c] = a.ckpt_t[c * a.n + i];
        n0 = fma(t0[c], t0[c], n0);
    }
    const double w0 = n0 > 0.0 ? gg / n0 : 0.0;
    for (int c = 0; c < 6; ++c) {
        a.grad0[6 * i + c] = l[c].d;
        a.gradt0[6 * i + c] = fma(-w0, t0[c], l[c].v);
    }
}

#define GLISSE_DIFF_SWITCH(KERNEL)                                         \
    switch (np) {                                                          \
        case 0: KERNEL<0><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 1: KERNEL<1><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 2: KERNEL<2><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 3: KERNEL<3><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 4: KERNEL<4><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 5: KERNEL<5><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 6: KERNEL<6><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 7: KERNEL<7><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        case 8: KERNEL<8><<<grid, kDiffBlock, 0, s>>>(a, pc); break;       \
        default: return cudaErrorInvalidValue;                             \
    }

template <int TMAX>
static cudaError_t launch_diff_forward_t(int np, const DiffArgs& a, const ParticleConsts& pc, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.n + kDiffBlock - 1) / kDiffBlock);
    switch (np) {
#define GLISSE_FWD_CASE(N) \
    case N: diff_forward_kernel<N, TMAX><<<grid, kDiffBlock, 0, s>>>(a, pc); break;
        GLISSE_FWD_CASE(0)
        GLISSE_FWD_CASE(1)
        GLISSE_FWD_CASE(2)
        GLISSE_FWD_CASE(3)
        GLISSE_FWD_CASE(4)
        GLISSE_FWD_CASE(5)
        GLISSE_FWD_CASE(6)
        GLISSE_FWD_CASE(7)
        GLISSE_FWD_CASE(8)
#undef GLISSE_FWD_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Blocks of four warps per SM for a task launch over `groups` 32-particle groups, or 0 for
// the plain launch: the groups must outnumber the resident warps by half again (so that a
// task's predecessor has nearly always finished when it is taken), with two blocks per SM
// at least (one warp per partition leaves the FP64 pipe ~30% idle) and at most four.
static int diff_task_blocks(int64_t groups, int nsm, bool force) {
    const int64_t k = (2 * groups) / (3 * 4 * (int64_t)nsm);
    if (k >= 2) return (int)std::min<int64_t>(k, 4);
    return force ? 2 : 0;
}

template <int TMAX>
static cudaError_t launch_diff_forward_tasks(int np, const DiffArgs& a, const ParticleConsts& pc, cudaStream_t s,
                                             const DiffTaskArgs& b, int k, int nsm) {
    const unsigned grid = (unsigned)(k * nsm);
    size_t smem = 0;
    cudaError_t e = cudaSuccess;
    switch (np) {
#define GLISSE_FWDT_CASE(N)                                                                                  \
    case N:                                                                                                  \
        e = residency_cap_smem(reinterpret_cast<const void*>(diff_forward_tasks_kernel<N, TMAX>), k, 4, &smem); \
        if (e != cudaSuccess) return e;                                                                      \
        diff_forward_tasks_kernel<N, TMAX><<<grid, kDiffBlock, smem, s>>>(a, pc, b);                         \
        break;
        GLISSE_FWDT_CASE(0)
        GLISSE_FWDT_CASE(1)
        GLISSE_FWDT_CASE(2)
        GLISSE_FWDT_CASE(3)
        GLISSE_FWDT_CASE(4)
        GLISSE_FWDT_CASE(5)
        GLISSE_FWDT_CASE(6)
        GLISSE_FWDT_CASE(7)
        GLISSE_FWDT_CASE(8)
#undef GLISSE_FWDT_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// tb: task buffers, or null for the plain launch; force_tasks: the task launch whatever the
// size (GLISSE_LAUNCH_TASKS).  The task launch carries no tangent or one (six keep the
// plain launch, one block per SM).
static cudaError_t launch_diff_forward(int np, const DiffArgs& a, const ParticleConsts& pc, cudaStream_t s,
                                       const DiffTaskArgs* tb = nullptr, bool force_tasks = false) {
    if (a.n <= 0) return cudaSuccess;
    if (tb && a.ntan <= 1) {
        int dev = 0, nsm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int64_t groups = (a.n + 31) / 32;
        const int k = diff_task_blocks(groups, nsm, force_tasks);
        if (k > 0) {
            DiffTaskArgs b = *tb;
            b.sub = kFwdSub;
            b.n_groups = (int32_t)groups;
            b.n_sub = (int32_t)std::max<int64_t>((a.nsteps + b.sub - 1) / b.sub, 1);
            e = cudaMemsetAsync(b.task_counter, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(b.group_done, 0, sizeof(int32_t) * (size_t)groups, s);
            if (e != cudaSuccess) return e;
            return a.ntan == 0 ? launch_diff_forward_tasks<0>(np, a, pc, s, b, k, nsm)
                               : launch_diff_forward_tasks<1>(np, a, pc, s, b, k, nsm);
        }
    }
    if (a.ntan == 0) return launch_diff_forward_t<0>(np, a, pc, s);
    if (a.ntan == 1) return launch_diff_forward_t<1>(np, a, pc, s);
    return launch_diff_forward_t<kMaxTangents>(np, a, pc, s);
}

// tb: task buffers (counter, group counters, status), or null for the plain launch.
// force_tasks: the task launch whatever the size (GLISSE_LAUNCH_TASKS).
static cudaError_t launch_diff_backward(int np, const DiffArgs& a, const ParticleConsts& pc, cudaStream_t s,
                                        const DiffTaskArgs* tb, bool force_tasks) {
    if (a.n <= 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t groups = (a.n + 31) / 32;
    const int k = tb ? diff_task_blocks(groups, nsm, force_tasks) : 0;
    if (k > 0) {
        DiffTaskArgs b = *tb;
        b.sub = a.tape ? kTapeSub : a.K;
        b.n_groups = (int32_t)groups;
        b.n_sub = (int32_t)((a.nsteps + b.sub - 1) / b.sub);
        if (b.n_sub == 0) b.n_sub = 1;
        e = cudaMemsetAsync(b.task_counter, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.group_done, 0, sizeof(int32_t) * (size_t)groups, s);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)(k * nsm);
        size_t smem = 0;
        switch (np) {
#define GLISSE_DIFF_TCASE(N)                                                                                 \
    case N:                                                                                                  \
        e = residency_cap_smem(reinterpret_cast<const void*>(diff_backward_tasks_kernel<N>), k, 4, &smem);   \
        if (e != cudaSuccess) return e;                                                                      \
        diff_backward_tasks_kernel<N><<<grid, kDiffBlock, smem, s>>>(a, pc, b);                              \
        break;
            GLISSE_DIFF_TCASE(0)
            GLISSE_DIFF_TCASE(1)
            GLISSE_DIFF_TCASE(2)
            GLISSE_DIFF_TCASE(3)
            GLISSE_DIFF_TCASE(4)
            GLISSE_DIFF_TCASE(5)
            GLISSE_DIFF_TCASE(6)
            GLISSE_DIFF_TCASE(7)
            GLISSE_DIFF_TCASE(8)
#undef GLISSE_DIFF_TCASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const unsigned grid = (unsigned)((a.n + kDiffBlock - 1) / kDiffBlock);
    GLISSE_DIFF_SWITCH(diff_backward_kernel)
    return cudaGetLastError();
}

static cudaError_t launch_diff_backward_growth(int np, const DiffArgs& a, const ParticleConsts& pc,
                                               cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.n + kDiffBlock - 1) / kDiffBlock);
    GLISSE_DIFF_SWITCH(diff_backward_growth_kernel)
    return cudaGetLastError();
}

static cudaError_t launch_diff_growth(int np, const DiffArgs& a, const ParticleConsts& pc, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((a.n + kDiffBlock - 1) / kDiffBlock), 6);
    GLISSE_DIFF_SWITCH(diff_growth_kernel)
    return cudaGetLastError();
}

// Self-test of the bounded waits of the task launches (which = 1: forward pass, 2: reverse
// sweep).  Two groups, two sub-chunks; the task counter starts past the first sub-chunk of
// both groups, so each task handed out waits for a sub-chunk that no task runs: its warp
// gives up after `polls` polls, sets *status to GLISSE_E_TIMEOUT and leaves before touching
// a particle (the other warps find no task left).  scratch: zeroed device memory holding
// the task counter (8 bytes) and the groups' counters (8 bytes); the particle arrays point
// at it too, never read.
cudaError_t diff_wait_selftest(int which, int polls, char* scratch, int* status, cudaStream_t s) {
    constexpr int kGroups = 2;
    double* d = reinterpret_cast<double*>(scratch);
    DiffArgs a{};
    a.log = d;
    a.n = 32 * kGroups;
    a.K = 1 << 20;
    a.state0 = d;
    a.state1 = d;
    a.rstep = reinterpret_cast<int64_t*>(scratch);
    a.reason = reinterpret_cast<int32_t*>(scratch);
    a.ckpt = d;
    a.scratch = d;
    a.grad1 = d;
    a.grad0 = d;
    DiffTaskArgs ta{};
    ta.n_groups = kGroups;
    ta.n_sub = 2;
    ta.task_counter = reinterpret_cast<unsigned long long*>(scratch);
    ta.group_done = reinterpret_cast<int32_t*>(scratch + 8);
    ta.status = status;
    ta.wait_polls = polls;
    const unsigned long long first = kGroups;
    cudaError_t e = cudaMemcpyAsync(ta.task_counter, &first, sizeof(first), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (which == 1) {
        ta.sub = kFwdSub;
        a.nsteps = 2 * kFwdSub;
        diff_forward_tasks_kernel<0, 0><<<4, kDiffBlock, 0, s>>>(a, ParticleConsts{}, ta);
    } else {
        ta.sub = kTapeSub;
        a.nsteps = 2 * kTapeSub;
        a.tape = 1;
        diff_backward_tasks_kernel<0><<<4, kDiffBlock, 0, s>>>(a, ParticleConsts{}, ta);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace glisse

using namespace glisse;

struct glisse_diff {
    int device = 0;
    int np = 0;
    int64_t n = 0, nsteps = 0;
    int K = 256;
    bool tape = false;      // checkpoint_every = 0: the forward pass records every step
    bool tan_tape = false;  // GLISSE_DIFF_TAPE_TANGENT: the record also keeps tangent 0
    ParticleConsts pc{};
    double* d_log = nullptr;
    double* d_ckpt = nullptr;
    double* d_scratch = nullptr;
    double* d_ckpt_t = nullptr;     // tangent 0 at each checkpoint
    double* d_scratch_g = nullptr;  // extended recompute (glisse_diff_backward_growth), on first use
    int64_t* d_rstep = nullptr;
    int32_t* d_reason = nullptr;
    // task launch of the backward pass: counter (8 B), status (4 B, padded), [ceil(n / 32)] group counters
    char* d_tasks = nullptr;
    int launch_mode = GLISSE_LAUNCH_AUTO;
    bool have_forward = false;
    int32_t last_ntan = 0;
};

static void diff_free(glisse_diff* d) {
    if (!d) return;
    void* ptrs[] = {d->d_log,   d->d_ckpt,   d->d_scratch, d->d_ckpt_t,
                    d->d_scratch_g, d->d_rstep, d->d_reason, d->d_tasks};
    for (void* p : ptrs) cudaFree(p);
    delete d;
}

extern "C" void glisse_diff_destroy(glisse_diff* d) { diff_free(d); }

// Rows of one step's record: the drift's, the closing kick's, and with
// GLISSE_DIFF_TAPE_TANGENT tangent 0's 9 (before the drift, and its position after).
static int32_t rec_rows(const glisse_diff* d) { return record_rows(d->np) + (d->tan_tape ? 9 : 0); }

static void set_record_layout(const glisse_diff* d, DiffArgs& a) {
    a.rec_rows = rec_rows(d);
    a.tan_row = d->tan_tape ? record_rows(d->np) : 0;
}

extern "C" int glisse_diff_checkpoint_every(glisse_diff* d, int32_t* checkpoint_every) {
    if (!d || !checkpoint_every) return GLISSE_E_INVAL;
    *checkpoint_every = d->tan_tape ? GLISSE_DIFF_TAPE_TANGENT : d->tape ? 0 : d->K;
    return GLISSE_OK;
}

#define GD_CUDA(x)                    \
    do {                              \
        cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) {      \
            (void)cudaGetLastError(); \
            rc = GLISSE_E_CUDA;       \
            goto fail;                \
        }                             \
    } while (0)

extern "C" int glisse_diff_create(glisse_diff** out, double star_mass, const double* planets, int32_t n_planets,
                                  int64_t n_particles, double dt, int64_t n_steps, int32_t checkpoint_every,
                                  const glisse_opts* opts) {
    glisse::NvtxRange range("glisse_diff_create");
    if (!out) return GLISSE_E_INVAL;
    *out = nullptr;
    glisse_opts o;
    glisse_opts_default(&o);
    if (opts) o = *opts;
    if (!(star_mass > 0.0) || n_planets < 0 || n_planets > GLISSE_MAX_PLANETS || (n_planets > 0 && !planets) ||
        n_particles < 0 || n_steps < 0 || n_steps > INT32_MAX || !(dt != 0.0) || !std::isfinite(dt) ||
        checkpoint_every < GLISSE_DIFF_TAPE_TANGENT)
        return GLISSE_E_INVAL;
    // derivatives are of the converged drift only
    if (o.kepler_mode != GLISSE_KEPLER_CONVERGE || o.sort_mode != GLISSE_SORT_NONE) return GLISSE_E_INVAL;
    if (o.launch_mode < GLISSE_LAUNCH_AUTO || o.launch_mode > GLISSE_LAUNCH_TASKS) return GLISSE_E_INVAL;
    for (int64_t k = 0; k < 7 * (int64_t)n_planets; ++k)
        if (!std::isfinite(planets[k])) return GLISSE_E_INVAL;
    glisse_diff* d = new (std::nothrow) glisse_diff();
    if (!d) return GLISSE_E_NOMEM;
    int rc = GLISSE_OK;
    const double G = 4.0 * 3.14159265358979323846 * 3.14159265358979323846;
    const int S = log_stride(n_planets);
    double* d_pl = nullptr;
    double* d_jac = nullptr;
    PlanetConsts* d_pc = nullptr;
    int* d_status = nullptr;
    PlanetConsts hpc;
    int status = 0;
    d->np = n_planets;
    d->n = n_particles;
    d->nsteps = n_steps;
    d->launch_mode = o.launch_mode;
    if (checkpoint_every == GLISSE_DIFF_AUTO) {
        // the per-step record when it fits in half of the free device memory
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = GLISSE_E_CUDA;
            goto fail;
        }
        const double tape_b = 8.0 * record_rows(n_planets) * (double)std::max<int64_t>(n_particles, 1) *
                              (double)std::max<int64_t>(n_steps, 1);
        checkpoint_every = tape_b <= 0.5 * (double)free_b ? 0 : 256;
    }
    d->tan_tape = checkpoint_every == GLISSE_DIFF_TAPE_TANGENT;
    d->tape = checkpoint_every == 0 || d->tan_tape;
    d->K = d->tape ? (int32_t)std::max<int64_t>(std::min<int64_t>(n_steps, INT32_MAX), 1) : checkpoint_every;
    if (d->tape && n_steps > INT32_MAX) {
        rc = GLISSE_E_INVAL;
        goto fail;
    }
    if (cudaGetDevice(&d->device) != cudaSuccess) {
        rc = GLISSE_E_CUDA;
        goto fail;
    }
    {
        const int64_t nck = std::max<int64_t>((n_steps + d->K - 1) / d->K, 1);
        const int64_t np1 = std::max<int64_t>(n_particles, 1);
        if (cudaMalloc(&d->d_log, sizeof(double) * (size_t)(n_steps + 1) * S) != cudaSuccess ||
            cudaMalloc(&d->d_ckpt, sizeof(double) * (size_t)nck * 6 * np1) != cudaSuccess ||
            cudaMalloc(&d->d_ckpt_t, sizeof(double) * (size_t)nck * 6 * np1) != cudaSuccess ||
            cudaMalloc(&d->d_scratch, sizeof(double) * (size_t)d->K * rec_rows(d) * np1) != cudaSuccess ||
            cudaMalloc(&d->d_rstep, sizeof(int64_t) * np1) != cudaSuccess ||
            cudaMalloc(&d->d_reason, sizeof(int32_t) * np1) != cudaSuccess ||
            cudaMalloc(&d->d_tasks, 16 + sizeof(int32_t) * (size_t)((np1 + 31) / 32)) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = GLISSE_E_NOMEM;
            goto fail;
        }
    }
    GD_CUDA(cudaMalloc(&d_pl, sizeof(double) * 7 * std::max(n_planets, 1)));
    GD_CUDA(cudaMalloc(&d_jac, sizeof(double) * 6 * std::max(n_planets, 1)));
    GD_CUDA(cudaMalloc(&d_pc, sizeof(PlanetConsts)));
    GD_CUDA(cudaMalloc(&d_status, sizeof(int)));
    if (n_planets > 0) GD_CUDA(cudaMemcpy(d_pl, planets, sizeof(double) * 7 * n_planets, cudaMemcpyHostToDevice));
    GD_CUDA(launch_eph_setup(d_pl, n_planets, star_mass, G, o.enc_mode, o.enc_value, d_pc, d_jac, d_status, 0));
    GD_CUDA(cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        rc = status;
        goto fail;
    }
    // planet log for the whole run (the ephemeris is serial in time)
    GD_CUDA(launch_eph_chunk(d_pc, d_jac, dt, (int)n_steps, d->d_log, nullptr, d_status, 0));
    GD_CUDA(cudaMemcpy(&hpc, d_pc, sizeof(PlanetConsts), cudaMemcpyDeviceToHost));
    GD_CUDA(cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        rc = status;
        goto fail;
    }
    std::memset(&d->pc, 0, sizeof(d->pc));
    d->pc.mu = hpc.mu0;
    d->pc.dt = dt;
    d->pc.half_dt = 0.5 * dt;
    for (int j = 0; j < n_planets; ++j) {
        d->pc.tgm_full[j] = dt * hpc.gm[j];
        d->pc.tgm_half[j] = 0.5 * dt * hpc.gm[j];
        d->pc.rc2[j] = hpc.rcrit[j] * hpc.rcrit[j];
    }
    d->pc.rmax2 = o.r_max > 0.0 ? o.r_max * o.r_max : 0.0;
    d->pc.rmax = o.r_max > 0.0 ? o.r_max : 0.0;
    cudaFree(d_pl);
    cudaFree(d_jac);
    cudaFree(d_pc);
    cudaFree(d_status);
    *out = d;
    return GLISSE_OK;
fail:
    cudaFree(d_pl);
    cudaFree(d_jac);
    cudaFree(d_pc);
    cudaFree(d_status);
    diff_free(d);
    return rc;
}

extern "C" int glisse_diff_forward(glisse_diff* d, const double* state0, double* state1, int32_t n_tangents,
                                   const double* tangent0, double* tangent1, double* log_growth,
                                   int64_t* removal_step, int32_t* removal_reason, void* stream) {
    glisse::NvtxRange range("glisse_diff_forward");
    if (!d || n_tangents < 0 || n_tangents > kMaxTangents) return GLISSE_E_INVAL;
    if (d->n > 0 && (!state0 || !state1)) return GLISSE_E_INVAL;
    if (n_tangents > 0 && (!tangent0 || !tangent1)) return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DiffArgs a{};
    a.log = d->d_log;
    a.n = d->n;
    a.nsteps = d->nsteps;
    a.K = d->K;
    a.tape = d->tape ? 1 : 0;
    set_record_layout(d, a);
    a.scratch = d->d_scratch;
    a.ntan = n_tangents;
    a.state0 = state0;
    a.state1 = state1;
    a.tan0 = tangent0;
    a.tan1 = tangent1;
    a.log_growth = log_growth;
    a.rstep = d->d_rstep;
    a.reason = d->d_reason;
    a.ckpt = d->d_ckpt;
    a.ckpt_t = d->d_ckpt_t;
    DiffTaskArgs tb{};
    tb.task_counter = reinterpret_cast<unsigned long long*>(d->d_tasks);
    tb.status = reinterpret_cast<int*>(d->d_tasks + 8);
    tb.group_done = reinterpret_cast<int32_t*>(d->d_tasks + 16);
    int status = 0;
    cudaError_t e = cudaMemsetAsync(tb.status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_diff_forward(d->np, a, d->pc, s, d->launch_mode == GLISSE_LAUNCH_PLAIN ? nullptr : &tb,
                                d->launch_mode == GLISSE_LAUNCH_TASKS);
    if (e == cudaSuccess && removal_step && d->n > 0)
        e = cudaMemcpyAsync(removal_step, d->d_rstep, sizeof(int64_t) * d->n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && removal_reason && d->n > 0)
        e = cudaMemcpyAsync(removal_reason, d->d_reason, sizeof(int32_t) * d->n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, tb.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    if (status != 0) return status;
    d->have_forward = true;
    d->last_ntan = n_tangents;
    return GLISSE_OK;
}

extern "C" int glisse_diff_backward(glisse_diff* d, const double* grad_state1, double* grad_state0, void* stream) {
    glisse::NvtxRange range("glisse_diff_backward");
    if (!d) return GLISSE_E_INVAL;
    if (!d->have_forward) return GLISSE_E_STATE;
    if (d->n > 0 && (!grad_state1 || !grad_state0)) return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DiffArgs a{};
    a.log = d->d_log;
    a.n = d->n;
    a.nsteps = d->nsteps;
    a.K = d->K;
    a.tape = d->tape ? 1 : 0;
    set_record_layout(d, a);
    a.rstep = d->d_rstep;
    a.reason = d->d_reason;
    a.ckpt = d->d_ckpt;
    a.scratch = d->d_scratch;
    a.grad1 = grad_state1;
    a.grad0 = grad_state0;
    DiffTaskArgs tb{};
    tb.task_counter = reinterpret_cast<unsigned long long*>(d->d_tasks);
    tb.status = reinterpret_cast<int*>(d->d_tasks + 8);
    tb.group_done = reinterpret_cast<int32_t*>(d->d_tasks + 16);
    int status = 0;
    cudaError_t e = cudaMemsetAsync(tb.status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_diff_backward(d->np, a, d->pc, s, d->launch_mode == GLISSE_LAUNCH_PLAIN ? nullptr : &tb,
                                 d->launch_mode == GLISSE_LAUNCH_TASKS);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, tb.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    return status == 0 ? GLISSE_OK : status;
}

extern "C" int glisse_diff_backward_growth(glisse_diff* d, const double* grad_state1, const double* grad_growth,
                                           const double* tangent1, double* grad_state0, double* grad_tangent0,
                                           void* stream) {
    glisse::NvtxRange range("glisse_diff_backward_growth");
    if (!d) return GLISSE_E_INVAL;
    if (!d->have_forward || d->last_ntan < 1 || (d->tape && !d->tan_tape)) return GLISSE_E_STATE;
    if (d->n > 0 && (!tangent1 || !grad_state0 || !grad_tangent0)) return GLISSE_E_INVAL;
    if (!d->tape && !d->d_scratch_g && d->n > 0) {
        const size_t bytes = sizeof(double) * (size_t)d->K * kScratchRowsG * (size_t)d->n;
        if (cudaMalloc(&d->d_scratch_g, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            d->d_scratch_g = nullptr;
            return GLISSE_E_NOMEM;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DiffArgs a{};
    a.log = d->d_log;
    a.n = d->n;
    a.nsteps = d->nsteps;
    a.K = d->K;
    a.rstep = d->d_rstep;
    a.reason = d->d_reason;
    a.ckpt = d->d_ckpt;
    a.ckpt_t = d->d_ckpt_t;
    a.tape = d->tape ? 1 : 0;
    set_record_layout(d, a);
    a.scratch = d->tape ? d->d_scratch : d->d_scratch_g;  // the forward call's record, or the recompute's
    a.grad1 = grad_state1;
    a.gradg = grad_growth;
    a.tanN = tangent1;
    a.grad0 = grad_state0;
    a.gradt0 = grad_tangent0;
    cudaError_t e = launch_diff_backward_growth(d->np, a, d->pc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    return GLISSE_OK;
}

extern "C" int glisse_diff_growth_gradient(glisse_diff* d, const double* state0, const double* tangent0,
                                           double* grad_state0, double* log_growth, void* stream) {
    glisse::NvtxRange range("glisse_diff_growth_gradient");
    if (!d) return GLISSE_E_INVAL;
    if (d->n > 0 && (!state0 || !tangent0 || !grad_state0)) return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DiffArgs a{};
    a.log = d->d_log;
    a.n = d->n;
    a.nsteps = d->nsteps;
    a.K = d->K;
    a.state0 = state0;
    a.tan0 = tangent0;
    a.grad0 = grad_state0;
    a.log_growth = log_growth;
    cudaError_t e = launch_diff_growth(d->np, a, d->pc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    return GLISSE_OK;
}
