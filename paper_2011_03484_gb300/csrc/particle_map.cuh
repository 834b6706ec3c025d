// particle_map.cuh -- the test-particle map over one segment of a planet chunk
// (shared by the translation units that instantiate it for each drift mode).
//
// Section 2.2: one thread per particle; the particle is loaded once, carried
// in registers through every step of the chunk, and stored once.  Each step
// is kick(dt/2) - Kepler drift(dt) - kick(dt/2) with the kick
//   dv/dt = h0 - sum_j G m_j (r - r_j) / |r - r_j|^3,  h0 = -sum_j G m_j r_j / |r_j|^3,
// and the removal test (encounter |r - r_j| < R_crit,j, escape |r| > r_max)
// made at every kick time on the drifted position.  Inside a segment the
// closing half kick of step k and the opening half kick of step k+1 use the
// same planet positions, so they are applied as one kick of dt.  A context's
// segments end "open": the last step ends with the same full kick that an
// uncut launch would apply there, the stored velocities already carry the
// next step's opening half kick, and the next segment skips it (open_in /
// close_out = 0).  Cuts then leave no trace: any split of a run into calls,
// pieces or sample stops gives the same bits.  The synchronised state the
// caller reads (velocities with only the closing half kick) is computed at
// the cut by one extra half kick from the same pre-kick velocities and
// written by id (publish).  close_out = 1 ends with the closing half kick
// instead, leaving the synchronised state in the slots (batched systems).
//
// The batched kernel may hold one particle in a lane pair (TPP = 2): both
// lanes run the same state and drift, each takes half of the planets in the
// kick, and the pair adds its two partial kicks (kick_test_pair).
//
// A removed particle keeps the state it had after the drift and before the
// closing kick, gets removal_step = k+1 and the reason (planet 1..N_p, lowest
// index first; encounter before escape), and its lane idles until the warp
// finishes or compaction drops it.  A failed Kepler solve or a non-finite
// result keeps the state from before the drift (reasons -2 / -3).
#pragma once
#include <algorithm>
#include "glisse_internal.h"
#include "kepler.cuh"

namespace glisse {

constexpr int kParticleBlock = 128;
// Resident blocks per SM the particle kernel is compiled for (register budget
// 65536 / (128 x blocks)).  A chunk's warps all do the same work, so a launch
// that spills past one wave leaves a tail in which a lone warp per SM
// partition cannot keep the FP64 pipe busy.
#ifndef GLISSE_PARTICLE_MIN_BLOCKS
#define GLISSE_PARTICLE_MIN_BLOCKS 8
#endif

// drift used by the particle map: the converged fast solver (default) or the
// paper's fixed-iteration solve (GLISSE_KEPLER_PAPER_FIXED)
constexpr int kDriftConverge = 0;
constexpr int kDriftPaper = 1;

// Read-only broadcast load of one 32-byte log record.
__device__ __forceinline__ void load_rec(const double* __restrict__ p, double& x, double& y, double& z) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    x = a.x;
    y = a.y;
    z = __ldg(p + 2);
}

// Kick with the log step L by tau (tgm[j] = tau G m_j), and the encounter test.
// Returns the lowest 1-based planet index whose test fires, or 0.
template <int NP>
__device__ __forceinline__ int kick_test(double x, double y, double z, double& vx, double& vy, double& vz,
                                         const double* __restrict__ L, double tau, const double (&tgm)[kMaxPlanets],
                                         const double (&rc2)[kMaxPlanets]) {
    double hx, hy, hz;
    load_rec(L + kRec * NP, hx, hy, hz);
    vx = fma(tau, hx, vx);
    vy = fma(tau, hy, vy);
    vz = fma(tau, hz, vz);
    int hit = 0;
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        double px, py, pz;
        load_rec(L + kRec * j, px, py, pz);
        const double dx = x - px, dy = y - py, dz = z - pz;
        const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
        hit = lt_nonneg(d2, rc2[j]) ? (j + 1) : hit;
        const double s = k_rcube(d2, tgm[j]);
        vx = fma(-s, dx, vx);
        vy = fma(-s, dy, vy);
        vz = fma(-s, dz, vz);
    }
    return hit;
}

// kick_test with the planets split over a lane pair (two lanes per particle,
// both holding the same state): lane parity p takes planets p, p + 2, ...,
// each lane sums its partial kick, and the pair adds the two partial sums (the
// same sum on both lanes: addition commutes) and takes the lower encounter
// index.  The h0 term is applied by both lanes as in kick_test.
template <int NP>
__device__ __forceinline__ int kick_test_pair(double x, double y, double z, double& vx, double& vy, double& vz,
                                              const double* __restrict__ L, double tau,
                                              const double (&tgm)[kMaxPlanets], const double (&rc2)[kMaxPlanets]) {
    const int parity = threadIdx.x & 1;
    double hx, hy, hz;
    load_rec(L + kRec * NP, hx, hy, hz);
    vx = fma(tau, hx, vx);
    vy = fma(tau, hy, vy);
    vz = fma(tau, hz, vz);
    double ax = 0.0, ay = 0.0, az = 0.0;
    int hit = 0;
#pragma unroll
    for (int jj = (NP + 1) / 2 - 1; jj >= 0; --jj) {
        const int j = 2 * jj + parity;
        if (j < NP) {
            double px, py, pz;
            load_rec(L + kRec * j, px, py, pz);
            const double dx = x - px, dy = y - py, dz = z - pz;
            const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
            hit = lt_nonneg(d2, rc2[j]) ? (j + 1) : hit;
            const double s = k_rcube(d2, tgm[j]);
            ax = fma(-s, dx, ax);
            ay = fma(-s, dy, ay);
            az = fma(-s, dz, az);
        }
    }
    vx += ax + __shfl_xor_sync(kFullMask, ax, 1);
    vy += ay + __shfl_xor_sync(kFullMask, ay, 1);
    vz += az + __shfl_xor_sync(kFullMask, az, 1);
    const int other = __shfl_xor_sync(kFullMask, hit, 1);
    return (hit != 0 && other != 0) ? min(hit, other) : (hit | other);
}

// The kick of a particle held by TPP lanes (1, or 2: kick_test_pair).
template <int NP, int TPP>
__device__ __forceinline__ int kick_lanes(double x, double y, double z, double& vx, double& vy, double& vz,
                                          const double* __restrict__ L, double tau, const double (&tgm)[kMaxPlanets],
                                          const double (&rc2)[kMaxPlanets]) {
    if constexpr (TPP == 2)
        return kick_test_pair<NP>(x, y, z, vx, vy, vz, L, tau, tgm, rc2);
    else
        return kick_test<NP>(x, y, z, vx, vy, vz, L, tau, tgm, rc2);
}

// Removal test without a kick (used at t_0).
template <int NP>
__device__ __forceinline__ int test_only(double x, double y, double z, const double* __restrict__ L,
                                         const double (&rc2)[kMaxPlanets], double rmax2) {
    int hit = 0;
    const double r2 = fma(x, x, fma(y, y, z * z));
    if (__double_as_longlong(rmax2) != 0 && lt_nonneg(rmax2, r2)) hit = GLISSE_REMOVED_ESCAPE;
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        double px, py, pz;
        load_rec(L + kRec * j, px, py, pz);
        const double dx = x - px, dy = y - py, dz = z - pz;
        const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
        hit = lt_nonneg(d2, rc2[j]) ? (j + 1) : hit;
    }
    return hit;
}

// The map for one lane over nsteps steps of the log L (L step 0 = the lane's
// current time).  State in registers; act / reason / rstep record removal.
// open_in: the velocities already carry the opening half kick of step 0.
// close_out: false leaves the state open, ending with the full kick that a
// single longer launch would apply there (the next segment then has open_in).
// A split with open_in / close_out is bit-identical to no split.
// pc may live in the constant bank (kernel parameter) or in shared memory.
// TPP = 2: the particle is held by a lane pair (batched kernel), each lane
// running the same state with half of the planets in the kicks.
// Where a lane publishes its synchronised state: out[6 id[slot] .. + 5] (out null: nowhere).
struct PublishTo {
    const int32_t* id;
    double* out;
    int64_t slot;
};

// PUBLISH (with close_out false): a lane still live at the segment's end also
// writes its synchronised state there (position; pre-kick velocities plus the
// closing half kick), straight to memory so that nothing stays live in
// registers across the steps.
template <int NP, int MODE = kDriftConverge, int TPP = 1, bool PUBLISH = false>
__device__ __forceinline__ void advance_lane(const ParticleConsts& pc, const double* __restrict__ L, int64_t step0,
                                             int nsteps, bool test_first, double& x, double& y, double& z, double& vx,
                                             double& vy, double& vz, bool& act, int& reason, int64_t& rstep,
                                             bool open_in = false, bool close_out = true, PublishTo pub = {}) {
    const float muf = d2f_bits(pc.mu), dtf = d2f_bits(pc.dt);
    const bool has_rmax = __double_as_longlong(pc.rmax) != 0;
    const int S = log_stride(NP);

    if (test_first) {
        const int h = test_only<NP>(x, y, z, L, pc.rc2, pc.rmax2);
        if (act && h != 0) {
            act = false;
            reason = h;
            rstep = step0;
        }
    }
    if (!open_in) {
        if constexpr (TPP == 2) {
            // the pair kick shuffles across the warp: every lane runs it, active lanes keep it
            double nvx = vx, nvy = vy, nvz = vz;
            kick_test_pair<NP>(x, y, z, nvx, nvy, nvz, L, pc.half_dt, pc.tgm_half, pc.rc2);
            if (act) {
                vx = nvx;
                vy = nvy;
                vz = nvz;
            }
        } else if (act) {
            kick_test<NP>(x, y, z, vx, vy, vz, L, pc.half_dt, pc.tgm_half, pc.rc2);
        }
    }
    double r0, mur0;
    radius_of(x, y, z, r0, mur0);
    mur0 *= pc.mu;

    for (int k = 0; k < nsteps; ++k) {
        if (!__any_sync(kFullMask, act)) break;
        const double* __restrict__ Ln = L + (size_t)(k + 1) * S;
        const double sx = x, sy = y, sz = z, svx = vx, svy = vy, svz = vz;
        const double sr0 = r0, smur0 = mur0;
        bool failed = false;
        if constexpr (MODE == kDriftConverge) {
            const bool done = drift_fast(pc.mu, muf, pc.dt, dtf, act, r0, mur0, x, y, z, vx, vy, vz);
            if (act && !done) {
                failed = !drift_general(pc.mu, pc.dt, x, y, z, vx, vy, vz);
                radius_of(x, y, z, r0, mur0);
                mur0 *= pc.mu;
            }
        } else {
            if (act) {
                failed = drift_paper(pc.mu, pc.dt, pc.kepler_iters, pc.kepler_tol, x, y, z, vx, vy, vz) != 0;
                radius_of(x, y, z, r0, mur0);
            }
        }
        const bool bad = nonfinite_bits(x) || nonfinite_bits(y) || nonfinite_bits(z) || nonfinite_bits(vx) ||
                         nonfinite_bits(vy) || nonfinite_bits(vz);
        if (act && (failed || bad)) {
            x = sx;
            y = sy;
            z = sz;
            vx = svx;
            vy = svy;
            vz = svz;
            r0 = sr0;
            mur0 = smur0;
            act = false;
            reason = failed ? GLISSE_REMOVED_KEPLER : GLISSE_REMOVED_NONFINITE;
            rstep = step0 + k + 1;
        }
        // escape: |r| > r_max, with |r| from the drift (integer compare of positive doubles)
        int hit = (has_rmax && lt_nonneg(pc.rmax, r0)) ? GLISSE_REMOVED_ESCAPE : 0;
        const bool last = close_out && (k + 1 == nsteps);
        double nvx = vx, nvy = vy, nvz = vz;
        int enc;
        if (last)
            enc = kick_lanes<NP, TPP>(x, y, z, nvx, nvy, nvz, Ln, pc.half_dt, pc.tgm_half, pc.rc2);
        else
            enc = kick_lanes<NP, TPP>(x, y, z, nvx, nvy, nvz, Ln, pc.dt, pc.tgm_full, pc.rc2);
        hit = enc ? enc : hit;
        if constexpr (PUBLISH) {
            if (pub.out && !close_out && k + 1 == nsteps && act && hit == 0) {
                double hx = vx, hy = vy, hz = vz;
                kick_test<NP>(x, y, z, hx, hy, hz, Ln, pc.half_dt, pc.tgm_half, pc.rc2);
                double* o = pub.out + 6 * (int64_t)pub.id[pub.slot];
                o[0] = x;
                o[1] = y;
                o[2] = z;
                o[3] = hx;
                o[4] = hy;
                o[5] = hz;
            }
        }
        if (act) {
            if (hit != 0) {
                act = false;
                reason = hit;
                rstep = step0 + k + 1;
            } else {
                vx = nvx;
                vy = nvy;
                vz = nvz;
            }
        }
    }
}

// Write a removed particle's result under its id.
__device__ __forceinline__ void store_removed(int64_t pid, double x, double y, double z, double vx, double vy,
                                              double vz, int64_t rstep, int reason, double* out_state,
                                              int64_t* out_step, int32_t* out_reason) {
    double* o = out_state + 6 * pid;
    o[0] = x;
    o[1] = y;
    o[2] = z;
    o[3] = vx;
    o[4] = vy;
    o[5] = vz;
    out_step[pid] = rstep;
    out_reason[pid] = reason;
}

template <int NP, int MODE>
__global__ void __launch_bounds__(kParticleBlock, GLISSE_PARTICLE_MIN_BLOCKS)
    particle_chunk_kernel(const ChunkArgs a, const ParticleConsts pc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = i < a.n;
    const int64_t ld = a.ld;
    double x, y, z, vx, vy, vz;
    if (in) {
        x = a.st[i];
        y = a.st[ld + i];
        z = a.st[2 * ld + i];
        vx = a.st[3 * ld + i];
        vy = a.st[4 * ld + i];
        vz = a.st[5 * ld + i];
    } else {
        // idle lanes carry a harmless circular orbit so the shared drift stays finite
        x = 1.0;
        y = 0.0;
        z = 0.0;
        vx = 0.0;
        vy = 6.283185307179586;
        vz = 0.0;
    }
    bool act = in && a.alive[i] != 0;
    const bool started = act;
    int reason = 0;
    int64_t rstep = -1;
    advance_lane<NP, MODE, 1, true>(pc, a.log, a.step0, a.nsteps, a.test_first != 0, x, y, z, vx, vy, vz, act,
                                    reason, rstep, a.open_in != 0, a.close_out != 0, PublishTo{a.id, a.out_state, i});
    if (a.steps_done) {
        // steps this particle actually advanced in the segment (exact work count)
        const unsigned adv = !started ? 0u : (rstep >= 0 ? (unsigned)(rstep - a.step0) : (unsigned)a.nsteps);
        const unsigned wsum = __reduce_add_sync(kFullMask, adv);
        if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(a.steps_done, (unsigned long long)wsum);
    }
    if (a.live_out) {
        // particles live at the segment's end
        const unsigned wl = __reduce_add_sync(kFullMask, act ? 1u : 0u);
        if ((threadIdx.x & 31) == 0 && wl) atomicAdd(a.live_out, (unsigned long long)wl);
    }
    if (in) {
        a.st[i] = x;
        a.st[ld + i] = y;
        a.st[2 * ld + i] = z;
        a.st[3 * ld + i] = vx;
        a.st[4 * ld + i] = vy;
        a.st[5 * ld + i] = vz;
        a.alive[i] = act ? 1 : 0;
        if (rstep >= 0) store_removed(a.id[i], x, y, z, vx, vy, vz, rstep, reason, a.out_state, a.out_step,
                                      a.out_reason);
    }
}

// ---------------------------------------------------------------------------
// Task mode: persistent warps over (group, sub-chunk) tasks.
//
// Every warp of a chunk does the same work, so with one thread per slot the
// chunk lasts as long as the SM partition holding the most warps: at 6.06
// warps per partition on average, the busiest has 7 and the pipe is 87%
// used.  A particle's steps are serial, so balance needs smaller units of
// work: the segment is cut into sub-chunks of sub_steps steps, and a task is
// one group of 32 slots (the members of one warp of the plain launch) over
// one sub-chunk.  Tasks are taken in order from a counter by a fixed number of
// resident warps, so every partition keeps the same number of busy warps
// until the last round of tasks.  Task (g, s) needs (g, s - 1) finished: it
// is taken n_groups tasks later, by when the launch has that many warps'
// worth of work behind it (the host uses task mode only when groups
// outnumber resident warps by half again), and the warp waits, bounded, on
// the group's counter of finished sub-chunks.  Sub-chunk cuts are open cuts,
// so the result is bit-identical to the plain launch: same members per warp,
// same steps, same kicks.
// ---------------------------------------------------------------------------
constexpr int kSubSteps = 32;
// a wait for the previous sub-chunk of a group gives up after this many polls
// (~64 ns each: seconds, where a sub-chunk takes a millisecond at most)
constexpr int kGroupWaitPolls = 1 << 25;

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// at most four blocks per SM (task_warps_per_partition), so up to 128 registers per thread
constexpr int kTaskMaxBlocks = 4;

template <int NP>
__global__ void __launch_bounds__(kParticleBlock, kTaskMaxBlocks)
    particle_tasks_kernel(const ChunkArgs a, const ParticleConsts pc, const TaskArgs ta) {
    const int lane = threadIdx.x & 31;
    const int64_t ld = a.ld;
    const int S = log_stride(NP);
    const int n_sub = (a.nsteps + ta.sub_steps - 1) / ta.sub_steps;
    const int64_t n_tasks = (int64_t)ta.n_groups * n_sub;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ta.task_counter, 1ull);
        t = __shfl_sync(kFullMask, t, 0);
        if ((int64_t)t >= n_tasks) break;
        const int64_t g = (int64_t)t % ta.n_groups;
        const int s = (int)((int64_t)t / ta.n_groups);
        if (s > 0) {
            int ok = 1;
            if (lane == 0) {
                const int limit = ta.wait_polls > 0 ? ta.wait_polls : kGroupWaitPolls;
                int polls = 0;
                while (ld_acquire(ta.group_done + g) < s && ++polls < limit) __nanosleep(64);
                ok = polls < limit;
            }
            ok = __shfl_sync(kFullMask, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(ta.status, GLISSE_E_TIMEOUT);
                break;
            }
        }
        __syncwarp();
        const int64_t i = g * 32 + lane;
        const bool in = i < a.n;
        double x = 1.0, y = 0.0, z = 0.0, vx = 0.0, vy = 6.283185307179586, vz = 0.0;
        bool act = false;
        if (in) {
            // written by another warp's task (L2 is coherent, this SM's L1 may not be)
            x = __ldcg(a.st + i);
            y = __ldcg(a.st + ld + i);
            z = __ldcg(a.st + 2 * ld + i);
            vx = __ldcg(a.st + 3 * ld + i);
            vy = __ldcg(a.st + 4 * ld + i);
            vz = __ldcg(a.st + 5 * ld + i);
            act = __ldcg(a.alive + i) != 0;
        }
        const bool started = act;
        int reason = 0;
        int64_t rstep = -1;
        const int k0 = s * ta.sub_steps;
        const int m = min(ta.sub_steps, a.nsteps - k0);
        const bool last = s + 1 == n_sub;
        advance_lane<NP, kDriftConverge, 1, true>(pc, a.log + (size_t)k0 * S, a.step0 + k0, m,
                                                  a.test_first != 0 && s == 0, x, y, z, vx, vy, vz, act, reason,
                                                  rstep, s > 0 || a.open_in != 0, last ? a.close_out != 0 : false,
                                                  PublishTo{a.id, last ? a.out_state : nullptr, i});
        if (a.steps_done) {
            const unsigned adv = !started ? 0u : (rstep >= 0 ? (unsigned)(rstep - (a.step0 + k0)) : (unsigned)m);
            const unsigned wsum = __reduce_add_sync(kFullMask, adv);
            if (lane == 0 && wsum) atomicAdd(a.steps_done, (unsigned long long)wsum);
        }
        if (last && a.live_out) {
            const unsigned wl = __reduce_add_sync(kFullMask, act ? 1u : 0u);
            if (lane == 0 && wl) atomicAdd(a.live_out, (unsigned long long)wl);
        }
        if (in) {
            __stcg(a.st + i, x);
            __stcg(a.st + ld + i, y);
            __stcg(a.st + 2 * ld + i, z);
            __stcg(a.st + 3 * ld + i, vx);
            __stcg(a.st + 4 * ld + i, vy);
            __stcg(a.st + 5 * ld + i, vz);
            __stcg(a.alive + i, (uint8_t)(act ? 1 : 0));
            if (rstep >= 0) store_removed(a.id[i], x, y, z, vx, vy, vz, rstep, reason, a.out_state, a.out_step,
                                          a.out_reason);
        }
        // every lane's stores before the group's counter moves on (release at device scope)
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(ta.group_done + g, s + 1);
    }
}

// Dynamic shared memory (unused by the kernel) that caps the resident blocks
// per SM at what an even spread of this grid needs.  Every block does the same
// work, so the chunk lasts as long as the SM holding the most blocks; the
// hardware may pack up to GLISSE_PARTICLE_MIN_BLOCKS on some SMs and fewer on
// others, and the ephemeris kernel holds one SM for itself (all of its shared
// memory).  Spread over the other SMs, ceil(grid / (SMs - 1)) per SM is the
// best any placement can do; the request makes more than that impossible.
inline cudaError_t particle_smem_cap(const void* kernel, int64_t grid, size_t* smem) {
    *smem = 0;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t per_sm = nsm > 1 ? (grid + nsm - 2) / (nsm - 1) : GLISSE_PARTICLE_MIN_BLOCKS;
    return residency_cap_smem(kernel, per_sm, GLISSE_PARTICLE_MIN_BLOCKS, smem);
}

// Warps per SM partition for task mode, or 0 for the plain launch: task mode
// pays when the groups outnumber the resident warps by half again (waits are
// then rare) with at least two busy warps per partition (one warp alone keeps
// the FP64 pipe ~70% busy); at most four (enough to saturate it).
inline int task_warps_per_partition(int64_t n, int nsteps, int n_sm) {
    const int64_t groups = (n + 31) / 32;
    const int64_t partitions = 4 * (int64_t)std::max(n_sm - 1, 1);
    if (nsteps < 2 * kSubSteps) return 0;
    const int64_t k = (2 * groups) / (3 * partitions);
    return k >= 2 ? (int)std::min<int64_t>(k, kTaskMaxBlocks) : 0;
}

// tb: the task-mode buffers (counter, per-group counters, status), or null for the plain launch.
// force_tasks: task mode whatever the size (two warps per partition at least; GLISSE_LAUNCH_TASKS).
template <int MODE>
cudaError_t launch_particle_chunk_mode(int np, const ChunkArgs& a, const ParticleConsts& pc, cudaStream_t s,
                                       const TaskArgs* tb = nullptr, bool force_tasks = false) {
    if (a.n <= 0) return cudaSuccess;
    if constexpr (MODE == kDriftConverge) {
        int dev = 0, nsm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        int k = tb ? task_warps_per_partition(a.n, a.nsteps, nsm) : 0;
        if (tb && force_tasks && k == 0) k = 2;
        if (k > 0) {
            TaskArgs b = *tb;
            b.sub_steps = kSubSteps;
            b.n_groups = (int32_t)((a.n + 31) / 32);
            e = cudaMemsetAsync(b.task_counter, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(b.group_done, 0, sizeof(int32_t) * (size_t)b.n_groups, s);
            if (e != cudaSuccess) return e;
            // k blocks of four warps per SM, one SM's worth short (the ephemeris holds one)
            const int64_t grid = (int64_t)k * std::max(nsm - 1, 1);
            size_t smem = 0;
            switch (np) {
#define GLISSE_TCASE(N)                                                                                  \
    case N:                                                                                              \
        e = particle_smem_cap(reinterpret_cast<const void*>(particle_tasks_kernel<N>), grid, &smem);     \
        if (e != cudaSuccess) return e;                                                                  \
        particle_tasks_kernel<N><<<(unsigned)grid, kParticleBlock, smem, s>>>(a, pc, b);                 \
        break;
                GLISSE_TCASE(0)
                GLISSE_TCASE(1)
                GLISSE_TCASE(2)
                GLISSE_TCASE(3)
                GLISSE_TCASE(4)
                GLISSE_TCASE(5)
                GLISSE_TCASE(6)
                GLISSE_TCASE(7)
                GLISSE_TCASE(8)
#undef GLISSE_TCASE
                default: return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
        }
    }
    const int64_t grid = (a.n + kParticleBlock - 1) / kParticleBlock;
    size_t smem = 0;
    cudaError_t e = cudaSuccess;
    switch (np) {
#define GLISSE_CASE(N)                                                                                    \
    case N:                                                                                               \
        e = particle_smem_cap(reinterpret_cast<const void*>(particle_chunk_kernel<N, MODE>), grid, &smem); \
        if (e != cudaSuccess) return e;                                                                   \
        particle_chunk_kernel<N, MODE><<<(unsigned)grid, kParticleBlock, smem, s>>>(a, pc);              \
        break;
        GLISSE_CASE(0)
        GLISSE_CASE(1)
        GLISSE_CASE(2)
        GLISSE_CASE(3)
        GLISSE_CASE(4)
        GLISSE_CASE(5)
        GLISSE_CASE(6)
        GLISSE_CASE(7)
        GLISSE_CASE(8)
#undef GLISSE_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace glisse
