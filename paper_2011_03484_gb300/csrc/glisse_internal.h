// glisse_internal.h -- types shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/glisse.h"

namespace glisse {

// Dynamic shared memory (unused by the kernel) to request so that at most
// per_sm blocks of `kernel` can reside on an SM: per_sm blocks fit, per_sm + 1
// do not.  *smem = 0 when no request is needed (per_sm >= max_blocks, what the
// registers already allow) or none can express the cap.  Sets the kernel's
// dynamic shared-memory limit to the request.
inline cudaError_t residency_cap_smem(const void* kernel, int64_t per_sm, int max_blocks, size_t* smem) {
    *smem = 0;
    if (per_sm >= max_blocks || per_sm < 1) return cudaSuccess;
    int dev = 0, smem_sm = 0, reserved = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    size_t b = (size_t)(smem_sm / per_sm - reserved) & ~(size_t)1023;
    b = std::min<size_t>(b, (size_t)optin);
    while (b > 0 && (size_t)(per_sm + 1) * (b + reserved) <= (size_t)smem_sm) b += 1024;
    if ((size_t)per_sm * (b + reserved) > (size_t)smem_sm) return cudaSuccess;  // cannot express the cap
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    if (e == cudaSuccess) *smem = b;
    return e;
}

constexpr int kMaxPlanets = GLISSE_MAX_PLANETS;

// One record per body per step in the planet log: heliocentric x, y, z and a pad.
// A log step holds N_p planet records followed by the record of the common
// term h0 = -sum_j G m_j r_j / |r_j|^3 (section 2.2).  32-byte records let a
// warp fetch a whole record with two 16-byte broadcast loads.
constexpr int kRec = 4;
__host__ __device__ constexpr int log_stride(int np) { return kRec * (np + 1); }
// The ephemeris kernel of a context's first chunk publishes its step count this often.
constexpr int kProgressEvery = 16;

// Planet system constants (written once by the set-up kernel, read by all kernels).
struct PlanetConsts {
    int np;
    double m0;
    double G;
    double mu0;                      // G m0: the particles' Kepler parameter
    double m[kMaxPlanets];
    double eta[kMaxPlanets + 1];     // eta[0] = m0, eta[i] = m0 + m_1 + ... + m_i
    double mu_jac[kMaxPlanets];      // G m0 eta_i / eta_{i-1}: Jacobi Kepler parameter of planet i
    double gm[kMaxPlanets];          // G m_j
    double rcrit[kMaxPlanets];       // encounter radius of planet j (0 disables)
};

// Particle-kernel constants derived from the planet constants and dt.
struct ParticleConsts {
    double mu;                        // G m0
    double dt;
    double half_dt;
    double tgm_full[kMaxPlanets];     // dt G m_j
    double tgm_half[kMaxPlanets];     // dt/2 G m_j
    double rc2[kMaxPlanets];          // R_crit,j^2 (0: no test)
    double rmax2;                     // r_max^2 (0: no test)
    double rmax;                      // r_max (0: no test)
    double kepler_tol;                // fixed-iteration mode: largest accepted last Newton step
    int32_t kepler_iters;             // fixed-iteration mode: Newton iterations per drift
    int32_t pad_;
};

// Arguments of one particle-chunk launch.
struct ChunkArgs {
    const ParticleConsts* pc;
    const double* log;    // log of this segment: step 0 = the particles' current time
    int64_t n;            // live slots
    int64_t ld;           // leading dimension of the state planes
    double* st;           // [6][ld] x, y, z, vx, vy, vz planes
    const int32_t* id;    // [n]
    uint8_t* alive;       // [n] out: 1 = still live after the segment
    int64_t step0;        // global index of the segment's first step
    int32_t nsteps;       // steps in the segment (>= 1)
    int32_t test_first;   // apply the removal test at the segment's step 0 first
    int32_t open_in;      // the velocities already hold the opening half kick of step 0
    int32_t close_out;    // 1: end with the closing half kick (synchronised state);
                          // 0: end with the full kick that also opens the next segment, and
                          //    write live particles' synchronised states to out_state by id
    // per-id outputs: particles removed during the segment (and, close_out = 0, live ones)
    double* out_state;    // [N][6]
    int64_t* out_step;    // [N]
    int32_t* out_reason;  // [N]
    unsigned long long* steps_done;  // optional: += steps advanced by live particles
    unsigned long long* live_out;    // optional: += particles live at the segment's end
};

// Task mode of the particle kernel (particle_tasks_kernel): the segment is cut into
// sub-chunks of sub_steps steps; task t = (group t mod n_groups, sub-chunk t / n_groups),
// where a group is the 32 slots one warp holds, is taken in order from task_counter by
// persistent warps.  (A separate argument: the plain kernel's registers are tight.)
struct TaskArgs {
    int32_t sub_steps;                 // steps per sub-chunk
    int32_t n_groups;                  // ceil(n / 32)
    unsigned long long* task_counter;  // zero before the launch
    int32_t* group_done;               // [n_groups] sub-chunks of each group finished; zero before the launch
    int* status;                       // set to GLISSE_E_TIMEOUT if a wait for a group gives up
    int32_t wait_polls;                // polls before a wait gives up; 0: the default (seconds)
};

// Device-resident clock of a batch (so a captured chunk graph can be replayed).
struct BatchClock {
    int64_t step;        // global index of the next chunk's first step
    int32_t test_first;  // 1 until the first chunk has run
    int32_t pad;
};

// Arguments of the persistent batched particle kernel.  Task t covers
// particles [task_start[t], task_start[t] + task_count[t]) of system task_sys[t]
// (task_count <= 32: one warp).
struct BatchArgs {
    const ParticleConsts* pcs;  // [n_sys]
    const int32_t* np_of;       // [n_sys]
    const double* log;          // all systems' planet logs
    const int64_t* log_off;     // [n_sys] offset of each system's log (doubles)
    const int32_t* task_sys;
    const int64_t* task_start;
    const int32_t* task_count;
    const int64_t* n_tasks;     // device scalar
    int* counter;               // work counter, zero before the launch
    const BatchClock* clock;
    int64_t ld;
    double* st;                 // [6][ld]
    const int32_t* id;
    uint8_t* alive;
    int64_t* cnt_new;           // [n_sys] += particles still live after the chunk
    int32_t nsteps;
    double* out_state;
    int64_t* out_step;
    int32_t* out_reason;
    unsigned long long* steps_done;
};

// Arguments of one element sample (section 3: osculating elements logged at a
// fixed interval; libration of a resonant argument).
struct SampleArgs {
    int64_t n;                 // live slots
    const double* sync;        // [N][6] by id: synchronised states (live slots' entries current)
    const int32_t* id;         // [n]
    const uint8_t* alive;      // [n]
    const double* planets;     // [np][6] heliocentric planet states at the sample step
    const PlanetConsts* pc;    // masses, m0, G
    int32_t frame;             // GLISSE_FRAME_*
    int32_t res_planet;        // 0-based planet of the resonance, -1: none
    int32_t res_p, res_q;      // phi = p lambda - q lambda_planet - (p - q) varpi
    double avoid;              // half-width of the windows around 0 and 180 degrees, radians
    double* elem;              // [N][6] by id, or null
    uint8_t* near0;            // [N] by id (res_planet >= 0)
    uint8_t* near180;          // [N]
    int32_t* count;            // [N] samples that entered the test
};

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t s);

}  // namespace glisse
