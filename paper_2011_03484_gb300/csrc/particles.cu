// particles.cu -- instantiates the test-particle map (particle_map.cuh) with the
// converged fast Kepler solver, and the persistent kernel of batched systems.
#include "particle_map.cuh"

namespace glisse {

// ---------------------------------------------------------------------------
// Batched systems: a persistent kernel.  Each warp takes the next task from
// the work counter, stages its system's constants in a warp-private slot of
// shared memory and runs advance_lane with that system's planet count.
// ---------------------------------------------------------------------------
// TPP = 1: lane k holds particle start + k.  TPP = 2: the lane pair (2k, 2k + 1)
// holds particle start + k (half of the task's 32 particles per call; `half`
// picks which), and only its even lane writes results and counts.
template <int NP, int TPP>
__device__ __forceinline__ void batch_task(const BatchArgs& a, const ParticleConsts& pc, int s, int64_t start,
                                           int cnt, int lane, int64_t step0, bool test_first, int half = 0) {
    const int slot = TPP == 2 ? 16 * half + (lane >> 1) : lane;
    const bool owner = TPP == 1 || (lane & 1) == 0;
    const int64_t i = start + slot;
    const bool in = slot < cnt;
    const int64_t ld = a.ld;
    double x = 1.0, y = 0.0, z = 0.0, vx = 0.0, vy = 6.283185307179586, vz = 0.0;
    if (in) {
        x = a.st[i];
        y = a.st[ld + i];
        z = a.st[2 * ld + i];
        vx = a.st[3 * ld + i];
        vy = a.st[4 * ld + i];
        vz = a.st[5 * ld + i];
    }
    bool act = in && a.alive[i] != 0;
    const bool started = act;
    int reason = 0;
    int64_t rstep = -1;
    advance_lane<NP, kDriftConverge, TPP>(pc, a.log + a.log_off[s], step0, a.nsteps, test_first, x, y, z, vx, vy, vz,
                                          act, reason, rstep);
    const unsigned live = __reduce_add_sync(kFullMask, (act && owner) ? 1u : 0u);
    if (lane == 0 && live) atomicAdd(reinterpret_cast<unsigned long long*>(a.cnt_new + s), (unsigned long long)live);
    if (a.steps_done) {
        const unsigned adv =
            (!started || !owner) ? 0u : (rstep >= 0 ? (unsigned)(rstep - step0) : (unsigned)a.nsteps);
        const unsigned wsum = __reduce_add_sync(kFullMask, adv);
        if (lane == 0 && wsum) atomicAdd(a.steps_done, (unsigned long long)wsum);
    }
    if (in && owner) {
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

constexpr int kBatchMaxWarps = 8;  // largest block of the batched kernel: 256 threads

template <int TPP>
__global__ void __launch_bounds__(32 * kBatchMaxWarps) batch_particle_kernel(const BatchArgs a) {
    __shared__ ParticleConsts s_pc[kBatchMaxWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntask = *a.n_tasks;
    const int64_t step0 = a.clock->step;
    const bool test_first = a.clock->test_first != 0;
    constexpr int kWords = (int)(sizeof(ParticleConsts) / sizeof(double));
    static_assert(sizeof(ParticleConsts) % sizeof(double) == 0, "constants must be whole doubles");
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(kFullMask, t, 0);
        if (t >= ntask) break;
        const int s = a.task_sys[t];
        const int64_t start = a.task_start[t];
        const int cnt = a.task_count[t];
        const double* src = reinterpret_cast<const double*>(a.pcs + s);
        double* dst = reinterpret_cast<double*>(&s_pc[warp]);
        for (int w = lane; w < kWords; w += 32) dst[w] = src[w];
        __syncwarp();
        const ParticleConsts& pc = s_pc[warp];
        switch (a.np_of[s]) {
#define GLISSE_BCASE(N)                                                          \
    case N:                                                                      \
        for (int h = 0; h < TPP; ++h) batch_task<N, TPP>(a, pc, s, start, cnt, lane, step0, test_first, h); \
        break;
            GLISSE_BCASE(0)
            GLISSE_BCASE(1)
            GLISSE_BCASE(2)
            GLISSE_BCASE(3)
            GLISSE_BCASE(4)
            GLISSE_BCASE(5)
            GLISSE_BCASE(6)
            GLISSE_BCASE(7)
            GLISSE_BCASE(8)
#undef GLISSE_BCASE
            default: break;
        }
        __syncwarp();
    }
}

// Persistent launch: `blocks` blocks of `threads` threads (a multiple of 32, <= 256),
// tpp (1 or 2) lanes per particle.
cudaError_t launch_batch_particles(const BatchArgs& a, int blocks, int threads, int tpp, cudaStream_t s) {
    if (threads < 32 || threads > 32 * kBatchMaxWarps || threads % 32) return cudaErrorInvalidValue;
    if (tpp == 2)
        batch_particle_kernel<2><<<blocks, threads, 0, s>>>(a);
    else if (tpp == 1)
        batch_particle_kernel<1><<<blocks, threads, 0, s>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t batch_particles_occupancy(int threads, int tpp, int* blocks_per_sm) {
    if (tpp == 2)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_particle_kernel<2>, threads, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_particle_kernel<1>, threads, 0);
}

cudaError_t launch_particle_chunk(int np, const ChunkArgs& a, const ParticleConsts& pc, cudaStream_t s,
                                  const TaskArgs* tb, bool force_tasks) {
    return launch_particle_chunk_mode<kDriftConverge>(np, a, pc, s, tb, force_tasks);
}

// Self-test of the task launch's bounded wait.  Two groups of 32 slots, two sub-chunks;
// the task counter starts past the first sub-chunk of both groups, so each task handed out
// waits for a sub-chunk that no task runs: its warp gives up after `polls` polls, sets
// *status to GLISSE_E_TIMEOUT and leaves before touching a particle (the other warps find
// no task left).  scratch: zeroed device memory holding the task counter (8 bytes) and
// the groups' counters (8 bytes); the particle arrays point at it too, never read.
cudaError_t particle_wait_selftest(int polls, char* scratch, int* status, cudaStream_t s) {
    constexpr int kGroups = 2;
    ChunkArgs a{};
    a.n = 32 * kGroups;
    a.ld = a.n;
    a.nsteps = 2 * kSubSteps;
    a.log = reinterpret_cast<const double*>(scratch);
    a.st = reinterpret_cast<double*>(scratch);
    a.id = reinterpret_cast<const int32_t*>(scratch);
    a.alive = reinterpret_cast<uint8_t*>(scratch);
    TaskArgs ta{};
    ta.sub_steps = kSubSteps;
    ta.n_groups = kGroups;
    ta.task_counter = reinterpret_cast<unsigned long long*>(scratch);
    ta.group_done = reinterpret_cast<int32_t*>(scratch + 8);
    ta.status = status;
    ta.wait_polls = polls;
    const unsigned long long first = kGroups;
    cudaError_t e = cudaMemcpyAsync(ta.task_counter, &first, sizeof(first), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    particle_tasks_kernel<0><<<4, kParticleBlock, 0, s>>>(a, ParticleConsts{}, ta);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace glisse
