// batch.cu -- many independent planetary systems in one context.
//
// Each system has its own star, planets (up to kMaxPlanets), particles and dt.
// Particles live in one set of SoA planes, systems contiguous and ordered by
// decreasing planet count (the costliest tasks are handed out first, which
// keeps the persistent kernel's tail short).  One chunk is:
//   1. eph_batch_kernel      planet chunk of every system (block = system)
//   2. batch_particle_kernel persistent; warps take 32-particle tasks, one lane
//                            (or, chosen by the autotuner, a lane pair) per particle
//   3. stable partition      count / scan / scatter, sizes read on the device
//   4. flags + task rebuild  per-system live counts -> offsets -> task table,
//                            clock advanced
// Every size stays on the device, so a chunk is captured once per (buffer
// parity, step count) as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "glisse_internal.h"
#include "nvtx_range.h"

namespace glisse {
cudaError_t launch_eph_setup(const double*, int, double, double, int, double, PlanetConsts*, double*, int*,
                             cudaStream_t);
cudaError_t launch_eph_batch(const PlanetConsts*, int, double*, const double*, int, double*, const int64_t*, int*,
                             cudaStream_t);
cudaError_t launch_batch_particles(const BatchArgs&, int, int, int, cudaStream_t);
cudaError_t batch_particles_occupancy(int, int, int*);
cudaError_t launch_export_live(int64_t, const double*, int64_t, const int32_t*, double*, cudaStream_t);
cudaError_t launch_import(int64_t, const double*, double*, int64_t, int32_t*, cudaStream_t);

constexpr int kBThreads = 256;
constexpr int kBRounds = 8;
constexpr int kBTile = kBThreads * kBRounds;

// ---- stable partition with the slot count read from device memory ---------------
__global__ void __launch_bounds__(kBThreads) bpart_count_kernel(const uint8_t* __restrict__ alive,
                                                                  const int64_t* __restrict__ n_dev,
                                                                  int64_t* __restrict__ counts) {
    const int64_t n = *n_dev;
    const int64_t base = (int64_t)blockIdx.x * kBTile;
    if (base >= n) return;
    int c = 0;
    for (int r = 0; r < kBRounds; ++r) {
        const int64_t idx = base + r * kBThreads + threadIdx.x;
        c += (idx < n && alive[idx] != 0) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __shared__ int ws[kBThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kBThreads / 32; ++w) t += ws[w];
        counts[blockIdx.x] = t;
    }
}

// exclusive scan of the tile counts of n_dev slots; kept total -> *n_out.  One block of 1024.
__global__ void __launch_bounds__(1024) bpart_scan_kernel(int64_t* __restrict__ counts,
                                                            const int64_t* __restrict__ n_dev,
                                                            int64_t* __restrict__ n_out) {
    const int64_t nb = (*n_dev + kBTile - 1) / kBTile;
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t idx = b0 + threadIdx.x;
        const int64_t v = idx < nb ? counts[idx] : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int64_t ws = wsum[lane];
            int64_t wi = ws;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;
        }
        __syncthreads();
        const int64_t excl = carry + wsum[warp] + incl - v;
        if (idx < nb) counts[idx] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = carry;
}

__global__ void __launch_bounds__(kBThreads) bpart_scatter_kernel(
    const uint8_t* __restrict__ alive, const int64_t* __restrict__ n_dev, const int64_t* __restrict__ offsets,
    const double* __restrict__ src, const int32_t* __restrict__ src_id, double* __restrict__ dst,
    int32_t* __restrict__ dst_id, int64_t ld) {
    const int64_t n = *n_dev;
    const int64_t base = (int64_t)blockIdx.x * kBTile;
    if (base >= n) return;
    __shared__ int wc[kBThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t out = offsets[blockIdx.x];
    for (int r = 0; r < kBRounds; ++r) {
        const int64_t idx = base + r * kBThreads + threadIdx.x;
        const bool f = idx < n && alive[idx] != 0;
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, f);
        const int rank = __popc(ball & ((1u << lane) - 1u));
        if (lane == 0) wc[warp] = __popc(ball);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int w = 0; w < kBThreads / 32; ++w) {
            woff += (w < warp) ? wc[w] : 0;
            tot += wc[w];
        }
        if (f) {
            const int64_t d = out + woff + rank;
            for (int c = 0; c < 6; ++c) dst[c * ld + d] = src[c * ld + idx];
            dst_id[d] = src_id[idx];
        }
        out += tot;
        __syncthreads();
    }
}

// alive[i] = 1 for i < *n_dev
__global__ void bpart_flags_kernel(uint8_t* __restrict__ alive, const int64_t* __restrict__ n_dev, int64_t cap) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < cap;
         i += (int64_t)gridDim.x * blockDim.x)
        alive[i] = 1;
}

// Per-system live counts -> task table; totals; counters reset; clock advanced.  One block of 1024.
__global__ void __launch_bounds__(1024) batch_tasks_kernel(int n_sys, int64_t* __restrict__ cnt,
                                                             int32_t* __restrict__ task_sys,
                                                             int64_t* __restrict__ task_start,
                                                             int32_t* __restrict__ task_count,
                                                             int64_t* __restrict__ n_tasks,
                                                             int64_t* __restrict__ n_live,
                                                             const int64_t* __restrict__ n_kept, int* counter,
                                                             BatchClock* clock, int64_t advanced) {
    __shared__ int64_t s_slots[1024], s_tasks[1024];
    __shared__ int64_t base_slot, base_task;
    if (threadIdx.x == 0) {
        base_slot = 0;
        base_task = 0;
    }
    __syncthreads();
    for (int s0 = 0; s0 < n_sys; s0 += 1024) {
        const int s = s0 + threadIdx.x;
        const int64_t c = s < n_sys ? cnt[s] : 0;
        const int64_t nt = (c + 31) / 32;
        s_slots[threadIdx.x] = c;
        s_tasks[threadIdx.x] = nt;
        __syncthreads();
        // inclusive scans (Hillis-Steele) over the 1024 entries
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t a = threadIdx.x >= o ? s_slots[threadIdx.x - o] : 0;
            const int64_t b = threadIdx.x >= o ? s_tasks[threadIdx.x - o] : 0;
            __syncthreads();
            s_slots[threadIdx.x] += a;
            s_tasks[threadIdx.x] += b;
            __syncthreads();
        }
        const int64_t slot0 = base_slot + s_slots[threadIdx.x] - c;
        const int64_t task0 = base_task + s_tasks[threadIdx.x] - nt;
        for (int64_t k = 0; k < nt; ++k) {
            task_sys[task0 + k] = s;
            task_start[task0 + k] = slot0 + 32 * k;
            const int64_t rest = c - 32 * k;
            task_count[task0 + k] = (int32_t)(rest < 32 ? rest : 32);
        }
        if (s < n_sys) cnt[s] = 0;
        __syncthreads();
        if (threadIdx.x == 1023) {
            base_slot += s_slots[1023];
            base_task += s_tasks[1023];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *n_tasks = base_task;
        *n_live = n_kept ? *n_kept : base_slot;
        *counter = 0;
        clock->step += advanced;
        if (advanced > 0) clock->test_first = 0;
    }
}

}  // namespace glisse

using namespace glisse;

namespace {
constexpr double kG = 4.0 * 3.14159265358979323846 * 3.14159265358979323846;

struct Snapshot {
    double* st = nullptr;
    int32_t* id = nullptr;
    uint8_t* alive = nullptr;
    double* jac = nullptr;
    double* out_state = nullptr;
    int64_t* out_step = nullptr;
    int32_t* out_reason = nullptr;
    int64_t* cnt = nullptr;
    BatchClock clock{};
};
}  // namespace

struct glisse_batch {
    int device = 0;
    cudaStream_t s = nullptr;
    bool own_s = false;
    glisse_opts o{};
    int n_sys = 0;
    int C = 1024;
    int threads = 128;
    int blocks = 0;
    int tpp = 1;  // lanes per particle in the particle kernel (1 or 2)
    int n_sm = 0;
    int64_t n_total = 0, cap = 0, n_live = 0, step = 0;
    std::vector<int> np_host;       // internal system order
    std::vector<int> order;         // internal index -> caller's system index
    PlanetConsts* d_pcs = nullptr;
    ParticleConsts* d_ppcs = nullptr;
    int32_t* d_np = nullptr;
    double* d_jac = nullptr;
    double* d_dt = nullptr;
    double* d_log = nullptr;
    int64_t* d_log_off = nullptr;
    int64_t log_len = 0;
    int* d_status = nullptr;
    double* d_st[2] = {};
    int32_t* d_id[2] = {};
    int cur = 0;
    uint8_t* d_alive = nullptr;
    double* d_out_state = nullptr;
    int64_t* d_out_step = nullptr;
    int32_t* d_out_reason = nullptr;
    int64_t* d_cnt = nullptr;
    int32_t* d_task_sys = nullptr;
    int64_t* d_task_start = nullptr;
    int32_t* d_task_count = nullptr;
    int64_t max_tasks = 0;
    int64_t* d_n_tasks = nullptr;
    int* d_counter = nullptr;
    BatchClock* d_clock = nullptr;
    int64_t* d_nlive = nullptr;
    int64_t* d_nkept = nullptr;
    int64_t* d_counts = nullptr;
    unsigned long long* d_steps = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    bool timing = false;
    cudaEvent_t ev[8] = {};
    glisse_timing acc{};
};

#define GB_CUDA(x)                    \
    do {                              \
        cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) {      \
            (void)cudaGetLastError(); \
            return GLISSE_E_CUDA;     \
        }                             \
    } while (0)

static int b_alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return GLISSE_E_NOMEM;
    }
    return e == cudaSuccess ? GLISSE_OK : GLISSE_E_CUDA;
}
#define GB_ALLOC(ptr, bytes)                                              \
    do {                                                                  \
        int r_ = b_alloc(reinterpret_cast<void**>(&(ptr)), (bytes));      \
        if (r_ != GLISSE_OK) return r_;                                   \
    } while (0)

static void drop_graphs(glisse_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

static void batch_free(glisse_batch* b) {
    if (!b) return;
    if (b->s) cudaStreamSynchronize(b->s);
    drop_graphs(b);
    void* ptrs[] = {b->d_pcs, b->d_ppcs, b->d_np, b->d_jac, b->d_dt, b->d_log, b->d_log_off, b->d_status,
                    b->d_st[0], b->d_st[1], b->d_id[0], b->d_id[1], b->d_alive, b->d_out_state, b->d_out_step,
                    b->d_out_reason, b->d_cnt, b->d_task_sys, b->d_task_start, b->d_task_count, b->d_n_tasks,
                    b->d_counter, b->d_clock, b->d_nlive, b->d_nkept, b->d_counts, b->d_steps};
    for (void* p : ptrs) cudaFree(p);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_s && b->s) cudaStreamDestroy(b->s);
    delete b;
}

extern "C" void glisse_batch_destroy(glisse_batch* b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    batch_free(b);
    cudaSetDevice(prev);
}

static int set_launch_shape(glisse_batch* b, int threads, int tpp) {
    if (threads < 32 || threads > 256 || threads % 32 || (tpp != 1 && tpp != 2)) return GLISSE_E_INVAL;
    int per_sm = 0;
    GB_CUDA(batch_particles_occupancy(threads, tpp, &per_sm));
    if (per_sm < 1) return GLISSE_E_INVAL;
    b->threads = threads;
    b->tpp = tpp;
    b->blocks = per_sm * b->n_sm;
    return GLISSE_OK;
}

// Enqueue one chunk of m steps (no host synchronisation).  In timing mode each
// stage is bracketed by events and the stream is synchronised afterwards.
static int enqueue_chunk(glisse_batch* b, int m) {
    const int nxt = b->cur ^ 1;
    cudaStream_t s = b->s;
    if (b->timing) GB_CUDA(cudaEventRecord(b->ev[0], s));
    GB_CUDA(launch_eph_batch(b->d_pcs, b->n_sys, b->d_jac, b->d_dt, m, b->d_log, b->d_log_off, b->d_status, s));
    if (b->timing) GB_CUDA(cudaEventRecord(b->ev[1], s));
    BatchArgs a;
    a.pcs = b->d_ppcs;
    a.np_of = b->d_np;
    a.log = b->d_log;
    a.log_off = b->d_log_off;
    a.task_sys = b->d_task_sys;
    a.task_start = b->d_task_start;
    a.task_count = b->d_task_count;
    a.n_tasks = b->d_n_tasks;
    a.counter = b->d_counter;
    a.clock = b->d_clock;
    a.ld = b->cap;
    a.st = b->d_st[b->cur];
    a.id = b->d_id[b->cur];
    a.alive = b->d_alive;
    a.cnt_new = b->d_cnt;
    a.nsteps = m;
    a.out_state = b->d_out_state;
    a.out_step = b->d_out_step;
    a.out_reason = b->d_out_reason;
    a.steps_done = b->d_steps;
    GB_CUDA(launch_batch_particles(a, b->blocks, b->threads, b->tpp, s));
    if (b->timing) GB_CUDA(cudaEventRecord(b->ev[2], s));
    const unsigned tiles = (unsigned)((b->cap + kBTile - 1) / kBTile);
    bpart_count_kernel<<<tiles, kBThreads, 0, s>>>(b->d_alive, b->d_nlive, b->d_counts);
    bpart_scan_kernel<<<1, 1024, 0, s>>>(b->d_counts, b->d_nlive, b->d_nkept);
    bpart_scatter_kernel<<<tiles, kBThreads, 0, s>>>(b->d_alive, b->d_nlive, b->d_counts, b->d_st[b->cur],
                                                      b->d_id[b->cur], b->d_st[nxt], b->d_id[nxt], b->cap);
    bpart_flags_kernel<<<2 * b->n_sm, 256, 0, s>>>(b->d_alive, b->d_nkept, b->cap);
    batch_tasks_kernel<<<1, 1024, 0, s>>>(b->n_sys, b->d_cnt, b->d_task_sys, b->d_task_start, b->d_task_count,
                                          b->d_n_tasks, b->d_nlive, b->d_nkept, b->d_counter, b->d_clock, m);
    GB_CUDA(cudaGetLastError());
    if (b->timing) {
        GB_CUDA(cudaEventRecord(b->ev[3], s));
        GB_CUDA(cudaEventSynchronize(b->ev[3]));
        float t01 = 0, t12 = 0, t23 = 0;
        GB_CUDA(cudaEventElapsedTime(&t01, b->ev[0], b->ev[1]));
        GB_CUDA(cudaEventElapsedTime(&t12, b->ev[1], b->ev[2]));
        GB_CUDA(cudaEventElapsedTime(&t23, b->ev[2], b->ev[3]));
        b->acc.ephemeris_ms += t01;
        ++b->acc.ephemeris_launches;
        b->acc.particle_ms += t12;
        ++b->acc.particle_launches;
        b->acc.compact_ms += t23;
        ++b->acc.compact_launches;
        unsigned long long st = 0;
        GB_CUDA(cudaMemcpy(&st, b->d_steps, sizeof(st), cudaMemcpyDeviceToHost));
        b->acc.particle_steps = (int64_t)st;
    }
    return GLISSE_OK;
}

static int run_chunk(glisse_batch* b, int m) {
    if (b->timing) return enqueue_chunk(b, m);
    const auto key = std::make_pair(b->cur, m);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        GB_CUDA(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_chunk(b, m);
        cudaError_t e = cudaStreamEndCapture(b->s, &g);
        if (rc != GLISSE_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return GLISSE_E_CUDA;
        }
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return GLISSE_E_CUDA;
        }
        it = b->graphs.emplace(key, ge).first;
    }
    GB_CUDA(cudaGraphLaunch(it->second, b->s));
    return GLISSE_OK;
}

static int refresh_host_counts(glisse_batch* b) {
    int status = 0;
    GB_CUDA(cudaMemcpyAsync(&b->n_live, b->d_nlive, sizeof(int64_t), cudaMemcpyDeviceToHost, b->s));
    GB_CUDA(cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->s));
    GB_CUDA(cudaStreamSynchronize(b->s));
    return status;
}

// Stream (the caller's or an own one), SM count and timing events of a batch.
static int batch_streams(glisse_batch* b) {
    GB_CUDA(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
    b->own_s = true;
    if (b->o.cuda_stream) {
        cudaStreamDestroy(b->s);
        b->s = static_cast<cudaStream_t>(b->o.cuda_stream);
        b->own_s = false;
    }
    GB_CUDA(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device));
    if (b->timing)
        for (auto& e : b->ev) GB_CUDA(cudaEventCreate(&e));
    return GLISSE_OK;
}

// Device buffers of a batch whose n_sys, np_host (internal order), C and n_total are
// set; log_off receives each system's offset in the planet log (doubles).
static int batch_alloc(glisse_batch* b, std::vector<int64_t>& log_off) {
    const int n = b->n_sys;
    // buffers
    b->cap = std::max<int64_t>(b->n_total, 1);
    log_off.assign(n, 0);
    int64_t L = 0;
    for (int k = 0; k < n; ++k) {
        log_off[k] = L;
        L += (int64_t)(b->C + 1) * log_stride(b->np_host[k]);
    }
    b->log_len = L;
    b->max_tasks = b->cap / 32 + n + 1;
    GB_ALLOC(b->d_pcs, sizeof(PlanetConsts) * n);
    GB_ALLOC(b->d_ppcs, sizeof(ParticleConsts) * n);
    GB_ALLOC(b->d_np, sizeof(int32_t) * n);
    GB_ALLOC(b->d_jac, sizeof(double) * 6 * kMaxPlanets * n);
    GB_ALLOC(b->d_dt, sizeof(double) * n);
    GB_ALLOC(b->d_log, sizeof(double) * std::max<int64_t>(L, 1));
    GB_ALLOC(b->d_log_off, sizeof(int64_t) * n);
    GB_ALLOC(b->d_status, sizeof(int) * (n + 1));
    for (int k = 0; k < 2; ++k) {
        GB_ALLOC(b->d_st[k], sizeof(double) * 6 * b->cap);
        GB_ALLOC(b->d_id[k], sizeof(int32_t) * b->cap);
    }
    GB_ALLOC(b->d_alive, b->cap);
    GB_ALLOC(b->d_out_state, sizeof(double) * 6 * b->cap);
    GB_ALLOC(b->d_out_step, sizeof(int64_t) * b->cap);
    GB_ALLOC(b->d_out_reason, sizeof(int32_t) * b->cap);
    GB_ALLOC(b->d_cnt, sizeof(int64_t) * n);
    GB_ALLOC(b->d_task_sys, sizeof(int32_t) * b->max_tasks);
    GB_ALLOC(b->d_task_start, sizeof(int64_t) * b->max_tasks);
    GB_ALLOC(b->d_task_count, sizeof(int32_t) * b->max_tasks);
    GB_ALLOC(b->d_n_tasks, sizeof(int64_t));
    GB_ALLOC(b->d_counter, sizeof(int));
    GB_ALLOC(b->d_clock, sizeof(BatchClock));
    GB_ALLOC(b->d_nlive, sizeof(int64_t));
    GB_ALLOC(b->d_nkept, sizeof(int64_t));
    GB_ALLOC(b->d_counts, sizeof(int64_t) * ((b->cap + kBTile - 1) / kBTile + 1));
    GB_ALLOC(b->d_steps, sizeof(unsigned long long));
    GB_CUDA(cudaMemsetAsync(b->d_steps, 0, sizeof(unsigned long long), b->s));
    GB_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int) * (n + 1), b->s));
    return GLISSE_OK;
}

static int batch_setup(glisse_batch* b, const double* star_mass, const int32_t* n_planets, const double* planets,
                       const int64_t* n_particles, const double* particles, const double* dt) {
    const int n = b->n_sys;
    const int src = batch_streams(b);
    if (src) return src;
    // internal order: decreasing planet count (stable)
    std::vector<int64_t> pl_off(n + 1, 0), pa_off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        pl_off[i + 1] = pl_off[i] + n_planets[i];
        pa_off[i + 1] = pa_off[i] + n_particles[i];
    }
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return n_planets[a] > n_planets[c]; });
    b->np_host.resize(n);
    for (int k = 0; k < n; ++k) b->np_host[k] = n_planets[b->order[k]];
    std::vector<int64_t> log_off;
    int arc = batch_alloc(b, log_off);
    if (arc) return arc;

    // planets: set-up kernel per system (constants, Jacobi state, encounter radii)
    std::vector<double> hpl(std::max<int64_t>(pl_off[n], 1) * 7);
    std::vector<double> hdt(n), hm0(n);
    std::vector<int64_t> hpl_off(n);
    int64_t q = 0;
    for (int k = 0; k < n; ++k) {
        const int src = b->order[k];
        hpl_off[k] = q;
        std::memcpy(&hpl[q * 7], planets + pl_off[src] * 7, sizeof(double) * 7 * n_planets[src]);
        q += n_planets[src];
        hdt[k] = dt[src];
        hm0[k] = star_mass[src];
    }
    double* d_pl = nullptr;
    GB_ALLOC(d_pl, sizeof(double) * hpl.size());
    cudaError_t e = cudaMemcpyAsync(d_pl, hpl.data(), sizeof(double) * hpl.size(), cudaMemcpyHostToDevice, b->s);
    for (int k = 0; k < n && e == cudaSuccess; ++k)
        e = launch_eph_setup(d_pl + hpl_off[k] * 7, b->np_host[k], hm0[k], kG, b->o.enc_mode, b->o.enc_value,
                             b->d_pcs + k, b->d_jac + (size_t)k * 6 * kMaxPlanets, b->d_status + 1 + k, b->s);
    std::vector<PlanetConsts> hpc(n);
    std::vector<int> st(n + 1, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hpc.data(), b->d_pcs, sizeof(PlanetConsts) * n, cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st.data(), b->d_status, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    cudaFree(d_pl);
    if (e != cudaSuccess) return GLISSE_E_CUDA;
    for (int k = 0; k < n; ++k)
        if (st[1 + k] != 0) return st[1 + k];
    std::vector<ParticleConsts> hppc(n);
    for (int k = 0; k < n; ++k) {
        ParticleConsts& p = hppc[k];
        std::memset(&p, 0, sizeof(p));
        p.mu = hpc[k].mu0;
        p.dt = hdt[k];
        p.half_dt = 0.5 * hdt[k];
        for (int j = 0; j < b->np_host[k]; ++j) {
            p.tgm_full[j] = hdt[k] * hpc[k].gm[j];
            p.tgm_half[j] = 0.5 * hdt[k] * hpc[k].gm[j];
            p.rc2[j] = hpc[k].rcrit[j] * hpc[k].rcrit[j];
        }
        p.rmax2 = b->o.r_max > 0.0 ? b->o.r_max * b->o.r_max : 0.0;
        p.rmax = b->o.r_max > 0.0 ? b->o.r_max : 0.0;
    }
    std::vector<int32_t> np32(b->np_host.begin(), b->np_host.end());
    GB_CUDA(cudaMemcpyAsync(b->d_ppcs, hppc.data(), sizeof(ParticleConsts) * n, cudaMemcpyHostToDevice, b->s));
    GB_CUDA(cudaMemcpyAsync(b->d_np, np32.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->s));
    GB_CUDA(cudaMemcpyAsync(b->d_dt, hdt.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->s));
    GB_CUDA(cudaMemcpyAsync(b->d_log_off, log_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, b->s));

    // particles in internal system order; ids = the caller's row index
    std::vector<int64_t> cnt(n);
    if (b->n_total > 0) {
        std::vector<double> hpa((size_t)b->n_total * 6);
        std::vector<int32_t> hid((size_t)b->n_total);
        int64_t r = 0;
        for (int k = 0; k < n; ++k) {
            const int src = b->order[k];
            std::memcpy(&hpa[r * 6], particles + pa_off[src] * 6, sizeof(double) * 6 * n_particles[src]);
            for (int64_t i = 0; i < n_particles[src]; ++i) hid[r + i] = (int32_t)(pa_off[src] + i);
            r += n_particles[src];
        }
        double* d_aos = nullptr;
        GB_ALLOC(d_aos, sizeof(double) * hpa.size());
        e = cudaMemcpyAsync(d_aos, hpa.data(), sizeof(double) * hpa.size(), cudaMemcpyHostToDevice, b->s);
        if (e == cudaSuccess) e = launch_import(b->n_total, d_aos, b->d_st[0], b->cap, b->d_id[0], b->s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_id[0], hid.data(), sizeof(int32_t) * hid.size(), cudaMemcpyHostToDevice, b->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
        cudaFree(d_aos);
        if (e != cudaSuccess) return GLISSE_E_CUDA;
    }
    for (int k = 0; k < n; ++k) cnt[k] = n_particles[b->order[k]];
    GB_CUDA(cudaMemcpyAsync(b->d_cnt, cnt.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, b->s));
    GB_CUDA(cudaMemsetAsync(b->d_alive, 1, b->cap, b->s));
    GB_CUDA(cudaMemsetAsync(b->d_out_state, 0, sizeof(double) * 6 * b->cap, b->s));
    GB_CUDA(cudaMemsetAsync(b->d_out_step, 0xFF, sizeof(int64_t) * b->cap, b->s));
    GB_CUDA(cudaMemsetAsync(b->d_out_reason, 0, sizeof(int32_t) * b->cap, b->s));
    BatchClock clk{0, 1, 0};
    GB_CUDA(cudaMemcpyAsync(b->d_clock, &clk, sizeof(clk), cudaMemcpyHostToDevice, b->s));
    batch_tasks_kernel<<<1, 1024, 0, b->s>>>(n, b->d_cnt, b->d_task_sys, b->d_task_start, b->d_task_count,
                                              b->d_n_tasks, b->d_nlive, nullptr, b->d_counter, b->d_clock, 0);
    GB_CUDA(cudaGetLastError());
    int rc = set_launch_shape(b, 128, 1);
    if (rc) return rc;
    rc = refresh_host_counts(b);
    return rc;
}

extern "C" int glisse_batch_create(glisse_batch** out, int32_t n_systems, const double* star_mass,
                                   const int32_t* n_planets, const double* planets, const int64_t* n_particles,
                                   const double* particles, const double* dt, const glisse_opts* opts) {
    glisse::NvtxRange range("glisse_batch_create");
    if (!out) return GLISSE_E_INVAL;
    *out = nullptr;
    glisse_opts o;
    glisse_opts_default(&o);
    if (opts) o = *opts;
    if (n_systems < 1 || !star_mass || !n_planets || !n_particles || !dt) return GLISSE_E_INVAL;
    if (o.chunk_steps < 1 || o.chunk_steps > (1 << 20)) return GLISSE_E_INVAL;
    if (o.kepler_mode != GLISSE_KEPLER_CONVERGE) return GLISSE_E_INVAL;  // batches use the converged solver
    if (o.sort_mode != GLISSE_SORT_NONE) return GLISSE_E_INVAL;          // and keep each system's order
    if (o.enc_mode != GLISSE_ENC_HILL && o.enc_mode != GLISSE_ENC_FIXED) return GLISSE_E_INVAL;
    if (!(o.enc_value >= 0.0) || !std::isfinite(o.enc_value) || !std::isfinite(o.r_max)) return GLISSE_E_INVAL;
    int64_t tot_pl = 0, tot_pa = 0;
    for (int i = 0; i < n_systems; ++i) {
        if (!(star_mass[i] > 0.0) || !std::isfinite(star_mass[i])) return GLISSE_E_INVAL;
        if (n_planets[i] < 0 || n_planets[i] > GLISSE_MAX_PLANETS || n_particles[i] < 0) return GLISSE_E_INVAL;
        if (!(dt[i] != 0.0) || !std::isfinite(dt[i])) return GLISSE_E_INVAL;
        tot_pl += n_planets[i];
        tot_pa += n_particles[i];
    }
    if (tot_pa > INT32_MAX) return GLISSE_E_INVAL;
    if ((tot_pl > 0 && !planets) || (tot_pa > 0 && !particles)) return GLISSE_E_INVAL;
    for (int64_t k = 0; k < 7 * tot_pl; ++k)
        if (!std::isfinite(planets[k])) return GLISSE_E_INVAL;
    for (int64_t j = 0; j < tot_pl; ++j)
        if (!(planets[7 * j] >= 0.0)) return GLISSE_E_INVAL;
    glisse_batch* b = new (std::nothrow) glisse_batch();
    if (!b) return GLISSE_E_NOMEM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return GLISSE_E_CUDA;
    }
    b->o = o;
    b->n_sys = n_systems;
    b->C = o.chunk_steps;
    b->n_total = tot_pa;
    b->timing = o.timing != 0;
    int rc = batch_setup(b, star_mass, n_planets, planets, n_particles, particles, dt);
    if (rc != GLISSE_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return GLISSE_OK;
}

extern "C" int glisse_batch_advance(glisse_batch* b, int64_t n_steps) {
    glisse::NvtxRange range("glisse_batch_advance");
    if (!b || n_steps < 0) return GLISSE_E_INVAL;
    int64_t remaining = n_steps;
    while (remaining > 0) {
        const int m = (int)std::min<int64_t>(remaining, b->C);
        int rc = run_chunk(b, m);
        if (rc) return rc;
        b->cur ^= 1;
        b->step += m;
        remaining -= m;
    }
    return refresh_host_counts(b);
}

extern "C" int glisse_batch_read(glisse_batch* b, double* state, uint8_t* alive, int64_t* removal_step,
                                 int32_t* removal_reason) {
    if (!b) return GLISSE_E_INVAL;
    const int64_t n = b->n_total;
    if (n == 0) return GLISSE_OK;
    GB_CUDA(launch_export_live(b->n_live, b->d_st[b->cur], b->cap, b->d_id[b->cur], b->d_out_state, b->s));
    std::vector<int64_t> tmp;
    int64_t* steps = removal_step;
    if (!steps && alive) {
        tmp.resize(n);
        steps = tmp.data();
    }
    if (state) GB_CUDA(cudaMemcpyAsync(state, b->d_out_state, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, b->s));
    if (steps) GB_CUDA(cudaMemcpyAsync(steps, b->d_out_step, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, b->s));
    if (removal_reason)
        GB_CUDA(cudaMemcpyAsync(removal_reason, b->d_out_reason, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->s));
    GB_CUDA(cudaStreamSynchronize(b->s));
    if (alive)
        for (int64_t i = 0; i < n; ++i) alive[i] = steps[i] < 0 ? 1 : 0;
    return GLISSE_OK;
}

extern "C" int glisse_batch_status(glisse_batch* b, int64_t* n_live, int64_t* step) {
    if (!b) return GLISSE_E_INVAL;
    if (n_live) *n_live = b->n_live;
    if (step) *step = b->step;
    return GLISSE_OK;
}

extern "C" int glisse_batch_steps_done(glisse_batch* b, int64_t* steps) {
    if (!b || !steps) return GLISSE_E_INVAL;
    unsigned long long st = 0;
    GB_CUDA(cudaStreamSynchronize(b->s));
    GB_CUDA(cudaMemcpy(&st, b->d_steps, sizeof(st), cudaMemcpyDeviceToHost));
    *steps = (int64_t)st;
    return GLISSE_OK;
}

extern "C" int glisse_batch_timings(glisse_batch* b, glisse_timing* out, int32_t reset) {
    if (!b) return GLISSE_E_INVAL;
    if (!b->timing) return GLISSE_E_STATE;
    if (out) *out = b->acc;
    if (reset) {
        std::memset(&b->acc, 0, sizeof(b->acc));
        GB_CUDA(cudaMemsetAsync(b->d_steps, 0, sizeof(unsigned long long), b->s));
        GB_CUDA(cudaStreamSynchronize(b->s));
    }
    return GLISSE_OK;
}

// ---- autotuner -----------------------------------------------------------------
static int snap_alloc(glisse_batch* b, Snapshot& sn) {
    GB_ALLOC(sn.st, sizeof(double) * 6 * b->cap);
    GB_ALLOC(sn.id, sizeof(int32_t) * b->cap);
    GB_ALLOC(sn.alive, b->cap);
    GB_ALLOC(sn.jac, sizeof(double) * 6 * kMaxPlanets * b->n_sys);
    GB_ALLOC(sn.out_state, sizeof(double) * 6 * b->cap);
    GB_ALLOC(sn.out_step, sizeof(int64_t) * b->cap);
    GB_ALLOC(sn.out_reason, sizeof(int32_t) * b->cap);
    GB_ALLOC(sn.cnt, sizeof(int64_t) * b->n_sys);
    return GLISSE_OK;
}

static void snap_free(Snapshot& sn) {
    void* ptrs[] = {sn.st, sn.id, sn.alive, sn.jac, sn.out_state, sn.out_step, sn.out_reason, sn.cnt};
    for (void* p : ptrs) cudaFree(p);
}

// save (to_snap) or restore the mutable state; both on the batch's stream
static int snap_copy(glisse_batch* b, Snapshot& sn, bool to_snap) {
    auto cp = [&](void* live, void* snap, size_t bytes) {
        return cudaMemcpyAsync(to_snap ? snap : live, to_snap ? live : snap, bytes, cudaMemcpyDeviceToDevice, b->s);
    };
    GB_CUDA(cp(b->d_st[b->cur], sn.st, sizeof(double) * 6 * b->cap));
    GB_CUDA(cp(b->d_id[b->cur], sn.id, sizeof(int32_t) * b->cap));
    GB_CUDA(cp(b->d_alive, sn.alive, b->cap));
    GB_CUDA(cp(b->d_jac, sn.jac, sizeof(double) * 6 * kMaxPlanets * b->n_sys));
    GB_CUDA(cp(b->d_out_state, sn.out_state, sizeof(double) * 6 * b->cap));
    GB_CUDA(cp(b->d_out_step, sn.out_step, sizeof(int64_t) * b->cap));
    GB_CUDA(cp(b->d_out_reason, sn.out_reason, sizeof(int32_t) * b->cap));
    if (to_snap) {
        GB_CUDA(cudaMemcpyAsync(&sn.clock, b->d_clock, sizeof(BatchClock), cudaMemcpyDeviceToHost, b->s));
    } else {
        GB_CUDA(cudaMemcpyAsync(b->d_clock, &sn.clock, sizeof(BatchClock), cudaMemcpyHostToDevice, b->s));
        // task table and live counts from the restored live count per system
        GB_CUDA(cudaMemcpyAsync(b->d_cnt, sn.cnt, sizeof(int64_t) * b->n_sys, cudaMemcpyDeviceToDevice, b->s));
        batch_tasks_kernel<<<1, 1024, 0, b->s>>>(b->n_sys, b->d_cnt, b->d_task_sys, b->d_task_start,
                                                  b->d_task_count, b->d_n_tasks, b->d_nlive, nullptr, b->d_counter,
                                                  b->d_clock, 0);
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaStreamSynchronize(b->s));
    return GLISSE_OK;
}

// per-system live counts of the current layout (from the task table)
__global__ void batch_counts_from_tasks(const int32_t* __restrict__ task_sys, const int32_t* __restrict__ task_count,
                                        const int64_t* __restrict__ n_tasks, int64_t* __restrict__ cnt) {
    const int64_t nt = *n_tasks;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + task_sys[t]), (unsigned long long)task_count[t]);
}

extern "C" int glisse_batch_tune(glisse_batch* b, int32_t trial_steps, int32_t* chunk_steps, int32_t* block_threads,
                                 int32_t* threads_per_particle) {
    glisse::NvtxRange range("glisse_batch_tune");
    if (!b) return GLISSE_E_INVAL;
    if (trial_steps <= 0) trial_steps = 256;
    Snapshot sn;
    int rc = snap_alloc(b, sn);
    if (rc) {
        snap_free(sn);
        return rc;
    }
    GB_CUDA(cudaMemsetAsync(sn.cnt, 0, sizeof(int64_t) * b->n_sys, b->s));
    batch_counts_from_tasks<<<2 * b->n_sm, 256, 0, b->s>>>(b->d_task_sys, b->d_task_count, b->d_n_tasks, sn.cnt);
    rc = snap_copy(b, sn, true);
    const int cur0 = b->cur, C0 = b->C, T0 = b->threads, P0 = b->tpp;
    const int64_t step0 = b->step;
    const bool timing0 = b->timing;
    b->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = GLISSE_E_CUDA;
    double best = -1.0;
    int bestC = C0, bestT = T0, bestP = P0;
    auto trial = [&](int C, int T, int P, int64_t steps, double* rate) -> int {
        int r = set_launch_shape(b, T, P);
        if (r) return r;
        r = snap_copy(b, sn, false);
        if (r) return r;
        b->cur = cur0;
        unsigned long long s0 = 0, s1 = 0;
        GB_CUDA(cudaMemcpy(&s0, b->d_steps, sizeof(s0), cudaMemcpyDeviceToHost));
        GB_CUDA(cudaEventRecord(e0, b->s));
        for (int64_t left = steps; left > 0;) {
            const int m = (int)std::min<int64_t>(left, C);
            r = enqueue_chunk(b, m);
            if (r) return r;
            b->cur ^= 1;
            left -= m;
        }
        GB_CUDA(cudaEventRecord(e1, b->s));
        GB_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        GB_CUDA(cudaMemcpy(&s1, b->d_steps, sizeof(s1), cudaMemcpyDeviceToHost));
        *rate = (double)(s1 - s0) / (ms * 1e-3);
        return GLISSE_OK;
    };
    // block size and lanes per particle at the current chunk length, then the chunk length
    const int Ts[3] = {64, 128, 256};
    for (int k = 0; k < 3 && !rc; ++k) {
        double rate = 0;
        rc = trial(C0, Ts[k], 1, trial_steps, &rate);
        if (!rc && rate > best) {
            best = rate;
            bestT = Ts[k];
            bestP = 1;
        }
    }
    if (!rc) {
        double rate = 0;
        rc = trial(C0, bestT, 2, trial_steps, &rate);
        if (!rc && rate > best) {
            best = rate;
            bestP = 2;
        }
    }
    best = -1.0;
    const int Cs[4] = {256, 512, 1024, 2048};
    for (int k = 0; k < 4 && !rc; ++k) {
        if (Cs[k] > C0) {
            // the log buffers hold C0 + 1 steps per system; longer chunks need a new batch
            continue;
        }
        double rate = 0;
        rc = trial(Cs[k], bestT, bestP, std::max<int64_t>(2 * Cs[k], trial_steps), &rate);
        if (!rc && rate > best) {
            best = rate;
            bestC = Cs[k];
        }
    }
    // put the state back and keep the choice
    if (!rc) rc = snap_copy(b, sn, false);
    b->cur = cur0;
    b->step = step0;
    b->timing = timing0;
    if (!rc) rc = set_launch_shape(b, bestT, bestP);
    if (!rc) {
        b->C = bestC;
        drop_graphs(b);
        rc = refresh_host_counts(b);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    snap_free(sn);
    if (chunk_steps) *chunk_steps = b->C;
    if (block_threads) *block_threads = b->threads;
    if (threads_per_particle) *threads_per_particle = b->tpp;
    return rc;
}

extern "C" int glisse_batch_set_launch(glisse_batch* b, int32_t block_threads, int32_t threads_per_particle) {
    if (!b) return GLISSE_E_INVAL;
    const int rc = set_launch_shape(b, block_threads, threads_per_particle);
    if (rc == GLISSE_OK) drop_graphs(b);
    return rc;
}

// ---- checkpoint / resume ----------------------------------------------------------
// Buffer: a fixed header, then (each at an 8-byte offset) the internal system
// order [n_sys] and planet counts [n_sys] (int32), the planet and particle
// constants [n_sys], the steps dt [n_sys], the planets' Jacobi states
// [n_sys][kMaxPlanets][6], the live particles per system [n_sys] (int64), the
// particle slots [6][n_live], slot ids [n_live], slot flags [n_live], and the
// per-id frozen states [n_total][6], removal steps and reasons.  Between calls
// the planets and particles of every system are at the same step (the planet
// chunks run inside each chunk), so the Jacobi states are the current ones.
namespace {
constexpr char kBCkptMagic[8] = {'G', 'L', 'I', 'S', 'S', 'E', 'B', 'K'};
constexpr int32_t kBCkptVersion = 1;

struct BCkptHeader {
    char magic[8];
    int32_t version, header_bytes;
    int32_t n_sys, chunk_steps, threads, tpp, enc_mode, pad;
    double enc_value, r_max;
    int64_t n_total, n_live, step, total_bytes;
    BatchClock clock;
};

struct BCkptLayout {
    size_t order, np, pcs, ppcs, dt, jac, cnt, st, id, alive, out_state, out_step, out_reason, total;
};

BCkptLayout bckpt_layout(int n_sys, int64_t n_total, int64_t n_live) {
    BCkptLayout L{};
    size_t off = (sizeof(BCkptHeader) + 7) & ~size_t(7);
    auto take = [&off](size_t bytes) {
        const size_t o = off;
        off += (bytes + 7) & ~size_t(7);
        return o;
    };
    const size_t n = (size_t)n_sys;
    L.order = take(sizeof(int32_t) * n);
    L.np = take(sizeof(int32_t) * n);
    L.pcs = take(sizeof(PlanetConsts) * n);
    L.ppcs = take(sizeof(ParticleConsts) * n);
    L.dt = take(sizeof(double) * n);
    L.jac = take(sizeof(double) * 6 * kMaxPlanets * n);
    L.cnt = take(sizeof(int64_t) * n);
    L.st = take(sizeof(double) * 6 * (size_t)n_live);
    L.id = take(sizeof(int32_t) * (size_t)n_live);
    L.alive = take((size_t)n_live);
    L.out_state = take(sizeof(double) * 6 * (size_t)n_total);
    L.out_step = take(sizeof(int64_t) * (size_t)n_total);
    L.out_reason = take(sizeof(int32_t) * (size_t)n_total);
    L.total = off;
    return L;
}
}  // namespace

extern "C" int glisse_batch_sizes(glisse_batch* b, int64_t* n_particles, int32_t* n_systems) {
    if (!b) return GLISSE_E_INVAL;
    if (n_particles) *n_particles = b->n_total;
    if (n_systems) *n_systems = b->n_sys;
    return GLISSE_OK;
}

extern "C" int glisse_batch_checkpoint_size(glisse_batch* b, int64_t* bytes) {
    if (!b || !bytes) return GLISSE_E_INVAL;
    *bytes = (int64_t)bckpt_layout(b->n_sys, b->n_total, b->n_live).total;
    return GLISSE_OK;
}

extern "C" int glisse_batch_checkpoint(glisse_batch* b, void* buf, int64_t bytes) {
    glisse::NvtxRange range("glisse_batch_checkpoint");
    if (!b || !buf) return GLISSE_E_INVAL;
    const int n = b->n_sys;
    const BCkptLayout L = bckpt_layout(n, b->n_total, b->n_live);
    if (bytes < (int64_t)L.total) return GLISSE_E_INVAL;
    char* out = static_cast<char*>(buf);
    std::memset(out, 0, L.total);  // the gaps between arrays too: equal batches, equal bytes
    // live particles per system in the current layout, from the task table
    int64_t* d_cnt = nullptr;
    GB_ALLOC(d_cnt, sizeof(int64_t) * n);
    cudaError_t e = cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * n, b->s);
    if (e == cudaSuccess) {
        batch_counts_from_tasks<<<2 * b->n_sm, 256, 0, b->s>>>(b->d_task_sys, b->d_task_count, b->d_n_tasks, d_cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    BCkptHeader h;
    std::memset(&h, 0, sizeof(h));
    auto d2h = [&](size_t off, const void* src, size_t nbytes) {
        if (e == cudaSuccess && nbytes > 0) e = cudaMemcpy(out + off, src, nbytes, cudaMemcpyDeviceToHost);
    };
    d2h(L.cnt, d_cnt, sizeof(int64_t) * n);
    d2h(L.pcs, b->d_pcs, sizeof(PlanetConsts) * n);
    d2h(L.ppcs, b->d_ppcs, sizeof(ParticleConsts) * n);
    d2h(L.dt, b->d_dt, sizeof(double) * n);
    d2h(L.jac, b->d_jac, sizeof(double) * 6 * kMaxPlanets * n);
    d2h(L.id, b->d_id[b->cur], sizeof(int32_t) * (size_t)b->n_live);
    d2h(L.alive, b->d_alive, (size_t)b->n_live);
    d2h(L.out_state, b->d_out_state, sizeof(double) * 6 * (size_t)b->n_total);
    d2h(L.out_step, b->d_out_step, sizeof(int64_t) * (size_t)b->n_total);
    d2h(L.out_reason, b->d_out_reason, sizeof(int32_t) * (size_t)b->n_total);
    if (e == cudaSuccess && b->n_live > 0)
        e = cudaMemcpy2D(out + L.st, sizeof(double) * (size_t)b->n_live, b->d_st[b->cur], sizeof(double) * b->cap,
                         sizeof(double) * (size_t)b->n_live, 6, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h.clock, b->d_clock, sizeof(BatchClock), cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    std::vector<int32_t> np32(b->np_host.begin(), b->np_host.end());
    std::memcpy(out + L.order, b->order.data(), sizeof(int32_t) * n);
    std::memcpy(out + L.np, np32.data(), sizeof(int32_t) * n);
    std::memcpy(h.magic, kBCkptMagic, sizeof(kBCkptMagic));
    h.version = kBCkptVersion;
    h.header_bytes = (int32_t)sizeof(BCkptHeader);
    h.n_sys = n;
    h.chunk_steps = b->C;
    h.threads = b->threads;
    h.tpp = b->tpp;
    h.enc_mode = b->o.enc_mode;
    h.enc_value = b->o.enc_value;
    h.r_max = b->o.r_max;
    h.n_total = b->n_total;
    h.n_live = b->n_live;
    h.step = b->step;
    h.total_bytes = (int64_t)L.total;
    std::memcpy(out, &h, sizeof(h));
    return GLISSE_OK;
}

static int batch_restore(glisse_batch* b, const BCkptHeader& h, const char* in, const BCkptLayout& L) {
    const int n = b->n_sys;
    const int src = batch_streams(b);
    if (src) return src;
    b->order.resize(n);
    std::memcpy(b->order.data(), in + L.order, sizeof(int32_t) * n);
    std::vector<int32_t> np32(n);
    std::memcpy(np32.data(), in + L.np, sizeof(int32_t) * n);
    b->np_host.assign(np32.begin(), np32.end());
    std::vector<int64_t> log_off;
    const int arc = batch_alloc(b, log_off);
    if (arc) return arc;
    auto h2d = [&](void* dst, size_t off, size_t nbytes) {
        return nbytes ? cudaMemcpyAsync(dst, in + off, nbytes, cudaMemcpyHostToDevice, b->s) : cudaSuccess;
    };
    GB_CUDA(h2d(b->d_pcs, L.pcs, sizeof(PlanetConsts) * n));
    GB_CUDA(h2d(b->d_ppcs, L.ppcs, sizeof(ParticleConsts) * n));
    GB_CUDA(h2d(b->d_np, L.np, sizeof(int32_t) * n));
    GB_CUDA(h2d(b->d_dt, L.dt, sizeof(double) * n));
    GB_CUDA(h2d(b->d_jac, L.jac, sizeof(double) * 6 * kMaxPlanets * n));
    GB_CUDA(cudaMemcpyAsync(b->d_log_off, log_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, b->s));
    GB_CUDA(h2d(b->d_cnt, L.cnt, sizeof(int64_t) * n));
    if (h.n_live > 0) {
        GB_CUDA(cudaMemcpy2DAsync(b->d_st[0], sizeof(double) * b->cap, in + L.st, sizeof(double) * (size_t)h.n_live,
                                  sizeof(double) * (size_t)h.n_live, 6, cudaMemcpyHostToDevice, b->s));
        GB_CUDA(h2d(b->d_id[0], L.id, sizeof(int32_t) * (size_t)h.n_live));
        GB_CUDA(h2d(b->d_alive, L.alive, (size_t)h.n_live));
    }
    GB_CUDA(h2d(b->d_out_state, L.out_state, sizeof(double) * 6 * (size_t)b->n_total));
    GB_CUDA(h2d(b->d_out_step, L.out_step, sizeof(int64_t) * (size_t)b->n_total));
    GB_CUDA(h2d(b->d_out_reason, L.out_reason, sizeof(int32_t) * (size_t)b->n_total));
    GB_CUDA(cudaMemcpyAsync(b->d_clock, &h.clock, sizeof(BatchClock), cudaMemcpyHostToDevice, b->s));
    batch_tasks_kernel<<<1, 1024, 0, b->s>>>(n, b->d_cnt, b->d_task_sys, b->d_task_start, b->d_task_count,
                                              b->d_n_tasks, b->d_nlive, nullptr, b->d_counter, b->d_clock, 0);
    GB_CUDA(cudaGetLastError());
    b->cur = 0;
    b->step = h.step;
    int rc = set_launch_shape(b, h.threads, h.tpp);
    if (rc) return rc;
    return refresh_host_counts(b);
}

extern "C" int glisse_batch_resume(glisse_batch** out, const void* buf, int64_t bytes, const glisse_opts* opts) {
    glisse::NvtxRange range("glisse_batch_resume");
    if (!out) return GLISSE_E_INVAL;
    *out = nullptr;
    if (!buf || bytes < (int64_t)sizeof(BCkptHeader)) return GLISSE_E_INVAL;
    BCkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kBCkptMagic, sizeof(kBCkptMagic)) != 0 || h.version != kBCkptVersion ||
        h.header_bytes != (int32_t)sizeof(BCkptHeader))
        return GLISSE_E_INVAL;
    if (h.n_sys < 1 || h.chunk_steps < 1 || h.chunk_steps > (1 << 20)) return GLISSE_E_INVAL;
    if (h.threads < 32 || h.threads > 256 || h.threads % 32 || (h.tpp != 1 && h.tpp != 2)) return GLISSE_E_INVAL;
    if (h.enc_mode != GLISSE_ENC_HILL && h.enc_mode != GLISSE_ENC_FIXED) return GLISSE_E_INVAL;
    if (!(h.enc_value >= 0.0) || !std::isfinite(h.enc_value) || !std::isfinite(h.r_max)) return GLISSE_E_INVAL;
    if (h.n_total < 0 || h.n_total > INT32_MAX || h.n_live < 0 || h.n_live > h.n_total || h.step < 0 ||
        h.clock.step != h.step || (h.clock.test_first != 0 && h.clock.test_first != 1))
        return GLISSE_E_INVAL;
    const BCkptLayout L = bckpt_layout(h.n_sys, h.n_total, h.n_live);
    if (h.total_bytes != (int64_t)L.total || bytes < h.total_bytes) return GLISSE_E_INVAL;
    const char* in = static_cast<const char*>(buf);
    const int n = h.n_sys;
    // the system order is a permutation, planet counts in range and matching the constants,
    // live counts summing to the slots, every slot id a distinct particle (the kernels write
    // per-id results through them)
    {
        std::vector<int32_t> order(n), np(n);
        std::memcpy(order.data(), in + L.order, sizeof(int32_t) * n);
        std::memcpy(np.data(), in + L.np, sizeof(int32_t) * n);
        std::vector<bool> seen_sys(n, false);
        int64_t sum = 0;
        for (int k = 0; k < n; ++k) {
            if (order[k] < 0 || order[k] >= n || seen_sys[order[k]]) return GLISSE_E_INVAL;
            seen_sys[order[k]] = true;
            if (np[k] < 0 || np[k] > GLISSE_MAX_PLANETS) return GLISSE_E_INVAL;
            PlanetConsts pc;
            std::memcpy(&pc, in + L.pcs + sizeof(PlanetConsts) * (size_t)k, sizeof(pc));
            if (pc.np != np[k]) return GLISSE_E_INVAL;
            int64_t c = 0;
            std::memcpy(&c, in + L.cnt + sizeof(int64_t) * (size_t)k, sizeof(c));
            if (c < 0) return GLISSE_E_INVAL;
            sum += c;
        }
        if (sum != h.n_live) return GLISSE_E_INVAL;
        std::vector<bool> seen((size_t)h.n_total, false);
        for (int64_t k = 0; k < h.n_live; ++k) {
            int32_t id = 0;
            std::memcpy(&id, in + L.id + sizeof(int32_t) * (size_t)k, sizeof(id));
            if (id < 0 || (int64_t)id >= h.n_total || seen[(size_t)id]) return GLISSE_E_INVAL;
            seen[(size_t)id] = true;
        }
    }
    glisse_opts o;
    glisse_opts_default(&o);
    o.chunk_steps = h.chunk_steps;
    o.enc_mode = h.enc_mode;
    o.enc_value = h.enc_value;
    o.r_max = h.r_max;
    if (opts) {
        o.cuda_stream = opts->cuda_stream;
        o.timing = opts->timing;
    }
    glisse_batch* b = new (std::nothrow) glisse_batch();
    if (!b) return GLISSE_E_NOMEM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return GLISSE_E_CUDA;
    }
    b->o = o;
    b->n_sys = n;
    b->C = h.chunk_steps;
    b->n_total = h.n_total;
    b->timing = o.timing != 0;
    const int rc = batch_restore(b, h, in, L);
    if (rc != GLISSE_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return GLISSE_OK;
}
