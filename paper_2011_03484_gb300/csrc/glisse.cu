// glisse.cu -- host runtime behind the C ABI of include/glisse.h.
//
// Layout in device memory (one context):
//   particles   two sets of [6][cap] double planes (x, y, z, vx, vy, vz) plus
//               [cap] int32 ids; the live particles occupy slots 0..n_live-1 of
//               the current set, in id order (stable compaction keeps it)
//   alive       [cap] uint8 written by the particle kernel, reset after compaction
//   per-id out  [N][6] state, [N] removal step, [N] reason
//   planets     constants, Jacobi state [2][N_p][3]
//   planet log  a ring of 3 chunk buffers, each [(C+1)][4 (N_p+1)] doubles of
//               positions + h0, and [(C+1)][N_p][6] synchronised heliocentric
//               states (for glisse_read_planets)
//
// Scheduling: chunk j of the planet log covers steps [jC, (j+1)C] of the
// run.  The ephemeris kernel for chunk j+1 runs on a high-priority side stream
// while the particle kernel works through chunk j on the main stream (section
// 2.2 computes the planets one chunk ahead in the same way); events order the
// ring-buffer reuse.  Within a long glisse_advance call the ring grows and the
// planets run further ahead, up to the call's last chunk (grow_ring, kEphQueue).  The first chunk has nothing to overlap with: its planet
// kernel starts in glisse_create, publishes its progress to host-mapped memory,
// and the particles of that chunk run in segments launched as their planet steps
// appear.  Every segment (a particle launch over at most one chunk) ends open:
// the slots keep the velocities with the next opening half kick applied and the
// kernel publishes the synchronised states by id, so cuts -- call ends, the
// first chunk's pieces, sample steps -- leave no trace in the results.  Live
// particles are compacted at chunk boundaries, every resync_chunks chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "glisse_internal.h"
#include "nvtx_range.h"

namespace glisse {
cudaError_t launch_eph_setup(const double*, int, double, double, int, double, PlanetConsts*, double*, int*,
                             cudaStream_t);
cudaError_t launch_eph_chunk(const PlanetConsts*, double*, double, int, double*, double*, int*, cudaStream_t,
                             int* progress = nullptr);
cudaError_t launch_eph_external(const PlanetConsts*, const double*, int64_t, double*, cudaStream_t);
cudaError_t launch_particle_chunk(int, const ChunkArgs&, const ParticleConsts&, cudaStream_t, const TaskArgs*, bool);
cudaError_t launch_particle_chunk_paper(int, const ChunkArgs&, const ParticleConsts&, cudaStream_t);
cudaError_t launch_compact(int64_t, const uint8_t*, const double*, const int32_t*, int64_t, double*, int32_t*,
                           int64_t, int64_t*, int64_t*, cudaStream_t);
cudaError_t launch_compact_sorted(int64_t, const uint8_t*, const double*, const int32_t*, int64_t, double*, int32_t*,
                                  int64_t, int64_t*, uint8_t*, double, double, int64_t*, cudaStream_t);
int64_t compact_scratch_entries(int64_t);
cudaError_t launch_export_live(int64_t, const double*, int64_t, const int32_t*, double*, cudaStream_t);
cudaError_t launch_import(int64_t, const double*, double*, int64_t, int32_t*, cudaStream_t);
}  // namespace glisse

#include <chrono>
#include <thread>
#include <vector>

using namespace glisse;

namespace {
// Planet-log ring: 3 slots (the chunk the particles run, the next one, one
// spare), more for a long glisse_advance call, so that the planets can run ahead
// of the particles up to the call's last step (see grow_ring), within this budget.
constexpr size_t kRingMin = 3;
constexpr size_t kRingBudgetBytes = size_t(512) << 20;
// Planet kernels enqueued beyond the last one known complete: enough that the
// side stream never runs dry between two particle chunks (it completes ~3
// chunks of planets per chunk of 131072 particles), few enough that the launch
// queue never fills (a full queue blocks the host in the launch call).
constexpr int64_t kEphQueue = 8;
// The first chunk of planets has no particle work to overlap with.  Its kernel
// publishes its step count to host-mapped memory, and the particles of that chunk
// run in segments ending at steps kFirstPiece * g^k, each launched once the host
// sees its planet steps written: the particles follow the planets from the first
// piece on, while the planet kernel keeps its SM.  A piece g times as long as the
// steps before it never waits for its planets when a particle step takes at least
// g planet steps: g = 4 when the particles fill kFourfoldWarps warps per SM
// partition or more (a planet step is ~1.2 warp-steps of particles on a partition:
// ~146 against ~109 FP64 instructions, at a busier pipe), else g = 2.  Fewer
// pieces mean fewer launch tails (measured on 131072 particles: the first chunk
// 26.41 ms with g = 4 against 26.75 ms with g = 2).
constexpr int kMaxPieces = 8;
constexpr int64_t kFirstPiece = kProgressEvery;
constexpr int64_t kFourfoldWarps = 5;
// A count that has not arrived after this long means the GPU is busy with other
// work (the planet kernel has not started): the rest of the chunk then waits for
// the planet kernel's completion event instead.  The longest piece the host polls
// for is 1024 planet steps, ~10-20 ms of planet kernel.
constexpr double kProgressPollSeconds = 0.5;
constexpr int kPollGaveUp = 1;
constexpr double kG = 4.0 * 3.14159265358979323846 * 3.14159265358979323846;
}  // namespace

// One chunk of planets on the device: log [(C+1)][4 (N_p+1)] (positions + h0)
// and history [(C+2)][N_p][6]: rows 0..C the synchronised heliocentric states,
// row C+1 the planets' Jacobi state at the chunk's first step (what the planet
// kernel started from; a checkpoint saves it so that resume recomputes the
// chunk bit for bit).
struct Slot {
    double* log = nullptr;
    double* hist = nullptr;
    int64_t chunk = -1;           // chunk held (-1: none)
    cudaEvent_t ev_eph = nullptr;  // planet kernel done (side stream)
    cudaEvent_t ev_use = nullptr;  // particles done with it (main stream)
    cudaEvent_t te0 = nullptr, te1 = nullptr;  // timing mode
    bool used = false, pending = false;
    bool in_arena = false;  // buffers carved from the context's arena (not freed one by one)
};

struct glisse_ctx {
    int device = 0;
    cudaStream_t s = nullptr, se = nullptr;
    bool own_s = false;
    glisse_opts o{};
    int np = 0;
    double m0 = 0, dt = 0;
    int C = 1024;
    int64_t n_total = 0, cap = 0, n_live = 0, step = 0;
    bool tested_first = false;
    PlanetConsts hpc{};
    ParticleConsts ppc{};
    PlanetConsts* d_pc = nullptr;
    double* d_jac = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;
    std::vector<Slot> ring;  // planet-log slots; chunk j lives in ring[j % ring.size()]
    cudaEvent_t ev_order = nullptr;
    int64_t next_chunk = 0;
    int64_t eph_done = 0;  // chunks whose planet kernel is known complete (host view)
    int64_t piece_end[kMaxPieces] = {};     // first chunk: step each particle segment may end at
    int n_pieces = 0;
    void* d_arena = nullptr;                // the fixed-size device buffers, in one allocation
    void* h_block = nullptr;                // the pinned host words below, in one mapped allocation
    int* h_prog = nullptr;                  // host-mapped: planet steps of the first chunk written
    int* d_prog = nullptr;
    double* d_st[2] = {};
    int32_t* d_id[2] = {};
    int cur = 0;
    uint8_t* d_alive = nullptr;
    uint8_t* d_key = nullptr;  // sort keys (sort_mode != NONE)
    double* d_out_state = nullptr;
    int64_t* d_out_step = nullptr;
    int32_t* d_out_reason = nullptr;
    int64_t* d_counts = nullptr;
    int64_t* d_nlive = nullptr;
    int64_t* h_nlive = nullptr;
    unsigned long long* d_steps = nullptr;   // exact particle-step counter (timing mode)
    unsigned long long* h_steps = nullptr;
    unsigned long long* d_task = nullptr;    // task counter of the particle kernel's task mode
    int32_t* d_group_done = nullptr;         // [ceil(cap / 32)] sub-chunks finished per 32-slot group
    unsigned long long* d_live = nullptr;    // particles live at the end of the last segment
    unsigned long long* h_live = nullptr;
    int64_t n_alive = 0;                     // live particles (n_live counts slots, dead ones included
                                             // until the next compaction)
    int since_compact = 0;
    bool external = false, planets_valid = true;
    double* d_ext_log = nullptr;
    int64_t ext_n = 0, ext_off = 0;
    // optional per-launch timing
    bool timing = false;
    cudaEvent_t tp0 = nullptr, tp1 = nullptr, tc0 = nullptr, tc1 = nullptr;

    glisse_timing acc{};
    // element sampling / libration test (glisse_set_sampling)
    bool samp_on = false;
    glisse_sampling samp{};
    double* d_elem = nullptr;               // [max_samples][n_total][6] by id
    std::vector<int64_t> samp_steps;        // global step of each kept sample
    int64_t samp_seen = 0;                  // samples taken (kept or not)
    uint8_t* d_near0 = nullptr;
    uint8_t* d_near180 = nullptr;
    int32_t* d_count = nullptr;
};

#define GL_CUDA(x)                               \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) {                 \
            (void)cudaGetLastError();            \
            return GLISSE_E_CUDA;                \
        }                                        \
    } while (0)

static int alloc_dev(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return GLISSE_E_NOMEM;
    }
    return e == cudaSuccess ? GLISSE_OK : GLISSE_E_CUDA;
}

#define GL_ALLOC(ptr, bytes)                                      \
    do {                                                          \
        int r_ = alloc_dev(reinterpret_cast<void**>(&(ptr)), (bytes)); \
        if (r_ != GLISSE_OK) return r_;                           \
    } while (0)

extern "C" void glisse_opts_default(glisse_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->chunk_steps = 1024;
    o->resync_chunks = 1;
    o->kepler_mode = GLISSE_KEPLER_CONVERGE;
    o->kepler_iters = 5;
    o->enc_mode = GLISSE_ENC_HILL;
    o->timing = 0;
    o->sort_mode = GLISSE_SORT_NONE;
    o->enc_value = 1.0;
    o->r_max = 1000.0;
    o->cuda_stream = nullptr;
}

extern "C" const char* glisse_strerror(int code) {
    switch (code) {
        case GLISSE_OK: return "ok";
        case GLISSE_E_INVAL: return "invalid argument";
        case GLISSE_E_NOMEM: return "out of memory";
        case GLISSE_E_CUDA: return "CUDA error";
        case GLISSE_E_KEPLER: return "Kepler solve did not converge";
        case GLISSE_E_TIMEOUT: return "wait for device work timed out";
        case GLISSE_E_STATE: return "invalid in the current state";
        default: return "unknown status";
    }
}

static void free_slot(Slot& sl) {
    if (!sl.in_arena) {
        cudaFree(sl.log);
        cudaFree(sl.hist);
    }
    for (cudaEvent_t e : {sl.ev_eph, sl.ev_use, sl.te0, sl.te1})
        if (e) cudaEventDestroy(e);
    sl = Slot{};
}

static size_t hist_doubles(const glisse_ctx* c) { return (size_t)(c->C + 2) * 6 * std::max(c->np, 1); }

static size_t slot_bytes(const glisse_ctx* c) {
    return sizeof(double) * ((size_t)(c->C + 1) * (size_t)log_stride(c->np) + hist_doubles(c));
}

// Buffers (unless the slot already has arena buffers) and events of an empty
// slot; false (nothing of its own left allocated) on failure.
static bool alloc_slot(const glisse_ctx* c, Slot& sl) {
    const int S = log_stride(c->np);
    bool ok = sl.in_arena ||
              (cudaMalloc(&sl.log, sizeof(double) * (size_t)(c->C + 1) * S) == cudaSuccess &&
               cudaMalloc(&sl.hist, sizeof(double) * hist_doubles(c)) == cudaSuccess);
    ok = ok && cudaEventCreateWithFlags(&sl.ev_eph, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&sl.ev_use, cudaEventDisableTiming) == cudaSuccess;
    if (ok && c->timing) ok = cudaEventCreate(&sl.te0) == cudaSuccess && cudaEventCreate(&sl.te1) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_slot(sl);
    }
    return ok;
}

static void ctx_free(glisse_ctx* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    if (c->se) cudaStreamSynchronize(c->se);
    for (Slot& sl : c->ring) free_slot(sl);
    for (cudaEvent_t e : {c->tp0, c->tp1, c->tc0, c->tc1, c->ev_order})
        if (e) cudaEventDestroy(e);
    if (c->h_block) cudaFreeHost(c->h_block);
    cudaFree(c->d_arena);
    cudaFree(c->d_elem);
    cudaFree(c->d_near0);
    cudaFree(c->d_near180);
    cudaFree(c->d_count);
    cudaFree(c->d_ext_log);
    if (c->se) cudaStreamDestroy(c->se);
    if (c->own_s && c->s) cudaStreamDestroy(c->s);
    delete c;
}

extern "C" void glisse_destroy(glisse_ctx* c) {
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    ctx_free(c);
    cudaSetDevice(prev);
}

// Enqueue the ephemeris for chunk j (and every earlier chunk not yet enqueued).
static int ensure_chunk(glisse_ctx* c, int64_t j) {
    NvtxRange range("glisse: enqueue planet chunks");
    while (c->next_chunk <= j) {
        Slot& sl = c->ring[(size_t)(c->next_chunk % (int64_t)c->ring.size())];
        if (sl.used) GL_CUDA(cudaStreamWaitEvent(c->se, sl.ev_use, 0));
        if (c->timing) GL_CUDA(cudaEventRecord(sl.te0, c->se));
        int* prog = nullptr;
        if (c->next_chunk == 0) {
            int dev = 0, nsm = 0;
            GL_CUDA(cudaGetDevice(&dev));
            GL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            const int64_t partitions = 4 * (int64_t)std::max(nsm - 1, 1);  // the ephemeris holds one SM
            const int shift = c->n_live >= kFourfoldWarps * 32 * partitions ? 2 : 1;
            c->n_pieces = 0;
            for (int64_t b = 0; b < c->C; b = c->piece_end[c->n_pieces++])
                c->piece_end[c->n_pieces] = c->n_pieces == kMaxPieces - 1
                                                ? c->C
                                                : std::min<int64_t>(c->C, kFirstPiece << (shift * c->n_pieces));
            prog = c->d_prog;
        }
        if (c->np > 0)
            GL_CUDA(cudaMemcpyAsync(sl.hist + (size_t)(c->C + 1) * 6 * c->np, c->d_jac, sizeof(double) * 6 * c->np,
                                    cudaMemcpyDeviceToDevice, c->se));
        GL_CUDA(launch_eph_chunk(c->d_pc, c->d_jac, c->dt, c->C, sl.log, sl.hist, c->d_status, c->se, prog));
        if (c->timing) {
            GL_CUDA(cudaEventRecord(sl.te1, c->se));
            sl.pending = true;
        }
        GL_CUDA(cudaEventRecord(sl.ev_eph, c->se));
        sl.chunk = c->next_chunk;
        sl.used = false;
        ++c->next_chunk;
    }
    return GLISSE_OK;
}

// Give the ring at least `want` slots (capped by kRingBudgetBytes), so that a long
// glisse_advance call can enqueue the planets of all its chunks at once: the
// planet kernel then runs ahead while the particles are the slower stage and
// has the log ready when they become the faster one (few live particles).
// Between calls nothing of the main stream is in flight; the side stream is
// drained, and slots holding chunks move (pointers and events) to the position
// of their chunk in the larger ring.  An allocation failure keeps the ring as
// it is (the lookahead is an optimisation).
static int grow_ring(glisse_ctx* c, size_t want) {
    const size_t cap = std::max(kRingMin, kRingBudgetBytes / std::max<size_t>(slot_bytes(c), 1));
    want = std::min(want, cap);
    const size_t R = c->ring.size();
    if (want <= R) return GLISSE_OK;
    std::vector<Slot> fresh(want - R);
    for (size_t k = 0; k < fresh.size(); ++k) {
        if (!alloc_slot(c, fresh[k])) {
            for (Slot& f : fresh) free_slot(f);
            return GLISSE_OK;
        }
    }
    GL_CUDA(cudaStreamSynchronize(c->se));
    std::vector<Slot> next(want);
    std::vector<Slot> spare;
    for (Slot& old : c->ring) {
        if (old.chunk >= 0 && next[(size_t)(old.chunk % (int64_t)want)].log == nullptr)
            next[(size_t)(old.chunk % (int64_t)want)] = old;
        else
            spare.push_back(old);
    }
    for (Slot& f : fresh) spare.push_back(f);
    for (Slot& n : next) {
        if (n.log) continue;
        n = spare.back();
        spare.pop_back();
        n.chunk = -1;
    }
    c->ring.swap(next);
    return GLISSE_OK;
}

// Wait until the first chunk's planet kernel has written `steps` steps (host-mapped
// count).  GLISSE_OK; GLISSE_E_CUDA if the side stream errs or stops short of the
// count; kPollGaveUp after kProgressPollSeconds without it.
static int wait_progress(glisse_ctx* c, int64_t steps) {
    const volatile int* p = c->h_prog;
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned it = 0;; ++it) {
        if (*p >= steps) return GLISSE_OK;
        if ((it & 255u) == 255u) {
            const cudaError_t q = cudaStreamQuery(c->se);
            if (q == cudaSuccess) return *p >= steps ? GLISSE_OK : GLISSE_E_CUDA;
            if (q != cudaErrorNotReady) return GLISSE_E_CUDA;
            const std::chrono::duration<double> el = std::chrono::steady_clock::now() - t0;
            if (el.count() > kProgressPollSeconds) return kPollGaveUp;
        }
        std::this_thread::yield();
    }
}

static int check_status(glisse_ctx* c) {
    GL_CUDA(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    GL_CUDA(cudaStreamSynchronize(c->s));
    return *c->h_status;
}

// A context's state as a checkpoint holds it (host pointers into the caller's
// buffer), installed by setup() in place of the initial conditions.
struct Restore {
    PlanetConsts pc;
    const double* jac0;         // [np][6] Jacobi state at the first step of chunk step / C
    const double* st;           // [6][n_live] particle slots as laid out on the device
    const int32_t* id;          // [n_live]
    const uint8_t* alive;       // [n_live]
    const double* out_state;    // [n_total][6] by id
    const int64_t* out_step;    // [n_total]
    const int32_t* out_reason;  // [n_total]
    int64_t n_live = 0, step = 0, since_compact = 0;
    bool tested_first = false;
};

static int setup(glisse_ctx* c, const double* planets, const double* particles, const Restore* r = nullptr) {
    const int np = c->np;
    GL_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
    c->own_s = true;
    if (c->o.cuda_stream) {
        cudaStreamDestroy(c->s);
        c->s = static_cast<cudaStream_t>(c->o.cuda_stream);
        c->own_s = false;
    }
    int lo = 0, hi = 0;
    GL_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    GL_CUDA(cudaStreamCreateWithPriority(&c->se, cudaStreamNonBlocking, hi));
    // pinned host words: progress count (mapped), status, live count, step counter
    GL_CUDA(cudaHostAlloc(&c->h_block, 64, cudaHostAllocMapped));
    std::memset(c->h_block, 0, 64);
    char* hb = static_cast<char*>(c->h_block);
    c->h_prog = reinterpret_cast<int*>(hb);
    c->h_status = reinterpret_cast<int*>(hb + 8);
    c->h_nlive = reinterpret_cast<int64_t*>(hb + 16);
    c->h_steps = reinterpret_cast<unsigned long long*>(hb + 24);
    c->h_live = reinterpret_cast<unsigned long long*>(hb + 32);
    GL_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_prog), c->h_prog, 0));
    if (c->timing) {
        GL_CUDA(cudaEventCreate(&c->tp0));
        GL_CUDA(cudaEventCreate(&c->tp1));
        GL_CUDA(cudaEventCreate(&c->tc0));
        GL_CUDA(cudaEventCreate(&c->tc1));
    }
    const int S = log_stride(np);
    const int64_t cap = std::max<int64_t>(c->n_total, 1);
    c->cap = cap;
    // the fixed-size device buffers in one allocation, each at a 256-byte boundary
    // (one cudaMalloc and one cudaFree per context instead of ~20 of each)
    c->ring.resize(kRingMin);
    double* d_in = nullptr;  // planets [np][7] for the set-up kernel
    {
        size_t off = 0;
        auto take = [&off](size_t bytes) {
            const size_t o = off;
            off += (std::max<size_t>(bytes, 16) + 255) & ~size_t(255);
            return o;
        };
        const size_t o_pc = take(sizeof(PlanetConsts)), o_jac = take(sizeof(double) * 6 * std::max(np, 1)),
                     o_status = take(sizeof(int)), o_in = take(sizeof(double) * 7 * std::max(np, 1));
        size_t o_log[kRingMin], o_hist[kRingMin];
        for (size_t r = 0; r < kRingMin; ++r) {
            o_log[r] = take(sizeof(double) * (size_t)(c->C + 1) * S);
            o_hist[r] = take(sizeof(double) * hist_doubles(c));
        }
        size_t o_st[2], o_id[2];
        for (int b = 0; b < 2; ++b) {
            o_st[b] = take(sizeof(double) * 6 * (size_t)cap);
            o_id[b] = take(sizeof(int32_t) * (size_t)cap);
        }
        const size_t o_alive = take((size_t)cap), o_key = c->o.sort_mode == GLISSE_SORT_COST ? take((size_t)cap) : 0,
                     o_out_state = take(sizeof(double) * 6 * (size_t)cap), o_out_step = take(sizeof(int64_t) * (size_t)cap),
                     o_out_reason = take(sizeof(int32_t) * (size_t)cap),
                     o_counts = take(sizeof(int64_t) * (size_t)compact_scratch_entries(cap)),
                     o_nlive = take(sizeof(int64_t)), o_steps = take(sizeof(unsigned long long)),
                     o_live = take(sizeof(unsigned long long)), o_task = take(sizeof(unsigned long long)),
                     o_groups = take(sizeof(int32_t) * (size_t)((cap + 31) / 32));
        GL_ALLOC(c->d_arena, off);
        char* base = static_cast<char*>(c->d_arena);
        c->d_pc = reinterpret_cast<PlanetConsts*>(base + o_pc);
        c->d_jac = reinterpret_cast<double*>(base + o_jac);
        c->d_status = reinterpret_cast<int*>(base + o_status);
        d_in = reinterpret_cast<double*>(base + o_in);
        for (size_t r = 0; r < kRingMin; ++r) {
            c->ring[r].log = reinterpret_cast<double*>(base + o_log[r]);
            c->ring[r].hist = reinterpret_cast<double*>(base + o_hist[r]);
            c->ring[r].in_arena = true;
        }
        for (int b = 0; b < 2; ++b) {
            c->d_st[b] = reinterpret_cast<double*>(base + o_st[b]);
            c->d_id[b] = reinterpret_cast<int32_t*>(base + o_id[b]);
        }
        c->d_alive = reinterpret_cast<uint8_t*>(base + o_alive);
        if (c->o.sort_mode == GLISSE_SORT_COST) c->d_key = reinterpret_cast<uint8_t*>(base + o_key);
        c->d_out_state = reinterpret_cast<double*>(base + o_out_state);
        c->d_out_step = reinterpret_cast<int64_t*>(base + o_out_step);
        c->d_out_reason = reinterpret_cast<int32_t*>(base + o_out_reason);
        c->d_counts = reinterpret_cast<int64_t*>(base + o_counts);
        c->d_nlive = reinterpret_cast<int64_t*>(base + o_nlive);
        // the exact particle-step counter exists in timing mode only (the kernel skips a null one)
        c->d_steps = c->timing ? reinterpret_cast<unsigned long long*>(base + o_steps) : nullptr;
        c->d_live = reinterpret_cast<unsigned long long*>(base + o_live);
        c->d_task = reinterpret_cast<unsigned long long*>(base + o_task);
        c->d_group_done = reinterpret_cast<int32_t*>(base + o_groups);
    }
    for (Slot& sl : c->ring)
        if (!alloc_slot(c, sl)) return GLISSE_E_NOMEM;
    if (c->timing) GL_CUDA(cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned long long), c->s));

    cudaError_t e = cudaSuccess;
    if (r) {
        // restore: the saved constants and the Jacobi state the current chunk starts from
        c->hpc = r->pc;
        e = cudaMemcpyAsync(c->d_pc, &c->hpc, sizeof(PlanetConsts), cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess && np > 0)
            e = cudaMemcpyAsync(c->d_jac, r->jac0, sizeof(double) * 6 * np, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e != cudaSuccess) return GLISSE_E_CUDA;
    } else {
        // planets -> device, set-up kernel (Jacobi state, constants, encounter radii)
        if (np > 0) e = cudaMemcpyAsync(d_in, planets, sizeof(double) * 7 * np, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess)
            e = launch_eph_setup(d_in, np, c->m0, kG, c->o.enc_mode, c->o.enc_value, c->d_pc, c->d_jac, c->d_status,
                                 c->s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&c->hpc, c->d_pc, sizeof(PlanetConsts), cudaMemcpyDeviceToHost, c->s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e != cudaSuccess) return GLISSE_E_CUDA;
        if (*c->h_status != 0) return *c->h_status;
    }

    // particle constants (kernel parameters)
    ParticleConsts& p = c->ppc;
    std::memset(&p, 0, sizeof(p));
    p.mu = c->hpc.mu0;
    p.dt = c->dt;
    p.half_dt = 0.5 * c->dt;
    for (int j = 0; j < np; ++j) {
        p.tgm_full[j] = c->dt * c->hpc.gm[j];
        p.tgm_half[j] = 0.5 * c->dt * c->hpc.gm[j];
        p.rc2[j] = c->hpc.rcrit[j] * c->hpc.rcrit[j];
    }
    p.rmax2 = c->o.r_max > 0.0 ? c->o.r_max * c->o.r_max : 0.0;
    p.kepler_iters = c->o.kepler_mode == GLISSE_KEPLER_PAPER_FIXED ? c->o.kepler_iters : 0;
    p.kepler_tol = GLISSE_PAPER_KEPLER_TOL;
    p.rmax = c->o.r_max > 0.0 ? c->o.r_max : 0.0;

    // the first chunk of planets now, on the side stream: it overlaps the
    // particle upload below and whatever the caller does before advancing.  A
    // resumed context starts at the chunk holding its step, from that chunk's
    // saved Jacobi state.
    const int64_t j0 = r ? r->step / c->C : 0;
    c->next_chunk = j0;
    c->eph_done = j0;
    // the live count sizes the first chunk's particle segments (ensure_chunk)
    c->n_live = r ? r->n_live : c->n_total;
    if (c->n_total > 0) {
        const int er = ensure_chunk(c, j0);
        if (er != GLISSE_OK) return er;
    }

    if (r) {
        // particle slots exactly as the checkpointed context held them, per-id results
        if (r->n_live > 0) {
            GL_CUDA(cudaMemcpy2DAsync(c->d_st[0], sizeof(double) * (size_t)cap, r->st,
                                      sizeof(double) * (size_t)r->n_live, sizeof(double) * (size_t)r->n_live, 6,
                                      cudaMemcpyHostToDevice, c->s));
            GL_CUDA(cudaMemcpyAsync(c->d_id[0], r->id, sizeof(int32_t) * (size_t)r->n_live, cudaMemcpyHostToDevice,
                                    c->s));
            GL_CUDA(cudaMemcpyAsync(c->d_alive, r->alive, (size_t)r->n_live, cudaMemcpyHostToDevice, c->s));
        }
        if (c->n_total > 0) {
            GL_CUDA(cudaMemcpyAsync(c->d_out_state, r->out_state, sizeof(double) * 6 * (size_t)c->n_total,
                                    cudaMemcpyHostToDevice, c->s));
            GL_CUDA(cudaMemcpyAsync(c->d_out_step, r->out_step, sizeof(int64_t) * (size_t)c->n_total,
                                    cudaMemcpyHostToDevice, c->s));
            GL_CUDA(cudaMemcpyAsync(c->d_out_reason, r->out_reason, sizeof(int32_t) * (size_t)c->n_total,
                                    cudaMemcpyHostToDevice, c->s));
        }
        c->n_live = r->n_live;
        c->n_alive = 0;
        for (int64_t k = 0; k < r->n_live; ++k) c->n_alive += r->alive[k] != 0;
        c->step = r->step;
        c->since_compact = r->since_compact;
        c->tested_first = r->tested_first;
    } else {
        // particles -> device SoA, ids, flags.  The [N][6] per-id output buffer stages
        // the upload (it is cleared right after on the same stream): a temporary buffer
        // would have to be freed, and cudaFree waits for the planet kernel started above.
        if (c->n_total > 0) {
            GL_CUDA(cudaMemcpyAsync(c->d_out_state, particles, sizeof(double) * 6 * (size_t)c->n_total,
                                    cudaMemcpyHostToDevice, c->s));
            GL_CUDA(launch_import(c->n_total, c->d_out_state, c->d_st[0], cap, c->d_id[0], c->s));
        }
        GL_CUDA(cudaMemsetAsync(c->d_alive, 1, (size_t)cap, c->s));
        GL_CUDA(cudaMemsetAsync(c->d_out_state, 0, sizeof(double) * 6 * (size_t)cap, c->s));
        GL_CUDA(cudaMemsetAsync(c->d_out_step, 0xFF, sizeof(int64_t) * (size_t)cap, c->s));  // -1
        GL_CUDA(cudaMemsetAsync(c->d_out_reason, 0, sizeof(int32_t) * (size_t)cap, c->s));
        c->n_live = c->n_total;
        c->n_alive = c->n_total;
    }
    // the first two planet chunks
    GL_CUDA(cudaEventCreateWithFlags(&c->ev_order, cudaEventDisableTiming));
    GL_CUDA(cudaEventRecord(c->ev_order, c->s));  // order the side stream after the set-up
    GL_CUDA(cudaStreamWaitEvent(c->se, c->ev_order, 0));
    int rc = ensure_chunk(c, j0 + 1);
    if (rc) return rc;
    GL_CUDA(cudaStreamSynchronize(c->s));
    return GLISSE_OK;
}

extern "C" int glisse_create(glisse_ctx** out, double star_mass, const double* planets, int32_t n_planets,
                             const double* particles, int64_t n_particles, double dt, const glisse_opts* opts) {
    if (!out) return GLISSE_E_INVAL;
    *out = nullptr;
    glisse_opts o;
    glisse_opts_default(&o);
    if (opts) o = *opts;
    if (!(star_mass > 0.0) || !std::isfinite(star_mass)) return GLISSE_E_INVAL;
    if (n_planets < 0 || n_planets > GLISSE_MAX_PLANETS) return GLISSE_E_INVAL;
    if (n_planets > 0 && !planets) return GLISSE_E_INVAL;
    if (n_particles < 0 || n_particles > INT32_MAX) return GLISSE_E_INVAL;
    if (n_particles > 0 && !particles) return GLISSE_E_INVAL;
    if (!(dt != 0.0) || !std::isfinite(dt)) return GLISSE_E_INVAL;
    if (o.chunk_steps < 1 || o.chunk_steps > (1 << 20) || o.resync_chunks < 1) return GLISSE_E_INVAL;
    if (o.kepler_mode != GLISSE_KEPLER_CONVERGE && o.kepler_mode != GLISSE_KEPLER_PAPER_FIXED) return GLISSE_E_INVAL;
    if (o.kepler_mode == GLISSE_KEPLER_PAPER_FIXED && (o.kepler_iters < 1 || o.kepler_iters > GLISSE_MAX_KEPLER_ITERS))
        return GLISSE_E_INVAL;
    if (o.enc_mode != GLISSE_ENC_HILL && o.enc_mode != GLISSE_ENC_FIXED) return GLISSE_E_INVAL;
    if (o.sort_mode != GLISSE_SORT_NONE && o.sort_mode != GLISSE_SORT_COST) return GLISSE_E_INVAL;
    if (o.launch_mode < GLISSE_LAUNCH_AUTO || o.launch_mode > GLISSE_LAUNCH_TASKS) return GLISSE_E_INVAL;
    if (!(o.enc_value >= 0.0) || !std::isfinite(o.enc_value) || !std::isfinite(o.r_max)) return GLISSE_E_INVAL;
    for (int64_t k = 0; k < 7 * (int64_t)n_planets; ++k)
        if (!std::isfinite(planets[k])) return GLISSE_E_INVAL;
    for (int j = 0; j < n_planets; ++j)
        if (!(planets[7 * j] >= 0.0)) return GLISSE_E_INVAL;
    glisse_ctx* c = new (std::nothrow) glisse_ctx();
    if (!c) return GLISSE_E_NOMEM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return GLISSE_E_CUDA;
    }
    c->o = o;
    c->np = n_planets;
    c->m0 = star_mass;
    c->dt = dt;
    c->C = o.chunk_steps;
    c->n_total = n_particles;
    c->timing = o.timing != 0;
    NvtxRange range("glisse_create");
    int rc = setup(c, planets, particles);
    if (rc != GLISSE_OK) {
        ctx_free(c);
        return rc;
    }
    *out = c;
    return GLISSE_OK;
}

static int compact(glisse_ctx* c) {
    NvtxRange range("glisse: compaction");
    const int nxt = c->cur ^ 1;
    if (c->timing) GL_CUDA(cudaEventRecord(c->tc0, c->s));
    if (c->o.sort_mode == GLISSE_SORT_COST)
        GL_CUDA(launch_compact_sorted(c->n_live, c->d_alive, c->d_st[c->cur], c->d_id[c->cur], c->cap, c->d_st[nxt],
                                      c->d_id[nxt], c->cap, c->d_counts, c->d_key, c->ppc.mu, c->dt, c->d_nlive,
                                      c->s));
    else
        GL_CUDA(launch_compact(c->n_live, c->d_alive, c->d_st[c->cur], c->d_id[c->cur], c->cap, c->d_st[nxt],
                               c->d_id[nxt], c->cap, c->d_counts, c->d_nlive, c->s));
    if (c->timing) GL_CUDA(cudaEventRecord(c->tc1, c->s));
    GL_CUDA(cudaMemcpyAsync(c->h_nlive, c->d_nlive, sizeof(int64_t), cudaMemcpyDeviceToHost, c->s));
    GL_CUDA(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    GL_CUDA(cudaStreamSynchronize(c->s));
    if (c->timing) {
        float ms = 0.f;
        GL_CUDA(cudaEventElapsedTime(&ms, c->tc0, c->tc1));
        c->acc.compact_ms += ms;
        ++c->acc.compact_launches;
    }
    c->n_live = *c->h_nlive;
    c->n_alive = c->n_live;
    c->cur = nxt;
    if (c->n_live > 0) GL_CUDA(cudaMemsetAsync(c->d_alive, 1, (size_t)c->n_live, c->s));
    c->since_compact = 0;
    return *c->h_status;
}

// One element sample on the stream (after the particle segment, before compaction).
static int take_sample(glisse_ctx* c, const double* planets_at_step, int64_t step) {
    SampleArgs a;
    a.n = c->n_live;
    a.sync = c->d_out_state;
    a.id = c->d_id[c->cur];
    a.alive = c->d_alive;
    a.planets = planets_at_step;
    a.pc = c->d_pc;
    a.frame = c->samp.frame;
    a.res_planet = c->samp.res_planet;
    a.res_p = c->samp.res_p;
    a.res_q = c->samp.res_q;
    a.avoid = c->samp.avoid_deg * (3.14159265358979323846 / 180.0);
    a.elem = nullptr;
    if ((int64_t)c->samp_steps.size() < c->samp.max_samples) {
        a.elem = c->d_elem + (size_t)c->samp_steps.size() * 6 * c->n_total;
        // NaN rows (all-ones bit pattern) for ids not live at this sample
        GL_CUDA(cudaMemsetAsync(a.elem, 0xFF, sizeof(double) * 6 * c->n_total, c->s));
        c->samp_steps.push_back(step);
    }
    a.near0 = c->d_near0;
    a.near180 = c->d_near180;
    a.count = c->d_count;
    GL_CUDA(launch_sample(a, c->s));
    ++c->samp_seen;
    return GLISSE_OK;
}

// 48 n k bytes (k samples of n particles' six doubles), false if that overflows size_t
static bool elem_bytes(int64_t n, int64_t k, size_t* out) {
    size_t t = 0;
    if (n < 0 || k < 0 || __builtin_mul_overflow((size_t)n, sizeof(double) * 6, &t) ||
        __builtin_mul_overflow(t, (size_t)k, &t) || t > SIZE_MAX / 2)
        return false;
    *out = t;
    return true;
}

extern "C" int glisse_set_sampling(glisse_ctx* c, const glisse_sampling* sp) {
    if (!c) return GLISSE_E_INVAL;
    if (sp) {
        if (sp->every < 1 || (sp->frame != GLISSE_FRAME_HELIO && sp->frame != GLISSE_FRAME_BARY) ||
            sp->max_samples < 0 || sp->res_planet < -1 || sp->res_planet >= c->np)
            return GLISSE_E_INVAL;
        if (sp->res_planet >= 0 && (sp->res_p < 1 || sp->res_q < 0 || !(sp->avoid_deg > 0.0) ||
                                    !(sp->avoid_deg < 90.0)))
            return GLISSE_E_INVAL;
        if (c->external) return GLISSE_E_STATE;
        if (sp->max_samples > 0 && (uint64_t)sp->max_samples > (uint64_t)1 << 40) return GLISSE_E_NOMEM;
        size_t bytes = 0;  // the element log's size must be representable
        if (!elem_bytes(std::max<int64_t>(c->n_total, 1), sp->max_samples, &bytes)) return GLISSE_E_NOMEM;
    }
    GL_CUDA(cudaStreamSynchronize(c->s));
    cudaFree(c->d_elem);
    cudaFree(c->d_near0);
    cudaFree(c->d_near180);
    cudaFree(c->d_count);
    c->d_elem = nullptr;
    c->d_near0 = c->d_near180 = nullptr;
    c->d_count = nullptr;
    c->samp_steps.clear();
    c->samp_seen = 0;
    c->samp_on = false;
    if (!sp) return GLISSE_OK;
    c->samp = *sp;
    const size_t n = (size_t)std::max<int64_t>(c->n_total, 1);
    if (sp->max_samples > 0) GL_ALLOC(c->d_elem, sizeof(double) * 6 * n * (size_t)sp->max_samples);
    GL_ALLOC(c->d_near0, n);
    GL_ALLOC(c->d_near180, n);
    GL_ALLOC(c->d_count, sizeof(int32_t) * n);
    GL_CUDA(cudaMemsetAsync(c->d_near0, 0, n, c->s));
    GL_CUDA(cudaMemsetAsync(c->d_near180, 0, n, c->s));
    GL_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(int32_t) * n, c->s));
    GL_CUDA(cudaStreamSynchronize(c->s));
    c->samp_on = true;
    return GLISSE_OK;
}

extern "C" int glisse_read_elements(glisse_ctx* c, double* elements, int64_t* sample_steps, int64_t max_samples,
                                    int64_t* n_samples) {
    if (!c || max_samples < 0 || !n_samples) return GLISSE_E_INVAL;
    if (!c->samp_on) return GLISSE_E_STATE;
    const int64_t k = std::min<int64_t>(max_samples, (int64_t)c->samp_steps.size());
    if (k > 0 && !elements) return GLISSE_E_INVAL;
    GL_CUDA(cudaStreamSynchronize(c->s));
    if (k > 0)
        GL_CUDA(cudaMemcpy(elements, c->d_elem, sizeof(double) * 6 * (size_t)c->n_total * (size_t)k,
                           cudaMemcpyDeviceToHost));
    if (sample_steps)
        for (int64_t i = 0; i < k; ++i) sample_steps[i] = c->samp_steps[(size_t)i];
    *n_samples = k;
    return GLISSE_OK;
}

extern "C" int glisse_read_libration(glisse_ctx* c, uint8_t* near0, uint8_t* near180, int32_t* count) {
    if (!c) return GLISSE_E_INVAL;
    if (!c->samp_on || c->samp.res_planet < 0) return GLISSE_E_STATE;
    GL_CUDA(cudaStreamSynchronize(c->s));
    const size_t n = (size_t)c->n_total;
    if (n == 0) return GLISSE_OK;
    if (near0) GL_CUDA(cudaMemcpy(near0, c->d_near0, n, cudaMemcpyDeviceToHost));
    if (near180) GL_CUDA(cudaMemcpy(near180, c->d_near180, n, cudaMemcpyDeviceToHost));
    if (count) GL_CUDA(cudaMemcpy(count, c->d_count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    return GLISSE_OK;
}

extern "C" int glisse_advance(glisse_ctx* c, int64_t n_steps) {
    if (!c || n_steps < 0) return GLISSE_E_INVAL;
    NvtxRange range("glisse_advance");
    if (n_steps == 0) return GLISSE_OK;
    if (c->external && n_steps > c->ext_n - c->ext_off) return GLISSE_E_STATE;
    if (!c->external && !c->planets_valid) return GLISSE_E_STATE;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != c->device) GL_CUDA(cudaSetDevice(c->device));
    const int S = log_stride(c->np);
    int64_t remaining = n_steps;
    int rc = GLISSE_OK;
    if (c->o.sort_mode == GLISSE_SORT_COST && !c->tested_first && c->n_live > 0 && (rc = compact(c)) != GLISSE_OK)
        return rc;
    // the planets may run ahead of the particles up to the call's last chunk (+1)
    const int64_t j_last = c->external ? 0 : (c->step + n_steps - 1) / c->C;
    if (!c->external && (rc = grow_ring(c, (size_t)(j_last - c->step / c->C + kRingMin))) != GLISSE_OK) return rc;
    while (remaining > 0 && rc == GLISSE_OK) {
        const double* log = nullptr;
        int64_t m = 0;
        Slot* sl = nullptr;
        if (c->external) {
            m = std::min<int64_t>(remaining, c->C - c->step % c->C);
            log = c->d_ext_log + (size_t)c->ext_off * S;
        } else {
            const int64_t j = c->step / c->C;
            const int64_t off = c->step - j * c->C;
            while (c->eph_done < c->next_chunk &&
                   cudaEventQuery(c->ring[(size_t)(c->eph_done % (int64_t)c->ring.size())].ev_eph) == cudaSuccess)
                ++c->eph_done;
            const int64_t ahead = std::min({j + (int64_t)c->ring.size() - 1, j_last + 1, c->eph_done + kEphQueue});
            if ((rc = ensure_chunk(c, std::max<int64_t>(ahead, j + 1))) != GLISSE_OK) break;
            sl = &c->ring[(size_t)(j % (int64_t)c->ring.size())];
            if (sl->chunk != j) {
                rc = GLISSE_E_STATE;
                break;
            }
            m = std::min<int64_t>(remaining, c->C - off);
            int k = 0;
            while (j == 0 && c->piece_end[k] <= off && k < c->n_pieces - 1) ++k;
            int w = kPollGaveUp;
            if (j == 0 && k < c->n_pieces - 1) {
                // first chunk: wait (on the host) only for the planet steps of this piece
                w = wait_progress(c, c->piece_end[k]);
                if (w < 0) {
                    rc = w;
                    break;
                }
            }
            if (w == GLISSE_OK) {
                m = std::min<int64_t>(m, c->piece_end[k] - off);
            } else {
                if (j == 0) c->n_pieces = 1;  // no more cuts in this chunk
                GL_CUDA(cudaStreamWaitEvent(c->s, sl->ev_eph, 0));
            }
            log = sl->log + (size_t)off * S;
            if (c->samp_on) {
                // end the segment at the next sample step
                const int64_t next = (c->step / c->samp.every + 1) * c->samp.every;
                m = std::min<int64_t>(m, next - c->step);
            }
        }
        // Every segment ends open (the full kick that an uncut run applies there) and
        // publishes the live particles' synchronised states by id, so that cuts -- call
        // ends, first-chunk pieces, sample steps -- leave no trace in the trajectory.
        if (c->n_live > 0) {
            ChunkArgs a{};
            a.pc = nullptr;
            a.log = log;
            a.n = c->n_live;
            a.ld = c->cap;
            a.st = c->d_st[c->cur];
            a.id = c->d_id[c->cur];
            a.alive = c->d_alive;
            a.step0 = c->step;
            a.nsteps = (int32_t)m;
            a.test_first = c->tested_first ? 0 : 1;
            a.open_in = c->tested_first ? 1 : 0;  // after the first segment the slots hold open velocities
            a.close_out = 0;
            a.out_state = c->d_out_state;
            a.out_step = c->d_out_step;
            a.out_reason = c->d_out_reason;
            a.steps_done = c->d_steps;
            a.live_out = c->d_live;
            TaskArgs tasks{};
            tasks.task_counter = c->d_task;
            tasks.group_done = c->d_group_done;
            tasks.status = c->d_status;

            GL_CUDA(cudaMemsetAsync(c->d_live, 0, sizeof(unsigned long long), c->s));
            NvtxRange seg("glisse: particle segment");
            if (c->timing) GL_CUDA(cudaEventRecord(c->tp0, c->s));
            if (c->o.kepler_mode == GLISSE_KEPLER_PAPER_FIXED)
                GL_CUDA(launch_particle_chunk_paper(c->np, a, c->ppc, c->s));
            else
                GL_CUDA(launch_particle_chunk(c->np, a, c->ppc, c->s,
                                              c->o.launch_mode == GLISSE_LAUNCH_PLAIN ? nullptr : &tasks,
                                              c->o.launch_mode == GLISSE_LAUNCH_TASKS));
            if (c->timing) {
                GL_CUDA(cudaEventRecord(c->tp1, c->s));
                GL_CUDA(cudaEventSynchronize(c->tp1));
                float ms = 0.f;
                GL_CUDA(cudaEventElapsedTime(&ms, c->tp0, c->tp1));
                c->acc.particle_ms += ms;
                ++c->acc.particle_launches;
                GL_CUDA(cudaMemcpy(c->h_steps, c->d_steps, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
                c->acc.particle_steps = (int64_t)*c->h_steps;
            }
        }
        if (c->timing && sl && sl->pending) {
            // the main stream has waited for this chunk's ephemeris: its events are complete
            GL_CUDA(cudaEventSynchronize(sl->te1));
            float ms = 0.f;
            GL_CUDA(cudaEventElapsedTime(&ms, sl->te0, sl->te1));
            c->acc.ephemeris_ms += ms;
            ++c->acc.ephemeris_launches;
            sl->pending = false;
        }
        c->tested_first = true;
        if (c->samp_on && sl && (c->step + m) % c->samp.every == 0) {
            // sample the particles live at step + m, with the planets of that step
            const int64_t off = c->step - (c->step / c->C) * c->C;
            if ((rc = take_sample(c, sl->hist + (size_t)(off + m) * 6 * c->np, c->step + m)) != GLISSE_OK)
                break;
        }
        if (sl) {
            GL_CUDA(cudaEventRecord(sl->ev_use, c->s));
            sl->used = true;
        }
        c->step += m;
        remaining -= m;
        if (c->external) c->ext_off += m;
        // compaction only at chunk boundaries (every resync_chunks chunks), at the same global
        // steps however the run is split into calls: warps keep their members in between
        if (c->step % c->C != 0) continue;
        ++c->since_compact;
        if (c->since_compact >= c->o.resync_chunks) rc = compact(c);
    }
    if (rc == GLISSE_OK && c->n_live > 0)
        GL_CUDA(cudaMemcpyAsync(c->h_live, c->d_live, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
    if (rc == GLISSE_OK) rc = check_status(c);
    if (rc == GLISSE_OK) c->n_alive = c->n_live > 0 ? (int64_t)*c->h_live : 0;
    if (prev != c->device) cudaSetDevice(prev);
    return rc;
}

extern "C" int glisse_read(glisse_ctx* c, double* state, uint8_t* alive, int64_t* removal_step,
                           int32_t* removal_reason) {
    if (!c) return GLISSE_E_INVAL;
    NvtxRange range("glisse_read");
    const int64_t n = c->n_total;
    if (n == 0) return GLISSE_OK;
    // before the first step the slots hold the synchronised states; afterwards every segment
    // has published them by id (the slots then hold open velocities)
    if (!c->tested_first)
        GL_CUDA(launch_export_live(c->n_live, c->d_st[c->cur], c->cap, c->d_id[c->cur], c->d_out_state, c->s));
    if (state) GL_CUDA(cudaMemcpyAsync(state, c->d_out_state, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->s));
    int64_t* steps = removal_step;
    int64_t* tmp = nullptr;
    if (!steps && alive) {
        tmp = new (std::nothrow) int64_t[n];
        if (!tmp) return GLISSE_E_NOMEM;
        steps = tmp;
    }
    cudaError_t e = cudaSuccess;
    if (steps) e = cudaMemcpyAsync(steps, c->d_out_step, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess && removal_reason)
        e = cudaMemcpyAsync(removal_reason, c->d_out_reason, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e == cudaSuccess && alive)
        for (int64_t i = 0; i < n; ++i) alive[i] = steps[i] < 0 ? 1 : 0;
    delete[] tmp;
    return e == cudaSuccess ? GLISSE_OK : GLISSE_E_CUDA;
}

extern "C" int glisse_status(glisse_ctx* c, int64_t* n_live, int64_t* step, double* t) {
    if (!c) return GLISSE_E_INVAL;
    if (n_live) *n_live = c->n_alive;
    if (step) *step = c->step;
    if (t) *t = (double)c->step * c->dt;
    return GLISSE_OK;
}

extern "C" int glisse_read_planets(glisse_ctx* c, double* planets, double* t) {
    if (!c) return GLISSE_E_INVAL;
    if (c->external || !c->planets_valid) return GLISSE_E_STATE;
    if (t) *t = (double)c->step * c->dt;
    if (c->np == 0) return GLISSE_OK;
    if (!planets) return GLISSE_E_INVAL;
    const int64_t j = c->step / c->C;
    const int64_t off = c->step - j * c->C;
    int rc = ensure_chunk(c, j);
    if (rc) return rc;
    const Slot& sl = c->ring[(size_t)(j % (int64_t)c->ring.size())];
    if (sl.chunk != j) return GLISSE_E_STATE;
    GL_CUDA(cudaStreamSynchronize(c->se));
    double buf[6 * GLISSE_MAX_PLANETS];
    GL_CUDA(cudaMemcpy(buf, sl.hist + (size_t)off * 6 * c->np, sizeof(double) * 6 * c->np,
                       cudaMemcpyDeviceToHost));
    for (int p = 0; p < c->np; ++p) {
        planets[7 * p] = c->hpc.m[p];
        for (int d = 0; d < 6; ++d) planets[7 * p + 1 + d] = buf[6 * p + d];
    }
    return GLISSE_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume.  Buffer: a fixed header, then the arrays, each at an
// 8-byte offset: the chunk-start Jacobi state [np][6], the particle slots
// [6][n_live], the per-id frozen states [n_total][6], removal steps [n_total],
// slot ids [n_live], reasons [n_total], slot flags [n_live]; with element
// sampling set, the kept samples' steps [kept] and elements [kept][n_total][6]
// and the libration flags and counts [n_total].
// ---------------------------------------------------------------------------
namespace {
constexpr char kCkptMagic[8] = {'G', 'L', 'I', 'S', 'S', 'E', 'C', 'K'};
constexpr int32_t kCkptVersion = 2;  // 2: slots hold open velocities after the first step

struct CkptHeader {
    char magic[8];
    int32_t version;
    int32_t header_bytes;
    int32_t np;
    int32_t chunk_steps, resync_chunks, kepler_mode, kepler_iters, enc_mode, sort_mode;
    int32_t tested_first;
    double m0, dt, enc_value, r_max;
    int64_t n_total, n_live, step, since_compact;
    int64_t total_bytes;
    PlanetConsts pc;
    // element sampling (glisse_set_sampling): on or off, its settings, samples taken and kept
    int32_t samp_on, pad2;
    int64_t samp_seen, samp_kept;
    glisse_sampling samp;
};

struct CkptLayout {
    size_t jac0, st, out_state, out_step, id, out_reason, alive, samp_steps, elem, near0, near180, count, total;
};

CkptLayout ckpt_layout(int np, int64_t n_total, int64_t n_live, bool samp_on = false, int64_t kept = 0) {
    CkptLayout L{};
    size_t off = (sizeof(CkptHeader) + 7) & ~size_t(7);
    auto take = [&off](size_t bytes) {
        const size_t o = off;
        off += (bytes + 7) & ~size_t(7);
        return o;
    };
    L.jac0 = take(sizeof(double) * 6 * (size_t)np);
    L.st = take(sizeof(double) * 6 * (size_t)n_live);
    L.out_state = take(sizeof(double) * 6 * (size_t)n_total);
    L.out_step = take(sizeof(int64_t) * (size_t)n_total);
    L.id = take(sizeof(int32_t) * (size_t)n_live);
    L.out_reason = take(sizeof(int32_t) * (size_t)n_total);
    L.alive = take((size_t)n_live);
    const size_t ns = samp_on ? (size_t)n_total : 0;
    L.samp_steps = take(sizeof(int64_t) * (samp_on ? (size_t)kept : 0));
    L.elem = take(sizeof(double) * 6 * ns * (samp_on ? (size_t)kept : 0));
    L.near0 = take(ns);
    L.near180 = take(ns);
    L.count = take(sizeof(int32_t) * ns);
    L.total = off;
    return L;
}

int ckpt_state_ok(const glisse_ctx* c) {
    if (c->external || !c->planets_valid) return GLISSE_E_STATE;
    return GLISSE_OK;
}

CkptLayout ckpt_layout_of(const glisse_ctx* c) {
    return ckpt_layout(c->np, c->n_total, c->n_live, c->samp_on, (int64_t)c->samp_steps.size());
}
}  // namespace

extern "C" int glisse_sizes(glisse_ctx* c, int64_t* n_particles, int32_t* n_planets) {
    if (!c) return GLISSE_E_INVAL;
    if (n_particles) *n_particles = c->n_total;
    if (n_planets) *n_planets = c->np;
    return GLISSE_OK;
}

extern "C" int glisse_checkpoint_size(glisse_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return GLISSE_E_INVAL;
    const int st = ckpt_state_ok(c);
    if (st != GLISSE_OK) return st;
    *bytes = (int64_t)ckpt_layout_of(c).total;
    return GLISSE_OK;
}

extern "C" int glisse_checkpoint(glisse_ctx* c, void* buf, int64_t bytes) {
    if (!c || !buf) return GLISSE_E_INVAL;
    const int st = ckpt_state_ok(c);
    if (st != GLISSE_OK) return st;
    const CkptLayout L = ckpt_layout_of(c);
    if (bytes < (int64_t)L.total) return GLISSE_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != c->device) GL_CUDA(cudaSetDevice(c->device));
    NvtxRange range("glisse_checkpoint");
    int rc = GLISSE_OK;
    char* out = static_cast<char*>(buf);
    std::memset(out, 0, L.total);  // the gaps between arrays too: equal contexts, equal bytes
    // the Jacobi state the current chunk's planet kernel started from
    const int64_t j = c->step / c->C;
    if ((rc = ensure_chunk(c, j)) == GLISSE_OK) {
        const Slot& sl = c->ring[(size_t)(j % (int64_t)c->ring.size())];
        cudaError_t e = sl.chunk == j ? cudaSuccess : cudaErrorInvalidValue;
        if (sl.chunk != j) rc = GLISSE_E_STATE;
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->se);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e == cudaSuccess && c->np > 0)
            e = cudaMemcpy(out + L.jac0, sl.hist + (size_t)(c->C + 1) * 6 * c->np, sizeof(double) * 6 * c->np,
                           cudaMemcpyDeviceToHost);
        const int64_t n = c->n_live, N = c->n_total;
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpy2D(out + L.st, sizeof(double) * (size_t)n, c->d_st[c->cur], sizeof(double) * (size_t)c->cap,
                             sizeof(double) * (size_t)n, 6, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpy(out + L.id, c->d_id[c->cur], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && n > 0) e = cudaMemcpy(out + L.alive, c->d_alive, (size_t)n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && N > 0)
            e = cudaMemcpy(out + L.out_state, c->d_out_state, sizeof(double) * 6 * (size_t)N, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && N > 0)
            e = cudaMemcpy(out + L.out_step, c->d_out_step, sizeof(int64_t) * (size_t)N, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && N > 0)
            e = cudaMemcpy(out + L.out_reason, c->d_out_reason, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost);
        if (c->samp_on && N > 0) {
            const size_t kept = c->samp_steps.size();
            if (kept > 0) std::memcpy(out + L.samp_steps, c->samp_steps.data(), sizeof(int64_t) * kept);
            if (e == cudaSuccess && kept > 0)
                e = cudaMemcpy(out + L.elem, c->d_elem, sizeof(double) * 6 * (size_t)N * kept, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(out + L.near0, c->d_near0, (size_t)N, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(out + L.near180, c->d_near180, (size_t)N, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                e = cudaMemcpy(out + L.count, c->d_count, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost);
        } else if (c->samp_on && !c->samp_steps.empty()) {
            std::memcpy(out + L.samp_steps, c->samp_steps.data(), sizeof(int64_t) * c->samp_steps.size());
        }
        if (rc == GLISSE_OK && e != cudaSuccess) {
            (void)cudaGetLastError();
            rc = GLISSE_E_CUDA;
        }
    }
    if (rc == GLISSE_OK) {
        CkptHeader h;
        std::memset(&h, 0, sizeof(h));
        std::memcpy(h.magic, kCkptMagic, sizeof(kCkptMagic));
        h.version = kCkptVersion;
        h.header_bytes = (int32_t)sizeof(CkptHeader);
        h.np = c->np;
        h.chunk_steps = c->o.chunk_steps;
        h.resync_chunks = c->o.resync_chunks;
        h.kepler_mode = c->o.kepler_mode;
        h.kepler_iters = c->o.kepler_iters;
        h.enc_mode = c->o.enc_mode;
        h.sort_mode = c->o.sort_mode;
        h.tested_first = c->tested_first ? 1 : 0;
        h.m0 = c->m0;
        h.dt = c->dt;
        h.enc_value = c->o.enc_value;
        h.r_max = c->o.r_max;
        h.n_total = c->n_total;
        h.n_live = c->n_live;
        h.step = c->step;
        h.since_compact = c->since_compact;
        h.total_bytes = (int64_t)L.total;
        h.pc = c->hpc;
        h.samp_on = c->samp_on ? 1 : 0;
        if (c->samp_on) {
            h.samp = c->samp;
            h.samp_seen = c->samp_seen;
            h.samp_kept = (int64_t)c->samp_steps.size();
        }
        std::memcpy(out, &h, sizeof(h));
    }
    if (prev != c->device) cudaSetDevice(prev);
    return rc;
}

extern "C" int glisse_resume(glisse_ctx** out, const void* buf, int64_t bytes, const glisse_opts* opts) {
    if (!out) return GLISSE_E_INVAL;
    *out = nullptr;
    if (!buf || bytes < (int64_t)sizeof(CkptHeader)) return GLISSE_E_INVAL;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, sizeof(kCkptMagic)) != 0 || h.version != kCkptVersion ||
        h.header_bytes != (int32_t)sizeof(CkptHeader))
        return GLISSE_E_INVAL;
    if (h.np < 0 || h.np > GLISSE_MAX_PLANETS || h.pc.np != h.np) return GLISSE_E_INVAL;
    if (h.n_total < 0 || h.n_total > INT32_MAX || h.n_live < 0 || h.n_live > h.n_total) return GLISSE_E_INVAL;
    if (h.step < 0 || h.since_compact < 0 || (h.tested_first != 0 && h.tested_first != 1)) return GLISSE_E_INVAL;
    if (!(h.m0 > 0.0) || !std::isfinite(h.m0) || !(h.dt != 0.0) || !std::isfinite(h.dt)) return GLISSE_E_INVAL;
    if (h.chunk_steps < 1 || h.chunk_steps > (1 << 20) || h.resync_chunks < 1) return GLISSE_E_INVAL;
    if (h.kepler_mode != GLISSE_KEPLER_CONVERGE && h.kepler_mode != GLISSE_KEPLER_PAPER_FIXED) return GLISSE_E_INVAL;
    if (h.kepler_mode == GLISSE_KEPLER_PAPER_FIXED && (h.kepler_iters < 1 || h.kepler_iters > GLISSE_MAX_KEPLER_ITERS))
        return GLISSE_E_INVAL;
    if (h.enc_mode != GLISSE_ENC_HILL && h.enc_mode != GLISSE_ENC_FIXED) return GLISSE_E_INVAL;
    if (h.sort_mode != GLISSE_SORT_NONE && h.sort_mode != GLISSE_SORT_COST) return GLISSE_E_INVAL;
    if (!(h.enc_value >= 0.0) || !std::isfinite(h.enc_value) || !std::isfinite(h.r_max)) return GLISSE_E_INVAL;
    if (h.samp_on != 0 && h.samp_on != 1) return GLISSE_E_INVAL;
    if (h.samp_on && (h.samp.max_samples < 0 || (uint64_t)h.samp.max_samples > (uint64_t)1 << 40 ||
                      h.samp_kept < 0 || h.samp_kept > h.samp.max_samples || h.samp_seen < h.samp_kept))
        return GLISSE_E_INVAL;
    if (h.samp_on) {  // the kept samples must fit in the buffer before the layout is computed from them
        size_t eb = 0;
        if (!elem_bytes(h.n_total, h.samp_kept, &eb) || eb > (size_t)bytes) return GLISSE_E_INVAL;
    }
    const CkptLayout L = ckpt_layout(h.np, h.n_total, h.n_live, h.samp_on != 0, h.samp_on ? h.samp_kept : 0);
    if (h.total_bytes != (int64_t)L.total || bytes < h.total_bytes) return GLISSE_E_INVAL;
    const char* in = static_cast<const char*>(buf);
    // every slot id must name a distinct particle: the kernels write per-id outputs through them
    {
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
    o.resync_chunks = h.resync_chunks;
    o.kepler_mode = h.kepler_mode;
    o.kepler_iters = h.kepler_iters;
    o.enc_mode = h.enc_mode;
    o.sort_mode = h.sort_mode;
    o.enc_value = h.enc_value;
    o.r_max = h.r_max;
    if (opts) {
        if (opts->launch_mode < GLISSE_LAUNCH_AUTO || opts->launch_mode > GLISSE_LAUNCH_TASKS) return GLISSE_E_INVAL;
        o.cuda_stream = opts->cuda_stream;
        o.timing = opts->timing;
        o.launch_mode = opts->launch_mode;
    }
    glisse_ctx* c = new (std::nothrow) glisse_ctx();
    if (!c) return GLISSE_E_NOMEM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return GLISSE_E_CUDA;
    }
    c->o = o;
    c->np = h.np;
    c->m0 = h.m0;
    c->dt = h.dt;
    c->C = o.chunk_steps;
    c->n_total = h.n_total;
    c->timing = o.timing != 0;
    Restore r;
    r.pc = h.pc;
    r.jac0 = reinterpret_cast<const double*>(in + L.jac0);
    r.st = reinterpret_cast<const double*>(in + L.st);
    r.id = reinterpret_cast<const int32_t*>(in + L.id);
    r.alive = reinterpret_cast<const uint8_t*>(in + L.alive);
    r.out_state = reinterpret_cast<const double*>(in + L.out_state);
    r.out_step = reinterpret_cast<const int64_t*>(in + L.out_step);
    r.out_reason = reinterpret_cast<const int32_t*>(in + L.out_reason);
    r.n_live = h.n_live;
    r.step = h.step;
    r.since_compact = h.since_compact;
    r.tested_first = h.tested_first != 0;
    NvtxRange range("glisse_resume");
    int rc = setup(c, nullptr, nullptr, &r);
    if (rc == GLISSE_OK && h.samp_on) {
        // sampling as it was: settings (validated as glisse_set_sampling does), kept
        // samples, libration flags and counts
        rc = glisse_set_sampling(c, &h.samp);
        const size_t N = (size_t)c->n_total, kept = (size_t)h.samp_kept;
        cudaError_t e = cudaSuccess;
        if (rc == GLISSE_OK && N > 0) {
            if (kept > 0)
                e = cudaMemcpy(c->d_elem, in + L.elem, sizeof(double) * 6 * N * kept, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->d_near0, in + L.near0, N, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->d_near180, in + L.near180, N, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->d_count, in + L.count, sizeof(int32_t) * N, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                rc = GLISSE_E_CUDA;
            }
        }
        if (rc == GLISSE_OK) {
            c->samp_steps.resize(kept);
            if (kept > 0) std::memcpy(c->samp_steps.data(), in + L.samp_steps, sizeof(int64_t) * kept);
            c->samp_seen = h.samp_seen;
        }
    }
    if (rc != GLISSE_OK) {
        ctx_free(c);
        return rc;
    }
    *out = c;
    return GLISSE_OK;
}

extern "C" int glisse_set_ephemeris(glisse_ctx* c, const double* log, int64_t n_steps) {
    if (!c || n_steps < 1 || (!log && c->np > 0)) return GLISSE_E_INVAL;
    if (c->samp_on) return GLISSE_E_STATE;  // sampling needs the planets' velocities
    const int S = log_stride(c->np);
    GL_CUDA(cudaStreamSynchronize(c->s));
    GL_CUDA(cudaStreamSynchronize(c->se));
    cudaFree(c->d_ext_log);
    c->d_ext_log = nullptr;
    GL_ALLOC(c->d_ext_log, sizeof(double) * (size_t)(n_steps + 1) * S);
    if (c->np > 0) {
        double* d_pos = nullptr;
        GL_ALLOC(d_pos, sizeof(double) * (size_t)(n_steps + 1) * 3 * c->np);
        cudaError_t e = cudaMemcpyAsync(d_pos, log, sizeof(double) * (size_t)(n_steps + 1) * 3 * c->np,
                                        cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = launch_eph_external(c->d_pc, d_pos, n_steps + 1, c->d_ext_log, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        cudaFree(d_pos);
        if (e != cudaSuccess) return GLISSE_E_CUDA;
    } else {
        GL_CUDA(cudaMemsetAsync(c->d_ext_log, 0, sizeof(double) * (size_t)(n_steps + 1) * S, c->s));
        GL_CUDA(cudaStreamSynchronize(c->s));
    }
    c->external = true;
    c->planets_valid = false;
    c->ext_n = n_steps;
    c->ext_off = 0;
    return GLISSE_OK;
}

extern "C" int glisse_partition_device(int64_t n, int64_t ld, const uint8_t* alive, const double* src,
                                       const int32_t* src_id, double* dst, int32_t* dst_id, int64_t* n_out,
                                       void* stream) {
    if (n < 0 || ld < n || !n_out) return GLISSE_E_INVAL;
    if (n > 0 && (!alive || !src || !src_id || !dst || !dst_id)) return GLISSE_E_INVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t* counts = nullptr;
    int rc = alloc_dev(reinterpret_cast<void**>(&counts), sizeof(int64_t) * (size_t)compact_scratch_entries(n));
    if (rc) return rc;
    cudaError_t e = launch_compact(n, alive, src, src_id, ld, dst, dst_id, ld, counts, n_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(counts);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    return GLISSE_OK;
}

extern "C" int glisse_timings(glisse_ctx* c, glisse_timing* out, int32_t reset) {
    if (!c) return GLISSE_E_INVAL;
    if (!c->timing) return GLISSE_E_STATE;
    if (out) *out = c->acc;
    if (reset) {
        std::memset(&c->acc, 0, sizeof(c->acc));
        GL_CUDA(cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned long long), c->s));
        GL_CUDA(cudaStreamSynchronize(c->s));
    }
    return GLISSE_OK;
}
