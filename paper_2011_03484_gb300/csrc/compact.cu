// compact.cu -- stable partition of live particles between chunks (section 2.2).
//
// Every resync interval the paper moves deactivated particles to the end of
// the arrays with a stable partition, so live particles keep their relative
// order and the kernel's threads only see live ones.  Here live entries are
// copied, in order, into a second set of planes:
//   1. count: live entries per tile of kTile slots
//   2. scan:  exclusive prefix of the tile counts (one block), total -> n_out
//   3. scatter: per tile, rounds of 256 slots; a warp ballot ranks the live
//      slots inside a warp, warp totals rank warps inside the block, and the
//      tile offset places the block; each live slot writes its six state
//      values and its id.
// The pass is bound by HBM traffic: 8 x 6 + 4 bytes read and written per
// live particle plus one byte of flag per slot.
//
// The same three kernels select slots whose key equals a given value and
// place them after a device-side base offset, so a stable partition into
// several groups is one pass per group (used to order live particles by the
// expected cost of their Kepler solve, section 2.2's sorting suggestion).
// A wanted value of 0 (kAnyNonZero) selects every slot whose key is non-zero:
// that is the plain live/removed partition, where any non-zero flag keeps.
#include <cuda_runtime.h>

#include "glisse_internal.h"

namespace glisse {

constexpr int kCompactThreads = 256;
constexpr int kCompactRounds = 8;
constexpr int kTile = kCompactThreads * kCompactRounds;
constexpr uint8_t kAnyNonZero = 0;

__device__ __forceinline__ bool selected(uint8_t key, uint8_t want) {
    return want == kAnyNonZero ? key != 0 : key == want;
}

__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(const uint8_t* __restrict__ key, uint8_t want,
                                                                         int64_t n, int64_t* __restrict__ counts) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int c = 0;
#pragma unroll
    for (int r = 0; r < kCompactRounds; ++r) {
        const int64_t idx = base + r * kCompactThreads + threadIdx.x;
        c += (idx < n && selected(key[idx], want)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    __shared__ int wsum[kCompactThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of counts[0..nb) in place, starting at *base (0 when base is
// null); base + total to *n_out.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) compact_scan_kernel(int64_t* __restrict__ counts, int64_t nb,
                                                              const int64_t* base, int64_t* n_out) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = base ? *base : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t idx = b0 + threadIdx.x;
        const int64_t v = idx < nb ? counts[idx] : 0;
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t ws = wsum[lane];
            int64_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;  // exclusive warp offsets
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

__global__ void __launch_bounds__(kCompactThreads) compact_scatter_kernel(
    const uint8_t* __restrict__ key, uint8_t want, int64_t n, const int64_t* __restrict__ offsets,
    const double* __restrict__ src,
    const int32_t* __restrict__ src_id, int64_t lds, double* __restrict__ dst, int32_t* __restrict__ dst_id,
    int64_t ldd) {
    __shared__ int wcnt[kCompactThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t out = offsets[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kCompactRounds; ++r) {
        const int64_t idx = base + r * kCompactThreads + threadIdx.x;
        const bool f = idx < n && selected(key[idx], want);
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, f);
        const int rank = __popc(ball & ((1u << lane) - 1u));
        if (lane == 0) wcnt[warp] = __popc(ball);
        __syncthreads();
        int woff = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kCompactThreads / 32; ++w) {
            woff += (w < warp) ? wcnt[w] : 0;
            tot += wcnt[w];
        }
        if (f) {
            const int64_t d = out + woff + rank;
#pragma unroll
            for (int c = 0; c < 6; ++c) dst[c * ldd + d] = src[c * lds + idx];
            dst_id[d] = src_id[idx];
        }
        out += tot;
        __syncthreads();
    }
}

// Stable partition of n slots.  counts needs ceil(n / kTile) int64 entries of scratch.
cudaError_t launch_compact(int64_t n, const uint8_t* alive, const double* src, const int32_t* src_id, int64_t lds,
                           double* dst, int32_t* dst_id, int64_t ldd, int64_t* counts, int64_t* n_out,
                           cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
    const int64_t nb = (n + kTile - 1) / kTile;
    compact_count_kernel<<<(unsigned)nb, kCompactThreads, 0, s>>>(alive, kAnyNonZero, n, counts);
    compact_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, nullptr, n_out);
    compact_scatter_kernel<<<(unsigned)nb, kCompactThreads, 0, s>>>(alive, kAnyNonZero, n, counts, src, src_id, lds,
                                                                      dst, dst_id, ldd);
    return cudaGetLastError();
}

// Expected cost tier of a particle's drift, from its osculating orbit: the
// fast path's polynomial degree follows z = beta s^2 ~ (n dt)^2 (a / r)^2,
// largest at pericentre, z_q = (n dt / (1 - e))^2.  Tiers 0..3: z_q <= 2^-9
// (degree 3), <= 2^-5 (degree 5), <= 0.1 (degree 7), beyond (the general
// solver near pericentre; also unbound and nearly radial orbits).
__device__ __forceinline__ int cost_tier(const double* st, int64_t ld, int64_t i, double mu, double dt) {
    const double x = st[i], y = st[ld + i], z = st[2 * ld + i];
    const double vx = st[3 * ld + i], vy = st[4 * ld + i], vz = st[5 * ld + i];
    const double r = sqrt(x * x + y * y + z * z);
    const double alpha = 2.0 / r - (vx * vx + vy * vy + vz * vz) / mu;  // 1 / a
    if (!(alpha > 0.0) || !(r * alpha >= 1e-3)) return 3;
    const double ec = 1.0 - r * alpha, rv = x * vx + y * vy + z * vz;
    const double e2 = ec * ec + rv * rv * alpha / mu;
    const double om = sqrt(fmax(1.0 - sqrt(e2), 0.0));  // sqrt(1 - e)
    const double zq = mu * alpha * alpha * alpha * dt * dt / (om * om * om * om);
    return zq <= 0.001953125 ? 0 : zq <= 0.03125 ? 1 : zq <= 0.1 ? 2 : 3;
}

// key[i] = 0 for a removed slot, 1 + cost tier for a live one.
__global__ void sort_key_kernel(int64_t n, const uint8_t* __restrict__ alive, const double* __restrict__ st,
                                int64_t ld, double mu, double dt, uint8_t* __restrict__ key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = alive[i] ? (uint8_t)(1 + cost_tier(st, ld, i, mu, dt)) : (uint8_t)0;
}

// Stable partition of the live slots ordered by cost tier, costliest first
// (section 2.2: the most expensive group starts first); one pass per tier,
// each placed after the previous ones on the device.  key needs n bytes of
// scratch, counts ceil(n / kTile) entries.
cudaError_t launch_compact_sorted(int64_t n, const uint8_t* alive, const double* src, const int32_t* src_id,
                                  int64_t lds, double* dst, int32_t* dst_id, int64_t ldd, int64_t* counts,
                                  uint8_t* key, double mu, double dt, int64_t* n_out, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
    const int64_t nb = (n + kTile - 1) / kTile;
    sort_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, alive, src, lds, mu, dt, key);
    for (int t = 4; t >= 1; --t) {
        compact_count_kernel<<<(unsigned)nb, kCompactThreads, 0, s>>>(key, (uint8_t)t, n, counts);
        compact_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, t == 4 ? nullptr : n_out, n_out);
        compact_scatter_kernel<<<(unsigned)nb, kCompactThreads, 0, s>>>(key, (uint8_t)t, n, counts, src, src_id,
                                                                          lds, dst, dst_id, ldd);
    }
    return cudaGetLastError();
}

int64_t compact_scratch_entries(int64_t n) { return n <= 0 ? 1 : (n + kTile - 1) / kTile; }

// Per-id export of live particles' current state (used by glisse_read).
__global__ void export_live_kernel(int64_t n, const double* __restrict__ st, int64_t ld, const int32_t* __restrict__ id,
                                   double* __restrict__ out_state) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t pid = id[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) out_state[6 * pid + c] = st[c * ld + i];
}

cudaError_t launch_export_live(int64_t n, const double* st, int64_t ld, const int32_t* id, double* out_state,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bs = 256;
    export_live_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(n, st, ld, id, out_state);
    return cudaGetLastError();
}

// Initial SoA planes and ids from the host layout [n][6] (already on the device).
__global__ void import_kernel(int64_t n, const double* __restrict__ aos, double* __restrict__ st, int64_t ld,
                              int32_t* __restrict__ id) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 6; ++c) st[c * ld + i] = aos[6 * i + c];
    id[i] = (int32_t)i;
}

cudaError_t launch_import(int64_t n, const double* aos, double* st, int64_t ld, int32_t* id, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bs = 256;
    import_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(n, aos, st, ld, id);
    return cudaGetLastError();
}

}  // namespace glisse
