// partition_noalloc.cu -- stable partition with no memory allocation.
//
// glisse_partition_device allocates its scratch (one int64 per 2048-slot tile)
// with cudaMalloc on every call.  Some callers cannot allow that: programs
// whose device memory is all handed out by a framework or pool allocator that
// forbids allocations behind its back, programs that reserve a fixed memory
// budget at start-up, and loops where an allocation's implicit synchronisation
// or its failure part-way through a run is not acceptable.  This
// entry point runs the same three kernels but takes its scratch from a
// fixed-size array that lives in the library's device image: it is created
// when the library's module is loaded on a device and stays allocated there
// until the process exits (256 KiB per GPU that loads the library).
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side shadow), so the first call on each device asks the runtime
// for the address with cudaGetSymbolAddress, with that device current, and
// remembers it.
#include <cuda_runtime.h>

#include <mutex>

#include "glisse_internal.h"

namespace glisse {
cudaError_t launch_compact(int64_t, const uint8_t*, const double*, const int32_t*, int64_t, double*, int32_t*,
                           int64_t, int64_t*, int64_t*, cudaStream_t);
int64_t compact_scratch_entries(int64_t);

namespace {
// tile counts / offsets of one call: one int64 per 2048-slot tile of the partition
constexpr int64_t kNoAllocTiles = GLISSE_PARTITION_NOALLOC_MAX / 2048;

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
int64_t* g_addr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) int64_t g_partition_scratch[kNoAllocTiles];

// Device address of g_partition_scratch on the current device (looked up once per device).
static cudaError_t scratch_address(int64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partition_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<int64_t*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace glisse

extern "C" int glisse_partition_device_noalloc(int64_t n, int64_t ld, const uint8_t* alive, const double* src,
                                               const int32_t* src_id, double* dst, int32_t* dst_id, int64_t* n_out,
                                               void* stream) {
    using namespace glisse;
    if (n < 0 || ld < n || !n_out) return GLISSE_E_INVAL;
    if (n > GLISSE_PARTITION_NOALLOC_MAX || compact_scratch_entries(n) > kNoAllocTiles) return GLISSE_E_INVAL;
    if (n > 0 && (!alive || !src || !src_id || !dst || !dst_id)) return GLISSE_E_INVAL;
    int64_t* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    // Nothing in the array needs clearing: the count kernel writes every entry the
    // scan and scatter kernels read before they read it.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_compact(n, alive, src, src_id, ld, dst, dst_id, ld, scratch, n_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GLISSE_E_CUDA;
    }
    return GLISSE_OK;
}
