// partition_noalloc.cu -- stable partition with no memory allocation.
//
// glisse_partition_device allocates its scratch (one int64 per 2048-slot tile)
// with cudaMalloc on every call.  Some callers cannot allow that: programs
// whose device memory is all handed out by a framework or pool allocator that
// forbids allocations behind its back, programs that reserve a fixed memory
// budget at start-up, and loops where an allocation's implicit synchronisation
// or its failure part-way through a run is not acceptable.  This
// entry point runs the same three kernels but takes its scratch from a
// fixed-size array that lives in the library's device image (256 KiB).  The
// array exists on a device once the CUDA driver has loaded this library's
// module there.  With lazy module loading (CUDA's default) that happens at the
// first use of the module on the device -- possibly this entry point's first
// call, whose symbol lookup then makes the driver place the module, array
// included, in device memory.  From then on the array stays until the process
// exits (or the device's context is destroyed) and no call allocates.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side shadow), so every call asks the runtime for the address
// with cudaGetSymbolAddress, with the caller's device current.  The lookup is
// a host-side table query once the module is loaded; doing it per call (not
// caching it) keeps the address right if the context was reset and rebuilt.
#include <cuda_runtime.h>

#include "glisse_internal.h"

namespace glisse {
cudaError_t launch_compact(int64_t, const uint8_t*, const double*, const int32_t*, int64_t, double*, int32_t*,
                           int64_t, int64_t*, int64_t*, cudaStream_t);
int64_t compact_scratch_entries(int64_t);

namespace {
// tile counts / offsets of one call: one int64 per 2048-slot tile of the partition
constexpr int64_t kNoAllocTiles = GLISSE_PARTITION_NOALLOC_MAX / 2048;
}  // namespace

static __device__ __align__(256) int64_t g_partition_scratch[kNoAllocTiles];

// Device address of g_partition_scratch on the current device.
static cudaError_t scratch_address(int64_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partition_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<int64_t*>(p);
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
