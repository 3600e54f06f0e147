// noalloc.cu -- drt3d_planes_forward_noalloc: the planes forward transform
// with its intermediate buffers in a fixed, library-owned device array
// instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they run the
// transform: code running inside a host callback or a real-time loop that
// must not call into the allocator, plug-in hosts that hand out only the
// input and output buffers, or processes whose device memory is fully
// reserved up front by another framework.  This entry point lets them run
// the forward transform with nothing but the input and output they already
// have.
//
// The scratch is a file-scope __device__ array of kNoallocScratchBytes
// (16 MiB).  Every GPU on which this library's module is loaded holds it
// until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device looks the address up
// with cudaGetSymbolAddress (with that device current) and caches it.
//
// Nothing in the scratch has to start at zero: each pass writes every
// element of an intermediate row before the next pass reads it, so stale
// contents from an earlier call are never observed.  All calls share the one
// array, so two calls that overlap on the GPU (different streams, or host
// threads on the same device) race on it and must be serialised by the
// caller.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).  Returns nullptr on failure.
void* noalloc_scratch_current_device(cudaError_t* err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_noalloc_ptr[dev] = p;
    }
    *err = cudaSuccess;
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" {

size_t drt3d_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

drt3d_status drt3d_planes_forward_noalloc(const drt3d_plan* plan, const void* d_in, void* d_out,
                                          uint32_t dodecant_mask, cudaStream_t stream) {
    if (!plan || !d_in || !d_out) return DRT3D_ERR_INVALID_ARG;
    // The scratch address below is the current device's: it must be the plan's.
    if (!drt3d::device_is_current(plan->device)) return DRT3D_ERR_INVALID_ARG;
    if (dodecant_mask == 0 || (dodecant_mask & ~DRT3D_ALL_DODECANTS)) return DRT3D_ERR_INVALID_ARG;
    // Scratch this call needs: two intermediate buffers per selected
    // dodecant (none when the schedule is a single pass).
    int nslots = 0;
    for (int k = 0; k < 12; ++k) nslots += (dodecant_mask >> k) & 1;
    const size_t need = plan->fused.npass > 1 ? (size_t)nslots * 2 * plan->fused.buf_bytes : 0;
    if (need > kNoallocScratchBytes) return DRT3D_ERR_SCRATCH_LIMIT;
    cudaError_t err = cudaSuccess;
    void* scratch = noalloc_scratch_current_device(&err);
    if (!scratch) return DRT3D_ERR_CUDA;
    return drt3d_planes_forward(plan, d_in, d_out, dodecant_mask, scratch, kNoallocScratchBytes, stream);
}

}  // extern "C"
