// rip_noalloc.cu -- rip_shuffle_noalloc: the shuffle with a workspace that is
// a fixed array in device memory, for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework's own
// device allocator or memory pool (allocating there would re-enter the pool),
// processes whose device memory is fully reserved up front by a pool owner, and
// latency-critical paths where cudaMalloc's implicit device synchronisation is
// not acceptable.  For them this entry point uses the file-scope array below as
// its workspace and performs no allocation of any kind.
//
// The array is part of the library's device image: every GPU that loads the
// library holds its RIP_NOALLOC_WS_BYTES until the process exits.  All calls
// share it and it keeps the last call's contents; everything a call needs to
// start at zero (list counts, counters, the slot table) is cleared by the call
// itself on its stream.  Calls that overlap on the GPU (several streams, or
// several host threads without ordering) race on the array and must be
// serialised by the caller.
#include <mutex>

#include "rip_internal.cuh"

namespace rip {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_ws[RIP_NOALLOC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device (the first call on a device does this set-up).
int noalloc_workspace(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RIP_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return RIP_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) {
            cudaGetLastError();
            return RIP_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RIP_OK;
}

}  // namespace
}  // namespace rip

extern "C" int rip_shuffle_noalloc(void* data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                                   const rip_plan* plan, rip_stream_t stream) {
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return RIP_EINVAL;
    if (n <= 1) return RIP_OK;
    const size_t need = rip_shuffle_workspace_size(n, elem_bytes, plan);
    if (need == 0) return RIP_EINVAL;
    if (need > (size_t)RIP_NOALLOC_WS_BYTES) return RIP_ETOOLARGE;
    void* ws = nullptr;
    const int rc = rip::noalloc_workspace(&ws);
    if (rc != RIP_OK) return rc;
    return rip_shuffle_ex(data, n, elem_bytes, seed, plan, ws, (size_t)RIP_NOALLOC_WS_BYTES, stream);
}
