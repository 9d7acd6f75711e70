// rip_digest.cu -- position-dependent 64-bit digest of an array, used to
// compare device outputs with the CPU oracle where a second host copy of the
// output does not fit:
//   H = sum_p splitmix64(p * 0x9E3779B97F4A7C15 ^ v(p)) mod 2^64,
//   v(p) = splitmix64 chained over the element's 8-byte little-endian words.
// splitmix64 is the finaliser published by Steele, Lea and Flood (2014).
#include "rip_internal.cuh"

namespace rip {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t elem_hash(uint32_t v) { return mix64((uint64_t)v); }
__device__ __forceinline__ uint64_t elem_hash(uint64_t v) { return mix64(v); }
__device__ __forceinline__ uint64_t elem_hash(uint4 v) {
    const uint64_t lo = (uint64_t)v.x | ((uint64_t)v.y << 32);
    const uint64_t hi = (uint64_t)v.z | ((uint64_t)v.w << 32);
    return mix64(mix64(lo) ^ hi);
}

template <int W>
__global__ void digest_kernel(const void* data, uint64_t n, unsigned long long* out) {
    using T = typename Elem<W>::T;
    const T* x = reinterpret_cast<const T*>(data);
    uint64_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        acc += mix64(p * 0x9E3779B97F4A7C15ull ^ elem_hash(x[p]));
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    __shared__ uint64_t part[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (blockDim.x >> 5) ? part[lane] : 0;
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        if (lane == 0) atomicAdd(out, (unsigned long long)acc);
    }
}

}  // namespace

cudaError_t launch_digest(const void* data, uint64_t n, uint32_t w, unsigned long long* out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = (uint32_t)(sms > 0 ? sms * 8 : 1024);
    ProfScope p("digest", s);
    switch (w) {
        case 4: digest_kernel<4><<<grid, 256, 0, s>>>(data, n, out); break;
        case 8: digest_kernel<8><<<grid, 256, 0, s>>>(data, n, out); break;
        default: digest_kernel<16><<<grid, 256, 0, s>>>(data, n, out); break;
    }
    return cudaGetLastError();
}

}  // namespace rip
