// rip_device.cuh -- device-side building blocks of the in-place scatter shuffle.
//
// Random numbers (Sec. 2.3 of the paper: a seedable generator reshaped into
// the needed distributions; Sec. 3.1: a generator that can be replayed):
// Philox-4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed.  Counter
// layouts (this library's reading, identical in the CPU oracle):
//   bucket of logical position pos, level L, subproblem start o:
//     ctr = (q_lo, q_hi, L | 1<<8, o_lo), q = pos >> 2, word pos & 3,
//     bucket = (word * k) >> 32 (k a power of two: the top log2 k bits).
//   Fisher-Yates partner for step i (position p = o + i), s = i + 1:
//     first word: ctr = (q_lo, q_hi, L | 2<<8, o_lo), q = p >> 2, word p & 3;
//     if Lemire rejects it, attempts a = 1, 2, ..:
//     ctr = (p_lo, p_hi, L | 3<<8 | a<<16, o_lo), words 0..3 in order.
// Lemire's bounded sampling ("Fast random integer generation in an
// interval", 2019; Sec. 2.3): x*s = hi:lo; accept hi unless lo < (2^32-s) mod s.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rip_shuffle.h"

namespace rip {

constexpr uint32_t kTagScatter = 1u;
constexpr uint32_t kTagFy = 2u;
constexpr uint32_t kTagFyRetry = 3u;
constexpr uint32_t kDepthCap = 64u;

// ----------------------------------------------------------------- status

// Device status word: first error code wins (atomicCAS from RIP_OK).
struct Status {
    uint32_t code;
    uint32_t where;   // kernel-specific detail for diagnostics
    uint64_t detail;
};

__device__ __forceinline__ void report(Status* st, uint32_t code, uint32_t where, uint64_t detail) {
    if (atomicCAS(&st->code, 0u, code) == 0u) {
        st->where = where;
        st->detail = detail;
    }
}

// Every call has its own status word (in its workspace).  Once a kernel of the call has
// recorded an error, the call's later kernels skip their work: their inputs (counts, slot
// words, lists) may be incomplete.  The call's last kernel copies the word into the
// device's status word, which rip_get_device_status returns.
__device__ __forceinline__ bool call_failed(const Status* st) {
    return *reinterpret_cast<const volatile uint32_t*>(&st->code) != 0u;
}

// The same verdict for every thread of the block (read once by thread 0); call it from every
// thread at the start of a kernel.
__device__ __forceinline__ bool block_call_failed(const Status* st) {
    __shared__ uint32_t failed;
    if (threadIdx.x == 0) failed = call_failed(st) ? 1u : 0u;
    __syncthreads();
    const bool r = failed != 0u;
    __syncthreads();
    return r;
}

// ----------------------------------------------------------------- Philox

struct PhiloxKey {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               PhiloxKey key) {
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;  // one wide multiply gives hi and lo
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Philox with the ten round keys computed once (they depend on the seed only).
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
    __device__ __forceinline__ void init(PhiloxKey key) {
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            k0[r] = key.k0 + (uint32_t)r * 0x9E3779B9u;
            k1[r] = key.k1 + (uint32_t)r * 0xBB67AE85u;
        }
    }
};

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys& ks) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ ks.k0[r];
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ ks.k1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ PhiloxKey make_key(uint64_t seed) {
    return PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
}

__device__ __forceinline__ uint32_t pick(uint4 r, uint32_t w) {
    return w == 0 ? r.x : (w == 1 ? r.y : (w == 2 ? r.z : r.w));
}

// Scatter word of 32 consecutive logical positions P0 .. P0+31 (lane l gets
// position P0 + l).  Only the <= 9 Philox calls the warp needs are evaluated;
// must be called by all 32 lanes.
__device__ __forceinline__ uint32_t warp_scatter_word(PhiloxKey key, uint32_t level, uint64_t o,
                                                      uint64_t P0) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t q0 = P0 >> 2;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (lane < 9u) {
        const uint64_t q = q0 + lane;
        r = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), level | (kTagScatter << 8), (uint32_t)o, key);
    }
    const uint64_t p = P0 + lane;
    const int src = (int)((p >> 2) - q0);
    const uint32_t w0 = __shfl_sync(0xffffffffu, r.x, src);
    const uint32_t w1 = __shfl_sync(0xffffffffu, r.y, src);
    const uint32_t w2 = __shfl_sync(0xffffffffu, r.z, src);
    const uint32_t w3 = __shfl_sync(0xffffffffu, r.w, src);
    const uint32_t sel = (uint32_t)(p & 3u);
    return sel == 0 ? w0 : (sel == 1 ? w1 : (sel == 2 ? w2 : w3));
}

// Groups of 128 consecutive positions starting at a multiple of four: lane l
// of the warp evaluates the Philox call of positions 4(Qg + l) .. 4(Qg + l) + 3,
// all 32 lanes busy.  Step s (0..3) of the group covers positions
// 4 Qg + 32 s + lane; group_step_word hands each lane the word of its position.
__device__ __forceinline__ uint4 group_philox(PhiloxKey key, uint32_t level, uint64_t o, uint64_t Qg) {
    const uint64_t q = Qg + (threadIdx.x & 31u);
    return philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), level | (kTagScatter << 8), (uint32_t)o, key);
}

__device__ __forceinline__ uint4 group_philox(const PhiloxKeys& ks, uint32_t level, uint64_t o, uint64_t Qg) {
    const uint64_t q = Qg + (threadIdx.x & 31u);
    return philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), level | (kTagScatter << 8), (uint32_t)o, ks);
}

__device__ __forceinline__ uint32_t group_step_word(const uint4& r, uint32_t s) {
    const uint32_t lane = threadIdx.x & 31u;
    const int src = (int)(8u * s + (lane >> 2));
    const uint32_t w0 = __shfl_sync(0xffffffffu, r.x, src);
    const uint32_t w1 = __shfl_sync(0xffffffffu, r.y, src);
    const uint32_t w2 = __shfl_sync(0xffffffffu, r.z, src);
    const uint32_t w3 = __shfl_sync(0xffffffffu, r.w, src);
    const uint32_t sel = lane & 3u;
    return sel == 0 ? w0 : (sel == 1 ? w1 : (sel == 2 ? w2 : w3));
}

__device__ __forceinline__ uint32_t bucket_of(uint32_t word, uint32_t k) { return __umulhi(word, k); }

// Lanes of the warp holding the same bucket as the calling lane (among lanes
// with `valid`), from one ballot per bucket bit: cheaper than match.any when
// most of the 32 buckets differ.  bits = log2 k <= 10; all lanes must call.
__device__ __forceinline__ uint32_t warp_peers(uint32_t b, uint32_t bits, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (uint32_t i = 0; i < 10; ++i) {
        if (i < bits) {
            const uint32_t bit = (b >> i) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
    }
    return peers;
}

__host__ __device__ __forceinline__ uint32_t log2_pow2(uint32_t k) {
    uint32_t l = 0;
    while ((1u << l) < k) ++l;
    return l;
}

// Lemire acceptance for s in [1, 2^32]: returns true and sets v on accept.
__device__ __forceinline__ bool lemire_accept(uint32_t x, uint64_t s, uint64_t& v) {
    const uint64_t m = (uint64_t)x * s;
    const uint64_t lo = m & 0xffffffffull;
    if (lo < s) {
        const uint64_t t = ((1ull << 32) - s) % s;
        if (lo < t) return false;
    }
    v = m >> 32;
    return true;
}

// Retry path of a Fisher-Yates draw (the first word was rejected).
static __device__ __noinline__ uint64_t fy_draw_retry(PhiloxKey key, uint32_t level, uint64_t o, uint64_t p,
                                               uint64_t s) {
    for (uint32_t a = 1; a < 65536u; ++a) {
        const uint4 r = philox4x32_10((uint32_t)p, (uint32_t)(p >> 32),
                                      level | (kTagFyRetry << 8) | (a << 16), (uint32_t)o, key);
        uint64_t v;
        if (lemire_accept(r.x, s, v)) return v;
        if (lemire_accept(r.y, s, v)) return v;
        if (lemire_accept(r.z, s, v)) return v;
        if (lemire_accept(r.w, s, v)) return v;
    }
    return 0;
}

// Sequential Fisher-Yates draw stream for one leaf, steps i = len-1 down to 1;
// caches the shared Philox call of the current group of four positions.
struct FyStream {
    PhiloxKey key;
    uint32_t level;
    uint64_t o;       // leaf start (logical global position of step 0)
    uint64_t cached_q;
    uint4 cached;

    __device__ __forceinline__ void init(PhiloxKey k, uint32_t L, uint64_t leaf_o) {
        key = k;
        level = L;
        o = leaf_o;
        cached_q = ~0ull;
    }
    __device__ __forceinline__ uint64_t draw(uint64_t i) {
        const uint64_t p = o + i;
        const uint64_t q = p >> 2;
        if (q != cached_q) {
            cached = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), level | (kTagFy << 8), (uint32_t)o, key);
            cached_q = q;
        }
        uint64_t v;
        if (lemire_accept(pick(cached, (uint32_t)(p & 3u)), i + 1, v)) return v;
        return fy_draw_retry(key, level, o, p, i + 1);
    }
};

// ----------------------------------------------------------------- division by invariants

// Unsigned 32-bit division by a run-time constant d >= 1 with one multiply-high
// and shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l,1))) >> max(l-1,0)
// with t = mulhi(m, n); exact for every n < 2^32.
struct FastDiv {
    uint32_t d, m, s1, s2;
    __host__ __device__ static FastDiv make(uint32_t div) {
        FastDiv f;
        f.d = div;
        uint32_t l = 0;
        while (l < 32 && (1ull << l) < div) ++l;
        f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
        f.s1 = l < 1 ? l : 1;
        f.s2 = l > 0 ? l - 1 : 0;
        return f;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        const uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
    __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

// ----------------------------------------------------------------- plan / descriptors

struct DevPlan {
    uint32_t num_levels;
    uint32_t cap;  // effective level cap (max_levels, or kDepthCap when 0)
    uint64_t base;
    uint32_t k[RIP_MAX_LEVEL_PARAMS];
    uint32_t B[RIP_MAX_LEVEL_PARAMS];
    uint64_t T[RIP_MAX_LEVEL_PARAMS];

    __device__ __host__ __forceinline__ uint32_t idx(uint32_t L) const {
        return L < num_levels ? L : num_levels - 1;
    }
    __device__ __host__ __forceinline__ bool is_leaf(uint64_t m, uint32_t L) const {
        return m <= base || L >= cap;
    }
};

struct ArrayDesc {
    char* data;          // device pointer of the array
    uint64_t n;          // elements
    uint64_t seed;       // Philox key of this array
};

// A subproblem: elements [o, o+m) of array `arr` (o is both the logical start
// used by the draws and the start of its physical region).  Logical index i
// lives at physical o + ((i + eps) mod m).
struct Sub {
    uint64_t o;
    uint64_t m;
    uint32_t arr;
    uint32_t level;
    uint32_t eps;
    uint32_t pad;
};

__device__ __forceinline__ uint64_t phys_index(const Sub& s, uint64_t i) {
    uint64_t j = i + s.eps;
    if (j >= s.m) j -= s.m;
    return s.o + j;
}

// ----------------------------------------------------------------- mbarriers and bulk copies

constexpr uint32_t kMbarPolls = 1u << 20;     // mbarrier polls before a wait gives up
constexpr uint32_t kMbarSuspendNs = 4000;     // each poll sleeps up to this long (about 4 s in all)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the phase with the given parity: one non-blocking test, then up to
// polls - 1 tries, each of which suspends the thread until the phase completes or
// kMbarSuspendNs pass (a waiting warp then issues nothing, instead of spinning on issue slots
// the working warps need); false when the phase has not completed by then.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t polls = kMbarPolls) {
    const uint32_t a = smem_addr(bar);
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    for (uint32_t i = 1; i < polls; ++i) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(kMbarSuspendNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One bulk copy global -> shared, completing `bytes` transactions on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// One bulk copy shared -> global (the TMA engine reads the chunk; no per-lane stores).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the sources of this thread's bulk stores have been read (shared memory may be rewritten)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic shared-memory accesses before later async-proxy accesses (bulk
// copies) of the same bytes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ----------------------------------------------------------------- element types

template <int W> struct Elem;
template <> struct Elem<4> { using T = uint32_t; };
template <> struct Elem<8> { using T = uint64_t; };
template <> struct Elem<16> { using T = uint4; };

// ----------------------------------------------------------------- memory ordering

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
// `scratch` needs 32 words of shared memory.  Returns the exclusive prefix;
// *total receives the block sum.
template <typename U>
__device__ __forceinline__ U block_exclusive_scan(U v, U* scratch, U* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwarps = (blockDim.x + 31u) >> 5;
    U x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        U y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31u) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        U w = lane < nwarps ? scratch[lane] : U(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            U y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= (uint32_t)d) w += y;
        }
        if (lane < nwarps) scratch[lane] = w;
    }
    __syncthreads();
    const U warp_prefix = warp ? scratch[warp - 1] : U(0);
    if (total) *total = scratch[nwarps - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

}  // namespace rip
