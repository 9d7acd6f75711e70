// rip_small.cu -- finishes whole subproblems that fit on one SM.
//
// A subproblem of m <= 48K elements is loaded once (through its rotation),
// its complete remaining recursion -- scatter levels (Sec. 2.2 ScatterShuffle,
// Sec. 3.2 recursion) down to Fisher-Yates leaves (Sec. 2.2, Fig. 1) -- runs
// on 16-bit index arrays in shared memory, and the result is written back in
// canonical (unrotated) order with one coalesced pass.  HBM traffic: one read
// and one write of the subproblem, whatever the number of levels inside.
//
// Shared memory: [fixed scratch | P0 (2m) | P1 (2m) | D (w*m + 16)].  D is
// filled by bulk (TMA) copies issued when the subproblem starts and completing
// on an mbarrier, so the load overlaps the whole index computation (which needs
// no data); D is shifted by up to 15 bytes so that the copy of the larger
// rotation piece starts 16-byte aligned on both sides, and the ragged rest is
// copied by the threads.  In "medium" mode D lives in a per-CTA slice of global
// scratch instead (m up to 48K) and is loaded by the threads.
#include "rip_internal.cuh"

namespace rip {

namespace {

constexpr uint32_t kThreads = kSmallThreads;
constexpr uint32_t kWarps = kThreads / 32;

struct GeneralScratch {         // scatter of a range with several tiles or k > 256
    uint32_t thr[kSmallCntCap];  // per (tile, bucket): count, then B*floor(count/B)
    uint32_t fb[kSmallCntCap];   // per (tile, bucket): first full-block destination
    uint32_t tb[kSmallCntCap];   // per (tile, bucket): tail destination minus thr
    uint32_t run[kMaxK];         // per bucket: elements seen so far in the current tile
    uint32_t tbl[kSmallTbl / 2]; // per (ranking warp, bucket): running count in a round
};
struct FastScratch {               // single-tile scatter with k <= 256
    uint16_t hist[kWarps * 256];   // per (warp, bucket): count, then the warp's next output index
    uint32_t start[256];           // per bucket: total, then first output index of the bucket
    uint32_t mask[kWarps * 64];    // per (warp, low 6 bucket bits): lanes of the current step
};

struct SmallShared {
    union {
        GeneralScratch g;
        FastScratch f;
    };
    uint64_t stack[kSmallStack]; // pending scatter ranges
    uint32_t scan[32];
    uint64_t load_bar;           // bulk copy of the subproblem's data into D
    uint32_t stack_top;
    uint32_t cur_hi, cur_lo;
    uint32_t flag;
};

__device__ __forceinline__ uint64_t pack_range(uint32_t a, uint32_t len, uint32_t L, uint32_t buf) {
    return (uint64_t)a | ((uint64_t)len << 20) | ((uint64_t)L << 40) | ((uint64_t)buf << 48);
}

// Lemire acceptance for s < 2^32 in 32-bit arithmetic (same decisions as lemire_accept).
__device__ __forceinline__ bool lemire32(uint32_t x, uint32_t s, uint32_t& v) {
    const uint64_t m = (uint64_t)x * s;
    const uint32_t lo = (uint32_t)m;
    if (lo < s && lo < (0u - s) % s) return false;
    v = (uint32_t)(m >> 32);
    return true;
}

// Partner draws H[i] (i >= 1) of a leaf, computed by the whole block.
__device__ void fy_draws(uint16_t* H, uint32_t len, PhiloxKey key, uint32_t L, uint64_t leaf_o) {
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        if (i == 0) continue;
        const uint64_t p = leaf_o + i;
        const uint64_t q = p >> 2;
        const uint4 r = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), L | (kTagFy << 8), (uint32_t)leaf_o, key);
        uint64_t v;
        if (!lemire_accept(pick(r, (uint32_t)(p & 3u)), i + 1, v)) v = fy_draw_retry(key, L, leaf_o, p, i + 1);
        H[i] = (uint16_t)v;
    }
    __syncthreads();
}

// 16-bit atomic maximum on shared memory, by compare-and-swap on the containing word.
__device__ __forceinline__ void atomic_max_u16(uint16_t* addr, uint32_t val) {
    uint32_t* word = reinterpret_cast<uint32_t*>(reinterpret_cast<uintptr_t>(addr) & ~uintptr_t(3));
    const uint32_t shift = (reinterpret_cast<uintptr_t>(addr) & 2u) ? 16u : 0u;
    uint32_t old = *word;
    for (;;) {
        if (((old >> shift) & 0xFFFFu) >= val) return;
        const uint32_t nv = (old & ~(0xFFFFu << shift)) | (val << shift);
        const uint32_t prev = atomicCAS(word, old, nv);
        if (prev == old) return;
        old = prev;
    }
}

__device__ __forceinline__ void atomic_max_r(uint16_t* addr, uint32_t val) { atomic_max_u16(addr, val); }
__device__ __forceinline__ void atomic_max_r(uint32_t* addr, uint32_t val) { atomicMax(addr, val); }

// Fisher-Yates of a leaf of up to 2^15 elements on the elements themselves, by deterministic
// reservations (Shun, Gu, Blelloch, Fineman, Gibbons, SODA 2015): every round commits each
// unfinished step that is the latest of all unfinished steps touching either of its two
// positions, which gives the sequential order's result.  Partner draws in H, reservations in R (16- or 32-bit); thread
// t owns steps t + j*blockDim and keeps the unfinished ones in a 64-bit mask, so a round
// touches only unfinished steps.
template <typename T, typename RT>
__device__ void fy_parallel_data(T* D, const uint16_t* H, RT* R, uint32_t len, Status* status) {
    __shared__ uint32_t remaining;
    const uint32_t nb = blockDim.x, tid = threadIdx.x;
    uint64_t mine = 0;
    for (uint32_t j = 0; j < 64u && tid + j * nb < len; ++j)
        if (tid + j * nb >= 1u) mine |= 1ull << j;  // step 0 does nothing
    for (uint32_t i = tid; i < len; i += nb) R[i] = 0;
    for (uint32_t round = 0;; ++round) {
        __syncthreads();
        if (tid == 0) remaining = 0;
        for (uint64_t mk = mine; mk; mk &= mk - 1) {
            const uint32_t i = tid + (uint32_t)(__ffsll((long long)mk) - 1) * nb;
            const uint32_t h = H[i];
            atomic_max_r(&R[i], i);
            atomic_max_r(&R[h], i);
        }
        __syncthreads();
        uint64_t left = 0;
        for (uint64_t mk = mine; mk; mk &= mk - 1) {
            const uint32_t j = (uint32_t)(__ffsll((long long)mk) - 1);
            const uint32_t i = tid + j * nb;
            const uint32_t h = H[i];
            if (R[i] == i && R[h] == i) {
                const T di = D[i];
                D[i] = D[h];
                D[h] = di;
            } else {
                left |= 1ull << j;
            }
        }
        if (left) remaining = 1;
        __syncthreads();
        const bool again = remaining != 0;
        for (uint64_t mk = mine; mk; mk &= mk - 1) {  // clear what this round reserved
            const uint32_t i = tid + (uint32_t)(__ffsll((long long)mk) - 1) * nb;
            R[i] = 0;
            R[H[i]] = 0;
        }
        mine = left;
        if (!again) break;
        if (round > 4 * len) {  // cannot happen: the latest unfinished step always commits
            if (tid == 0) report(status, RIP_EINTERNAL, 0x5108, len);
            break;
        }
    }
    __syncthreads();
}

// The same rounds with 32-bit reservations stamped by the round (round << 16 | step): an entry of
// an earlier round loses every comparison, so nothing is cleared between rounds.  Z is the data
// itself, or 16-bit indices whose final order a gather applies to the data afterwards.
template <typename T>
__device__ void fy_parallel_stamped(T* Z, const uint16_t* H, uint32_t* R, uint32_t len, Status* status) {
    __shared__ uint32_t remaining;
    const uint32_t nb = blockDim.x, tid = threadIdx.x;
    uint64_t mine = 0;
    for (uint32_t j = 0; j < 64u && tid + j * nb < len; ++j)
        if (tid + j * nb >= 1u) mine |= 1ull << j;  // step 0 does nothing
    for (uint32_t i = tid; i < len; i += nb) R[i] = 0;
    for (uint32_t round = 1;; ++round) {
        __syncthreads();
        if (tid == 0) remaining = 0;
        for (uint64_t mk = mine; mk; mk &= mk - 1) {
            const uint32_t i = tid + (uint32_t)(__ffsll((long long)mk) - 1) * nb;
            const uint32_t tag = (round << 16) | i;
            atomicMax(&R[i], tag);
            atomicMax(&R[H[i]], tag);
        }
        __syncthreads();
        uint64_t left = 0;
        for (uint64_t mk = mine; mk; mk &= mk - 1) {
            const uint32_t j = (uint32_t)(__ffsll((long long)mk) - 1);
            const uint32_t i = tid + j * nb;
            const uint32_t h = H[i];
            const uint32_t tag = (round << 16) | i;
            if (R[i] == tag && R[h] == tag) {
                const T zi = Z[i];
                Z[i] = Z[h];
                Z[h] = zi;
            } else {
                left |= 1ull << j;
            }
        }
        if (left) remaining = 1;
        __syncthreads();
        const bool again = remaining != 0;
        mine = left;
        if (!again) break;
        if (round >= 0xFFFFu) {  // cannot happen: the latest unfinished step always commits
            if (tid == 0) report(status, RIP_EINTERNAL, 0x510A, len);
            break;
        }
    }
    __syncthreads();
}

__device__ void fy_block(uint16_t* Z, uint16_t* draws, uint32_t len, PhiloxKey key, uint32_t L,
                         uint64_t leaf_o) {
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        if (i == 0) continue;
        const uint64_t p = leaf_o + i;
        const uint64_t q = p >> 2;
        const uint4 r = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), L | (kTagFy << 8), (uint32_t)leaf_o, key);
        uint64_t v;
        if (!lemire_accept(pick(r, (uint32_t)(p & 3u)), i + 1, v)) v = fy_draw_retry(key, L, leaf_o, p, i + 1);
        draws[i] = (uint16_t)v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (uint32_t i = len - 1; i >= 1; --i) {
            const uint32_t j = draws[i];
            const uint16_t zi = Z[i];
            Z[i] = Z[j];
            Z[j] = zi;
        }
    }
    __syncthreads();
}

// Partner draw of step i from word x when the multiply's low word fell below i + 1 (probability
// below 2^-16 here): Lemire's exact rejection test, then the retry stream.  Kept out of line so
// the common path stays short.
__device__ __noinline__ uint32_t fy_draw_slow(uint32_t x, uint32_t i, PhiloxKey key, uint32_t L, uint64_t leaf_o) {
    uint32_t v;
    if (lemire32(x, i + 1, v)) return v;
    return (uint32_t)fy_draw_retry(key, L, leaf_o, leaf_o + i, i + 1);
}

// The four partner draws of one Philox call whose first word belongs to step i0 (steps outside
// [1, len) are skipped); stored in H[step].
__device__ __forceinline__ void fy_store_group(uint16_t* H, uint4 r, int32_t i0, uint32_t len, PhiloxKey key,
                                               uint32_t L, uint64_t leaf_o) {
    const uint32_t w4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (uint32_t wd = 0; wd < 4; ++wd) {
        const int32_t si = i0 + (int32_t)wd;
        if (si < 1 || si >= (int32_t)len) continue;
        const uint32_t i = (uint32_t)si;
        const uint64_t mw = (uint64_t)w4[wd] * (i + 1u);
        const uint32_t v = (uint32_t)mw < i + 1u ? fy_draw_slow(w4[wd], i, key, L, leaf_o) : (uint32_t)(mw >> 32);
        H[i] = (uint16_t)v;
    }
}

// Partner draws of one leaf child, by `step` threads together: the calling thread takes the
// groups of four positions sub, sub + step, ...; two Philox calls are in flight at a time.
__device__ __forceinline__ void fy_draws_part(uint16_t* H, uint32_t len, PhiloxKey key, uint32_t L, uint64_t leaf_o,
                                              uint32_t sub, uint32_t step) {
    const uint64_t q_first = (leaf_o + 1) >> 2, q_last = (leaf_o + len - 1) >> 2;
    const uint32_t ng = (uint32_t)(q_last - q_first) + 1u;
    const int32_t i_first = (int32_t)(4 * q_first - leaf_o);  // step of the first group's word 0 (-2 .. 1)
    const uint32_t tag = L | (kTagFy << 8), o32 = (uint32_t)leaf_o;
    for (uint32_t g = sub; g < ng; g += 2u * step) {
        const uint64_t q = q_first + g, q2 = q + step;  // q2 may lie past the leaf: computed, not stored
        const uint4 r = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), tag, o32, key);
        const uint4 r2 = philox4x32_10((uint32_t)q2, (uint32_t)(q2 >> 32), tag, o32, key);
        fy_store_group(H, r, i_first + 4 * (int32_t)g, len, key, L, leaf_o);
        if (g + step < ng) fy_store_group(H, r2, i_first + 4 * (int32_t)(g + step), len, key, L, leaf_o);
    }
}

// Partner draws of the leaf children of a scattered range, by every thread (tpc = blockDim/k
// threads per child), into the range's source array X (not read any more, or never read).
// start(b) = first output index of bucket b.
template <typename StartFn>
__device__ void children_draws(uint16_t* X, uint32_t a, uint32_t len, uint32_t k, uint32_t L, const DevPlan& plan,
                               PhiloxKey key, uint64_t o_r, StartFn start) {
    const uint32_t tpc = k >= blockDim.x ? 1u : blockDim.x / k;
    for (uint32_t b = threadIdx.x / tpc; b < k; b += blockDim.x / tpc) {
        const uint32_t sb = start(b);
        const uint32_t se = b + 1 < k ? start(b + 1) : len;
        if (se > len || sb >= se) continue;
        const uint32_t size = se - sb;
        if (size > 1 && plan.is_leaf(size, L + 1))
            fy_draws_part(X + a + sb, size, key, L + 1, o_r + sb, threadIdx.x % tpc, tpc);
    }
}

// Children of a scattered range: leaves are finished right away, larger ones are pushed for
// another scatter.  start(b) = first output index of bucket b; draws_done: children_draws
// already ran (and a barrier followed).
template <typename StartFn>
__device__ void finish_children(SmallShared& sh, uint16_t* P0, uint16_t* X, uint16_t* Y, uint32_t a, uint32_t len,
                                uint32_t k, uint32_t L, uint32_t buf, const DevPlan& plan, PhiloxKey key,
                                uint64_t o_r, Status* status, bool draws_done, StartFn start) {
    // leaf children: partner draws first (the scatter's source range is free now and holds
    // them), then one thread per child runs the child's swap chain (consecutive threads: full
    // warps measured faster than chains spread over all warps)
    if (!draws_done) {
        children_draws(X, a, len, k, L, plan, key, o_r, start);
        __syncthreads();
    }
    for (uint32_t b = threadIdx.x; b < k; b += blockDim.x) {
        const uint32_t sb = start(b);
        const uint32_t se = b + 1 < k ? start(b + 1) : len;
        const uint32_t size = se - sb;
        if (size == 0) continue;
        if (se > len || sb > se) {
            report(status, RIP_EINTERNAL, 0x5104, se);
            continue;
        }
        if (size == 1 || plan.is_leaf(size, L + 1)) {
            uint16_t* Z = Y + a + sb;
            const uint16_t* H = X + a + sb;
            // The lanes of a warp run their chains staggered: a lane idles its first d steps, d
            // chosen so that at every step the lanes' positions i have distinct 16-bit indices
            // modulo 32, i.e. distinct shared-memory banks for H[i], Z[i] and out[i] (the chains
            // start at random offsets and otherwise collide; measured as most of the solver's
            // bank conflicts).  Each chain still takes its steps in order.
            const uint32_t d = ((threadIdx.x & 31u) - (a + sb + size - 1u)) & 31u;
            if (Y != P0) {
                // the swap chain writes each final position straight to P0: step i fixes
                // position i (later steps touch only positions below i), so only Z[j] is
                // written back; out may coincide with H, whose entry i is read before
                uint16_t* out = P0 + a + sb;
                uint32_t j = size > 1 ? H[size - 1] : 0u;
                if (size > 1) {
                    for (uint32_t i = size - 1 + d; i >= 1; --i) {
                        if (i >= size) continue;  // not started
                        const uint32_t jn = i > 1 ? H[i - 1] : 0u;  // entry i-1 is not written at step i
                        const uint16_t zj = Z[j];
                        const uint16_t zi = Z[i];
                        out[i] = zj;
                        Z[j] = zi;
                        j = jn;
                    }
                }
                out[0] = Z[0];
            } else if (size > 1) {
                for (uint32_t i = size - 1 + d; i >= 1; --i) {
                    if (i >= size) continue;  // not started
                    const uint32_t j = H[i];
                    const uint16_t zi = Z[i];
                    Z[i] = Z[j];
                    Z[j] = zi;
                }
            }
        } else {
            const uint32_t slot = atomicAdd(&sh.stack_top, 1u);
            if (slot < kSmallStack)
                sh.stack[slot] = pack_range(a + sb, size, L + 1, buf ^ 1u);
            else
                report(status, RIP_EINTERNAL, 0x5102, slot);
        }
    }
    __syncthreads();
}

// Scatter of a range that is a single tile with k <= 256: a stable partition
// by bucket.  Warp w owns a contiguous run of 128-position groups (aligned to
// multiples of four in the global position space).  Pass 1: each lane draws
// the four buckets of one Philox call per group (kept packed in registers) and
// counts them in the warp's histogram row.  Prefix: rows become the first
// output index of (warp, bucket).  Pass 2: the warp walks its run in position
// order, 32 positions per step; the lanes of the step with the same bucket
// (the rank inside the step) come from a shared-memory mask row indexed by the
// low six bucket bits (one atomic OR per lane) and one ballot per higher bit
// -- on GB300 a ballot costs more issue time than a shared atomic -- and the
// lowest of them advances the warp's row (only the warp itself touches it).
// Groups per warp of the single-tile scatter (its buckets stay in registers): enough for the
// largest subproblem that fits in shared memory with w-byte elements (16 warps x G x 128
// positions); larger ranges take the general path.
__host__ __device__ constexpr uint32_t fast_groups(int W) { return W == 4 ? 16u : (W == 8 ? 12u : 8u); }

template <uint32_t G>
__device__ bool scatter_range_fast(SmallShared& sh, uint16_t* P0, uint16_t* P1, uint32_t a, uint32_t len, uint32_t L,
                                   uint32_t buf, const DevPlan& plan, PhiloxKey key, uint64_t sub_o, bool x_iota,
                                   Status* status) {
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t k = plan.k[plan.idx(L)];
    const uint32_t kbits = log2_pow2(k);
    uint16_t* X = buf ? P1 : P0;
    uint16_t* Y = buf ? P0 : P1;
    const uint64_t o_r = sub_o + a;
    const uint32_t delta = (uint32_t)(o_r & 3u);
    const uint64_t Q0 = o_r >> 2;
    const uint32_t ngroups = (len + delta + 127u) / 128u;
    const uint32_t gpw = (ngroups + kWarps - 1) / kWarps;  // groups per warp (<= G)
    const uint32_t g0 = warp * gpw;
    uint16_t* hist = sh.f.hist;
    uint32_t* hist32 = reinterpret_cast<uint32_t*>(hist);  // two 16-bit counters per word
    for (uint32_t j = tid; j < kWarps * 128u; j += blockDim.x) hist32[j] = 0;
    for (uint32_t j = tid; j < kWarps * 64u; j += blockDim.x) sh.f.mask[j] = 0;
    __syncthreads();

    uint32_t bk[G];  // 4 packed 8-bit buckets per group: lane l holds positions 4l .. 4l+3
#pragma unroll
    for (uint32_t g = 0; g < G; ++g) {
        bk[g] = 0;
        if (g < gpw && g0 + g < ngroups) {
            const uint32_t vg = (g0 + g) * 128u;
            const uint4 r = group_philox(key, L, o_r, Q0 + vg / 4u);
            const uint32_t v0 = vg + 4u * lane;
            const uint32_t w4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                const uint32_t b = bucket_of(w4[j], k);
                bk[g] |= b << (8 * j);
                const uint32_t v = v0 + j;
                if (v >= delta && v - delta < len) atomicAdd(&hist32[warp * 128u + (b >> 1)], 1u << (16u * (b & 1u)));
            }
        }
    }
    __syncthreads();
    // rows -> first output index of (warp, bucket)
    for (uint32_t b = tid; b < k; b += blockDim.x) {
        uint32_t acc = 0;
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t c = hist[w * 256u + b];  // each 16-bit counter has one owner here
            hist[w * 256u + b] = (uint16_t)acc;
            acc += c;
        }
        sh.f.start[b] = acc;  // bucket total
    }
    __syncthreads();
    {
        const uint32_t i0 = 2 * tid, i1 = 2 * tid + 1;
        const uint32_t v0 = i0 < k ? sh.f.start[i0] : 0, v1 = i1 < k ? sh.f.start[i1] : 0;
        const uint32_t ex = block_exclusive_scan<uint32_t>(v0 + v1, sh.scan, nullptr);
        if (i0 < k) sh.f.start[i0] = ex;
        if (i1 < k) sh.f.start[i1] = ex + v0;
    }
    __syncthreads();
    for (uint32_t j = tid; j < kWarps * 256u; j += blockDim.x)
        if ((j & 255u) < k) hist[j] = (uint16_t)(hist[j] + sh.f.start[j & 255u]);
    __syncthreads();

    // X holds the identity and is not read: the children's partner draws go there now, so
    // the Philox-heavy draws and the shared-memory-heavy ranking below overlap across warps
    if (x_iota) children_draws(X, a, len, k, L, plan, key, o_r, [&](uint32_t b) { return sh.f.start[b]; });
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint16_t* row = hist + warp * 256u;
    uint32_t* mrow = sh.f.mask + warp * 64u;
#pragma unroll
    for (uint32_t g = 0; g < G; ++g) {
        if (g < gpw && g0 + g < ngroups) {
            const uint32_t vg = (g0 + g) * 128u;
#pragma unroll
            for (uint32_t st = 0; st < 4; ++st) {
                const uint32_t packed = __shfl_sync(0xffffffffu, bk[g], (int)(8u * st + (lane >> 2)));
                const uint32_t b = (packed >> (8u * (lane & 3u))) & 0xFFu;
                const uint32_t v = vg + 32u * st + lane;
                const bool valid = v >= delta && v - delta < len;
                if (valid) atomicOr(&mrow[b & 63u], 1u << lane);
                uint32_t peers = 0xffffffffu;
#pragma unroll
                for (uint32_t i = 6; i < 8; ++i) {
                    if (i < kbits) {
                        const uint32_t bit = (b >> i) & 1u;
                        const uint32_t m = __ballot_sync(0xffffffffu, bit);
                        peers &= bit ? m : ~m;
                    }
                }
                __syncwarp();
                peers &= valid ? mrow[b & 63u] : 0u;
                // the step's lanes with this bucket read the row together; the lowest writes it
                // back and clears the mask entry (a 16-bit store: the neighbour counter is untouched)
                const uint32_t base = valid ? (uint32_t)row[b] : 0u;
                __syncwarp();
                if (valid && (peers & lt_mask) == 0) {
                    row[b] = (uint16_t)(base + (uint32_t)__popc(peers));
                    mrow[b & 63u] = 0u;
                }
                __syncwarp();
                if (valid) {
                    const uint32_t d = base + __popc(peers & lt_mask);
                    if (d < len) Y[a + d] = x_iota ? (uint16_t)(a + (v - delta)) : X[a + (v - delta)];
                    else report(status, RIP_EINTERNAL, 0x5105, d);
                }
            }
        }
    }
    __syncthreads();
    finish_children(sh, P0, X, Y, a, len, k, L, buf, plan, key, o_r, status, x_iota,
                    [&](uint32_t b) { return sh.f.start[b]; });
    return true;
}

// One scatter level of the range [a, a+len) (level L) from X into Y, both
// index arrays; children ranges are finished (leaves) or pushed.  x_iota: X
// holds the identity there (the subproblem's first level; X is not read).
template <uint32_t G>
__device__ void scatter_range(SmallShared& sh, uint16_t* P0, uint16_t* P1, uint32_t a, uint32_t len,
                              uint32_t L, uint32_t buf, const DevPlan& plan, PhiloxKey key,
                              uint64_t sub_o, bool x_iota, Status* status) {
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t li = plan.idx(L);
    const uint32_t k = plan.k[li], B = plan.B[li];
    const uint64_t T64 = plan.T[li];
    const uint32_t T = T64 >= len ? len : (uint32_t)T64;
    const uint32_t tiles = (len + T - 1) / T;
    const FastDiv fdT = FastDiv::make(T), fdB = FastDiv::make(B);
    const uint32_t kbits = log2_pow2(k);
    const uint32_t ncnt = tiles * k;
    uint16_t* X = buf ? P1 : P0;
    uint16_t* Y = buf ? P0 : P1;
    const uint64_t o_r = sub_o + a;  // logical global start of this range

    if (ncnt > kSmallCntCap || k > kMaxK) {  // excluded by the host's eligibility rule
        if (tid == 0) report(status, RIP_EINTERNAL, 0x5101, ncnt);
        return;
    }
    if (tiles == 1 && k <= 256 && (len + 3u + 127u) / 128u <= kWarps * G) {
        scatter_range_fast<G>(sh, P0, P1, a, len, L, buf, plan, key, sub_o, x_iota, status);
        return;
    }
    for (uint32_t j = tid; j < ncnt; j += blockDim.x) sh.g.thr[j] = 0;
    __syncthreads();

    // counts per (tile, bucket); groups of 128 positions aligned to multiples of four
    {
        const uint32_t delta = (uint32_t)(o_r & 3u);
        const uint64_t Q0 = o_r >> 2;
        const uint32_t vlen = len + delta;
        for (uint32_t gb = warp * 128u; gb < vlen; gb += kWarps * 128u) {
            const uint4 rr = group_philox(key, L, o_r, Q0 + gb / 4u);
#pragma unroll
            for (uint32_t st = 0; st < 4; ++st) {
                const uint32_t v = gb + 32u * st + lane;
                const bool valid = v >= delta && v - delta < len;
                const uint32_t b = bucket_of(group_step_word(rr, st), k);
                const uint32_t key2 = valid ? (tiles == 1 ? 0u : fdT.div(v - delta)) * k + b : 0u;
                if (valid) atomicAdd(&sh.g.thr[key2], 1u);  // counts only: order does not matter
            }
        }
    }
    __syncthreads();

    // bucket sizes -> region starts s_b (exclusive scan over b)
    for (uint32_t b = tid; b < k; b += blockDim.x) {
        uint32_t size = 0;
        for (uint32_t t = 0; t < tiles; ++t) size += sh.g.thr[t * k + b];
        sh.g.run[b] = size;
    }
    __syncthreads();
    {
        // k <= kMaxK = 1024 = 2 * kThreads: two entries per thread
        const uint32_t i0 = 2 * tid, i1 = 2 * tid + 1;
        const uint32_t v0 = i0 < k ? sh.g.run[i0] : 0, v1 = i1 < k ? sh.g.run[i1] : 0;
        const uint32_t ex = block_exclusive_scan<uint32_t>(v0 + v1, sh.scan, nullptr);
        if (i0 < k) sh.g.run[i0] = ex;
        if (i1 < k) sh.g.run[i1] = ex + v0;
    }
    __syncthreads();
    // per (tile, bucket): full-block and tail destinations of the canonical layout
    for (uint32_t b = tid; b < k; b += blockDim.x) {
        const uint32_t sb = sh.g.run[b];
        uint32_t Fb = 0;
        for (uint32_t t = 0; t < tiles; ++t) Fb += fdB.div(sh.g.thr[t * k + b]);
        uint32_t fsum = 0, rsum = 0;
        for (uint32_t t = 0; t < tiles; ++t) {
            const uint32_t c = sh.g.thr[t * k + b];
            const uint32_t f = fdB.div(c);
            const uint32_t th = f * B;
            sh.g.fb[t * k + b] = sb + B * fsum;
            sh.g.tb[t * k + b] = sb + B * Fb + rsum - th;
            sh.g.thr[t * k + b] = th;
            fsum += f;
            rsum += c - th;
        }
    }
    __syncthreads();

    // stable ranks inside each (tile, bucket), then the move X -> Y.  A round covers
    // nwr groups of 128 positions; tbl[w][b] counts bucket b in warp w's group, then
    // holds the element rank base (running count of the tile + earlier warps).
    const uint32_t nwr = min(kWarps, (uint32_t)(kSmallTbl / 2) / k);
    const uint32_t round = nwr * 128u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint32_t t = 0; t < tiles; ++t) {
        const uint32_t lo = t * T, hi = min(lo + T, len);
        const uint64_t P0 = o_r + lo;
        const uint32_t delta = (uint32_t)(P0 & 3u);
        const uint64_t Q0 = P0 >> 2;
        const uint32_t tl = hi - lo, vlen = tl + delta;
        for (uint32_t b = tid; b < k; b += blockDim.x) sh.g.run[b] = 0;
        for (uint32_t j = tid; j < nwr * k; j += blockDim.x) sh.g.tbl[j] = 0;
        __syncthreads();
        for (uint32_t R = 0; R < vlen; R += round) {
            uint32_t bb[4], pr[4];
            if (warp < nwr) {
                const uint4 rr = group_philox(key, L, o_r, Q0 + (R >> 2) + warp * 32u);
#pragma unroll
                for (uint32_t st = 0; st < 4; ++st) {
                    const uint32_t v = R + warp * 128u + 32u * st + lane;
                    const bool valid = v >= delta && v - delta < tl;
                    const uint32_t b = bucket_of(group_step_word(rr, st), k);
                    const uint32_t peers = warp_peers(b, kbits, valid);
                    const uint32_t leader = valid ? (uint32_t)(__ffs(peers) - 1) : lane;
                    uint32_t pre = 0;
                    if (valid && lane == leader) pre = atomicAdd(&sh.g.tbl[warp * k + b], (uint32_t)__popc(peers));
                    pre = __shfl_sync(0xffffffffu, pre, (int)leader);
                    bb[st] = valid ? b : 0xffffffffu;
                    pr[st] = pre + __popc(peers & lt_mask);
                }
            }
            __syncthreads();
            // rank bases: running count of the tile plus the counts of earlier warps
            for (uint32_t b = tid; b < k; b += blockDim.x) {
                uint32_t acc = sh.g.run[b];
                for (uint32_t w = 0; w < nwr; ++w) {
                    const uint32_t c = sh.g.tbl[w * k + b];
                    sh.g.tbl[w * k + b] = acc;
                    acc += c;
                }
                sh.g.run[b] = acc;
            }
            __syncthreads();
            if (warp < nwr) {
#pragma unroll
                for (uint32_t st = 0; st < 4; ++st) {
                    const uint32_t b = bb[st];
                    if (b == 0xffffffffu) continue;
                    const uint32_t rank = sh.g.tbl[warp * k + b] + pr[st];
                    const uint32_t ci = t * k + b;
                    const uint32_t d = rank < sh.g.thr[ci] ? sh.g.fb[ci] + rank : sh.g.tb[ci] + rank;
                    const uint32_t i = lo + (R + warp * 128u + 32u * st + lane - delta);
                    if (d >= len) {  // cannot happen for consistent counts; never write out of range
                        report(status, RIP_EINTERNAL, 0x5103, d);
                        continue;
                    }
                    Y[a + d] = x_iota ? (uint16_t)(a + i) : X[a + i];
                }
                __syncwarp();
                // each warp reads only its own row: clear it for the next round
                for (uint32_t b = lane; b < k; b += 32u) sh.g.tbl[warp * k + b] = 0;
                __syncwarp();
            }
        }
        __syncthreads();
    }

    // children: leaves now, larger ones onto the stack (tile 0 entry of fb = s_b)
    finish_children(sh, P0, X, Y, a, len, k, L, buf, plan, key, o_r, status, false,
                    [&](uint32_t b) { return sh.g.fb[b]; });
}

// Starts the bulk (TMA) loads of a subproblem's data into shared memory after P1, through its
// rotation, completing on load_bar; the threads copy the ragged rest.  Returns where the data go.
template <int W>
__device__ __forceinline__ typename Elem<W>::T* load_smem(const Sub& s, typename Elem<W>::T* base, uint32_t m,
                                                         uint16_t* P1, uint64_t* load_bar) {
    using T = typename Elem<W>::T;
    const uint32_t tid = threadIdx.x;
    T* D;
    // the rotation's pieces: logical [0, nA) from physical o+eps.., [nA, m) from o..; each
    // piece's 16-byte-aligned middle goes by bulk copy when its shared-memory start is
    // aligned too (the larger piece fixes D's shift), the rest by the threads
    const uint32_t q = W >= 16 ? 1u : 16u / W;  // elements per 16 bytes
    const uint32_t nA = m - s.eps;
    const uintptr_t gA = reinterpret_cast<uintptr_t>(base + s.o + s.eps);
    const uintptr_t gB = reinterpret_cast<uintptr_t>(base + s.o);
    auto first_aligned = [&](uint32_t L0, uint32_t L1, uintptr_t g) -> uint32_t {
        return min(L1, L0 + (uint32_t)(((16u - (g & 15u)) & 15u) / W));
    };
    const uint32_t fa = first_aligned(0u, nA, gA), fb = first_aligned(nA, m, gB);
    const uint32_t dshift = nA >= s.eps ? (q - fa % q) % q : (q - fb % q) % q;
    D = reinterpret_cast<T*>(P1 + ((m + 7u) & ~7u)) + dshift;
    auto bulk_range = [&](uint32_t L0, uint32_t L1, uintptr_t g, uint32_t f, uint32_t& lo, uint32_t& hi) {
        lo = hi = L0;
        const uint32_t e = f + (L1 - f) / q * q;
        if (e > f && ((g + (uintptr_t)(f - L0) * W) & 15u) == 0 && (dshift + f) % q == 0) {
            lo = f;
            hi = e;
        }
    };
    uint32_t aLo, aHi, bLo, bHi;
    bulk_range(0u, nA, gA, fa, aLo, aHi);
    bulk_range(nA, m, gB, fb, bLo, bHi);
    if (bLo == bHi) bLo = bHi = m;
    // issued by the first thread of the last warp, which takes no part in the write-back of the
    // previous subproblem: a bulk copy issued after the thread's own global stores waits for them
    if (tid == blockDim.x - 32u) {
        const uint32_t bytes = (aHi - aLo + bHi - bLo) * (uint32_t)W;
        if (bytes) {
            mbar_arrive_expect_tx(load_bar, bytes);
            auto issue = [&](uint32_t lo, uint32_t hi, uintptr_t g, uint32_t L0) {
                const char* src = reinterpret_cast<const char*>(g + (uintptr_t)(lo - L0) * W);
                char* dst = reinterpret_cast<char*>(D + lo);
                const uint32_t nbytes = (hi - lo) * (uint32_t)W;
                for (uint32_t off = 0; off < nbytes; off += 32768u)
                    bulk_g2s(dst + off, src + off, min(32768u, nbytes - off), load_bar);
            };
            if (aHi > aLo) issue(aLo, aHi, gA, 0u);
            if (bHi > bLo) issue(bLo, bHi, gB, nA);
        } else {
            mbar_arrive(load_bar);
        }
    }
    for (uint32_t i = tid; i < aLo; i += blockDim.x) D[i] = base[phys_index(s, i)];
    for (uint32_t i = aHi + tid; i < bLo; i += blockDim.x) D[i] = base[phys_index(s, i)];
    for (uint32_t i = bHi + tid; i < m; i += blockDim.x) D[i] = base[phys_index(s, i)];
    return D;
}

// Leaves handled by leaf_kernel: Fisher-Yates leaves in shared memory whose 32-bit reservations do
// not fit after the data but 8 bytes per element of indices, draws and reservations do.
__device__ __forceinline__ bool leaf_by_index(const SmallArgs& args, const Sub& s, uint32_t w) {
    const uint64_t m = s.m, mr = (m + 7u) & ~7ull;
    return !args.medium && m > 1 && m <= 64u * kThreads && args.plan.is_leaf(m, s.level) &&
           8 * mr + w * mr + 16 > args.dyn_bytes && 8 * mr <= args.dyn_bytes;
}

// A Fisher-Yates leaf whose 32-bit reservations do not fit beside its data (8- and 16-byte
// elements near the on-SM limit): the steps run on 16-bit indices (indices, draws and stamped
// reservations take 8 bytes per element), then the data are loaded into the space the draws and
// reservations held and written back gathered through the indices.  Run by leaf_kernel, not by
// small_kernel, whose register allocation any added path perturbs.  False when the load's wait
// expired (reported).
template <int W>
__device__ __forceinline__ bool fy_leaf_by_index(const SmallArgs& args, const Sub& s, typename Elem<W>::T* base,
                                              uint32_t m, PhiloxKey key, unsigned char* dyn, uint64_t* load_bar,
                                              uint32_t parity, uint32_t item) {
    using T = typename Elem<W>::T;
    const uint32_t tid = threadIdx.x;
    const uint64_t mr = (m + 7u) & ~7u;
    uint16_t* Z = reinterpret_cast<uint16_t*>(dyn);
    uint16_t* H = Z + mr;
    for (uint32_t i = tid; i < m; i += blockDim.x) Z[i] = (uint16_t)i;
    fy_draws(H, m, key, s.level, s.o);  // ends with a barrier
    fy_parallel_stamped(Z, H, reinterpret_cast<uint32_t*>(dyn + 4 * mr), m, args.status);
    fence_proxy_async_smem();  // the reservations' bytes become the bulk copy's destination
    __syncthreads();
    const T* D = load_smem<W>(s, base, m, H, load_bar);
    const bool ok = __syncthreads_and(mbar_wait(load_bar, parity)) != 0;
    if (!ok) {
        if (tid == 0) report(args.status, RIP_ETIMEOUT, 0x510B, item);
        return false;
    }
    for (uint32_t i0 = tid; i0 < m; i0 += 4u * blockDim.x) {  // four gathers in flight per thread
        uint32_t j[4];
        T v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            j[u] = i < m ? (uint32_t)Z[i] : 0u;
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
            if (j[u] < m) v[u] = D[j[u]];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i >= m) break;
            base[s.o + i] = v[u];
        }
    }
    fence_proxy_async_smem();  // these reads of D come before the next bulk copy into it
    __syncthreads();
    return true;
}

template <int W>
__global__ void __launch_bounds__(kThreads, 1) small_kernel(SmallArgs args) {
    using T = typename Elem<W>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
    unsigned char* dyn = smem_raw + ((sizeof(SmallShared) + 15) & ~size_t(15));
    if (block_call_failed(args.status)) return;  // an earlier kernel of the call failed
    const uint32_t count = min(*args.count, args.capacity);
    const uint32_t tid = threadIdx.x;
    const DevPlan& plan = args.plan;
    if (tid == 0) {
        mbar_init(&sh.load_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t loads = 0;  // completed phases of load_bar

    for (uint32_t item = blockIdx.x; item < count; item += gridDim.x) {
        const Sub s = args.list[item];
        const ArrayDesc ad = args.arrays[s.arr];
        T* base = reinterpret_cast<T*>(ad.data);
        const uint32_t m = (uint32_t)s.m;
        const PhiloxKey key = make_key(ad.seed);
        uint16_t* P0 = reinterpret_cast<uint16_t*>(dyn);
        uint16_t* P1 = P0 + ((m + 7u) & ~7u);
        if (leaf_by_index(args, s, W)) continue;  // leaf_kernel's
        T* D;
        bool bulk = false;  // D arrives through load_bar
        if (args.medium) {
            // load through the rotation, eight independent loads in flight per thread
            D = reinterpret_cast<T*>(args.gscratch + (uint64_t)blockIdx.x * args.gslot_bytes);
            for (uint32_t i0 = tid; i0 < m; i0 += 8u * blockDim.x) {
                T v[8];
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    if (i < m) v[j] = base[phys_index(s, i)];
                }
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    if (i < m) D[i] = v[j];
                }
            }
        } else {
            D = load_smem<W>(s, base, m, P1, &sh.load_bar);
            bulk = true;  // the phase completes either way
        }
        if (tid == 0) sh.stack_top = 0;
        __syncthreads();
        // D is complete (bulk copy arrived, the threads' parts behind the barrier above)
        auto wait_data = [&]() -> bool {
            if (!bulk) return true;
            bulk = false;
            const bool ok = __syncthreads_and(mbar_wait(&sh.load_bar, loads & 1u)) != 0;  // one verdict
            ++loads;
            if (!ok && tid == 0) report(args.status, RIP_ETIMEOUT, 0x5109, item);
            return ok;
        };

        bool in_place = false;  // D already holds the output order
        if (plan.is_leaf(m, s.level)) {
            if (m > 1 && m <= 64u * kThreads) {
                fy_draws(P1, m, key, s.level, s.o);
                if (!wait_data()) break;
                // 32-bit reservations after D when they fit, else 16-bit ones in P0's place
                const uint64_t mr = (m + 7u) & ~7u;
                const uint64_t r32_off = 4 * mr + (args.medium ? 0 : (uint64_t)W * mr + 16);
                if (r32_off + 4 * mr <= args.dyn_bytes)  // stamped: nothing cleared between rounds
                    fy_parallel_stamped(D, P1, reinterpret_cast<uint32_t*>(dyn + r32_off), m, args.status);
                else
                    fy_parallel_data(D, P1, P0, m, args.status);
                in_place = true;
            } else if (m > 1) {
                for (uint32_t i = tid; i < m; i += blockDim.x) P0[i] = (uint16_t)i;  // fy_block permutes it
                fy_block(P0, P1, m, key, s.level, s.o);
            } else {
                in_place = true;  // one element
            }
        } else {
            if (tid == 0) {
                sh.stack[0] = pack_range(0, m, s.level, 0);
                sh.stack_top = 1;
            }
            for (;;) {
                __syncthreads();
                if (tid == 0) {
                    const uint32_t top = min(sh.stack_top, (uint32_t)kSmallStack);
                    if (top == 0) {
                        sh.flag = 1;
                    } else {
                        const uint64_t e = sh.stack[top - 1];
                        sh.stack_top = top - 1;
                        sh.cur_lo = (uint32_t)e;
                        sh.cur_hi = (uint32_t)(e >> 32);
                        sh.flag = 0;
                    }
                }
                __syncthreads();
                if (sh.flag) break;
                const uint64_t e = ((uint64_t)sh.cur_hi << 32) | sh.cur_lo;
                const uint32_t a = (uint32_t)(e & 0xFFFFFu);
                const uint32_t len = (uint32_t)((e >> 20) & 0xFFFFFu);
                const uint32_t L = (uint32_t)((e >> 40) & 0xFFu);
                const uint32_t buf = (uint32_t)((e >> 48) & 1u);
                __syncthreads();
                scatter_range<fast_groups(W)>(sh, P0, P1, a, len, L, buf, plan, key, s.o, L == s.level, args.status);
            }
        }
        __syncthreads();
        if (!wait_data()) break;
        // the write-back leaves out the last warp, which issues the next subproblem's bulk copy
        const uint32_t gth = blockDim.x - 32u;
        if (in_place) {
            if (tid < gth)
                for (uint32_t i = tid; i < m; i += gth) base[s.o + i] = D[i];
        } else if (tid < gth) {
            // four independent gathers in flight per thread
            for (uint32_t i0 = tid; i0 < m; i0 += 4u * gth) {
                uint32_t j[4];
                T v[4];
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    const uint32_t i = i0 + u * gth;
                    j[u] = i < m ? (uint32_t)P0[i] : 0u;
                }
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u)
                    if (j[u] < m) v[u] = D[j[u]];
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    const uint32_t i = i0 + u * gth;
                    if (i >= m) break;
                    if (j[u] < m) base[s.o + i] = v[u];
                    else report(args.status, RIP_EINTERNAL, 0x5107, j[u]);  // never read outside the subproblem
                }
            }
        }
        fence_proxy_async_smem();  // these reads of D come before the next bulk copy into it
        __syncthreads();
    }
}

// The leaves small_kernel skips (leaf_by_index), from the same list with the same shared memory.
template <int W>
__global__ void __launch_bounds__(kThreads, 1) leaf_kernel(SmallArgs args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallShared& sh = *reinterpret_cast<SmallShared*>(smem_raw);
    unsigned char* dyn = smem_raw + ((sizeof(SmallShared) + 15) & ~size_t(15));
    if (block_call_failed(args.status)) return;
    const uint32_t count = min(*args.count, args.capacity);
    if (threadIdx.x == 0) {
        mbar_init(&sh.load_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t loads = 0;
    // the list is scanned kSmallStack entries per CTA and pass, one per thread; this CTA's matches
    // are queued in the (here unused) stack and processed by the whole CTA
    uint32_t* queue = reinterpret_cast<uint32_t*>(sh.stack);
    for (uint32_t first = blockIdx.x * kSmallStack; first < count; first += gridDim.x * kSmallStack) {
        if (threadIdx.x == 0) sh.stack_top = 0;
        __syncthreads();
        const uint32_t i = first + threadIdx.x;
        if (threadIdx.x < kSmallStack && i < count && leaf_by_index(args, args.list[i], W))
            queue[atomicAdd(&sh.stack_top, 1u)] = i;
        __syncthreads();
        const uint32_t nq = sh.stack_top;
        bool ok = true;
        for (uint32_t q = 0; q < nq && ok; ++q) {
            const uint32_t item = queue[q];
            const Sub s = args.list[item];
            const ArrayDesc ad = args.arrays[s.arr];
            auto* base = reinterpret_cast<typename Elem<W>::T*>(ad.data);
            ok = fy_leaf_by_index<W>(args, s, base, (uint32_t)s.m, make_key(ad.seed), dyn, &sh.load_bar,
                                     loads & 1u, item);
            ++loads;
        }
        if (!ok) break;
        __syncthreads();
    }
}

}  // namespace

size_t small_fixed_smem() { return (sizeof(SmallShared) + 15) & ~size_t(15); }

size_t small_smem_bytes(uint64_t m, uint32_t w, bool medium) {
    const uint64_t mr = (m + 7u) & ~7ull;
    return small_fixed_smem() + 4 * mr + (medium ? 0 : w * mr + 16);
}

cudaError_t launch_small(const SmallArgs& args_in, uint32_t w, size_t smem, uint32_t grid, cudaStream_t stream) {
    cudaError_t err;
    SmallArgs args = args_in;
    args.dyn_bytes = (uint32_t)(smem - small_fixed_smem());
    {
        ProfScope p(args.medium ? "solve_medium" : "solve_small", stream);
        switch (w) {
            case 4:
                err = ensure_dyn_smem(reinterpret_cast<const void*>(small_kernel<4>), (int)smem);
                if (err != cudaSuccess) return err;
                small_kernel<4><<<grid, kThreads, smem, stream>>>(args);
                break;
            case 8:
                err = ensure_dyn_smem(reinterpret_cast<const void*>(small_kernel<8>), (int)smem);
                if (err != cudaSuccess) return err;
                small_kernel<8><<<grid, kThreads, smem, stream>>>(args);
                break;
            default:
                err = ensure_dyn_smem(reinterpret_cast<const void*>(small_kernel<16>), (int)smem);
                if (err != cudaSuccess) return err;
                small_kernel<16><<<grid, kThreads, smem, stream>>>(args);
                break;
        }
        err = cudaGetLastError();
    }
    if (err != cudaSuccess || args.medium) return err;
    ProfScope pl("solve_leaf", stream);
    switch (w) {
        case 4:
            err = ensure_dyn_smem(reinterpret_cast<const void*>(leaf_kernel<4>), (int)smem);
            if (err != cudaSuccess) return err;
            leaf_kernel<4><<<grid, kThreads, smem, stream>>>(args);
            break;
        case 8:
            err = ensure_dyn_smem(reinterpret_cast<const void*>(leaf_kernel<8>), (int)smem);
            if (err != cudaSuccess) return err;
            leaf_kernel<8><<<grid, kThreads, smem, stream>>>(args);
            break;
        default:
            err = ensure_dyn_smem(reinterpret_cast<const void*>(leaf_kernel<16>), (int)smem);
            if (err != cudaSuccess) return err;
            leaf_kernel<16><<<grid, kThreads, smem, stream>>>(args);
            break;
    }
    return cudaGetLastError();
}

}  // namespace rip
