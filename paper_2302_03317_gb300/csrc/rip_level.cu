// rip_level.cu -- one in-place scatter level over all large subproblems.
//
// The level computes the canonical layout of one ScatterShuffle level
// (Sec. 2.2; the in-place IpSc contract of Sec. 3.1 and Sec. 3.5: bucket b
// becomes a contiguous region) for every subproblem too large for one SM:
//
//  tiles     build the level's tile list (T elements per tile, per subproblem)
//  classify  one CTA streams one tile (rip_classify.cu): Philox bucket
//            draws, stable ranks per bucket, chunks staged in shared memory;
//            every completed block is written back into the tile's own,
//            already-read front ("home slots") or a small pool; the partial
//            streams (the tails) go to the pool
//  scan      per subproblem: bucket sizes, region starts, per-(tile, bucket)
//            prefix of full blocks and tails, child descriptors and rotations
//  resolve   turn each home slot's (bucket, block) into its destination slot
//  permute   move every block to its destination in place by following the
//            slot permutation; 8 lanes move one block, slots are claimed with
//            atomics (claim, read, then write), chains start anywhere
//  tails     write the tails (and the few blocks that straddle a region end)
//            from the pool to their final positions
//
// Children are stored rotated: logical index i of a child region lives at
// physical o + ((i + eps) mod m), eps chosen so that the child's full blocks
// sit on the B-aligned slot grid; every later reader goes through the rotation
// and the last one (the on-SM solver) writes canonical order.
#include "rip_internal.cuh"

namespace rip {

namespace {

// ------------------------------------------------------------------ helpers

// Acquire: a slot read out by a chain start (release store of 0) may be written
// only after that read; nothing written before this atomic needs ordering.
__device__ __forceinline__ uint32_t atom_or_acquire(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.or.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <typename U>
__device__ __forceinline__ U ld_cg(const U* p) {
    return __ldcg(p);
}

template <typename U>
__device__ __forceinline__ void cp_async_unit(U* dst, const U* src) {
    static_assert(sizeof(U) == 4 || sizeof(U) == 8 || sizeof(U) == 16, "cp.async sizes");
    if constexpr (sizeof(U) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(sizeof(U))
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool push_sub(Sub* list, uint32_t* count, uint32_t cap, const Sub& s, Status* st,
                                         uint32_t where) {
    const uint32_t i = atomicAdd(count, 1u);
    if (i < cap) {
        list[i] = s;
        return true;
    }
    report(st, RIP_EWORKSPACE, where, i);
    return false;
}

// Route a subproblem to the list that will process it.
__device__ void route_sub(const Sub& c, const DevPlan& plan, uint32_t small_max_m, Sub* next_big,
                          uint32_t* next_big_count, uint32_t big_cap, Sub* small, uint32_t* small_count,
                          Sub* medium, uint32_t* medium_count, uint32_t small_cap, uint32_t medium_cap, Sub* bigfy,
                          uint32_t* bigfy_count, uint32_t bigfy_cap, Status* st) {
    if (c.m <= 1) return;
    const bool leaf = plan.is_leaf(c.m, c.level);
    const bool solver_ok = leaf || small_solver_can_scatter(plan, c.m, c.level);
    if (c.m <= small_max_m && solver_ok)
        push_sub(small, small_count, small_cap, c, st, 0x6001);
    else if (c.m <= kMediumMaxM && solver_ok)
        push_sub(medium, medium_count, medium_cap, c, st, 0x6002);
    else if (leaf)
        push_sub(bigfy, bigfy_count, bigfy_cap, c, st, 0x6003);
    else
        push_sub(next_big, next_big_count, big_cap, c, st, 0x6004);
}

// ------------------------------------------------------------------ init

__global__ void init_kernel(InitArgs a) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        *a.status = Status{};  // this call's status word starts clean
        *a.lists.big_count[0] = 0;
        *a.lists.big_count[1] = 0;
        *a.lists.small_count = 0;
        *a.lists.medium_count = 0;
        *a.lists.bigfy_count = 0;
        for (int i = 0; i < 8; ++i) a.counters[i] = 0;
        *a.pool_used = 0;
        for (uint32_t i = 0; i < a.inline_count; ++i) a.arrays[i] = a.inline_arrays[i];
    }
    __syncthreads();
    for (uint32_t i = tid; i < a.narrays; i += gridDim.x * blockDim.x) {
        const ArrayDesc ad = a.arrays[i];
        Sub s{0, ad.n, i, 0, 0, 0};
        route_sub(s, a.plan, a.small_max_m, a.lists.big[0], a.lists.big_count[0], a.lists.big_cap,
                  a.lists.small, a.lists.small_count, a.lists.medium, a.lists.medium_count, a.lists.small_cap, a.lists.medium_cap,
                  a.lists.bigfy, a.lists.bigfy_count, a.lists.bigfy_cap, a.status);
    }
}

__global__ void descs_kernel(DescChunk c) {
    for (uint32_t i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.a[i];
}

// ------------------------------------------------------------------ tiles

__global__ void tiles_kernel(LevelArgs a) {
    __shared__ uint32_t scan[32];
    __shared__ uint64_t scan64[32];
    __shared__ uint32_t carry;
    __shared__ uint64_t scarry;
    const bool failed = block_call_failed(a.status);  // an earlier kernel failed: an empty wave
    const uint32_t nbig = min(*a.big_count, a.big_cap);
    const uint32_t we = nbig > a.wb && !failed ? min(nbig - a.wb, a.wcap) : 0u;  // subproblems of this wave
    const uint64_t B = a.B;
    if (threadIdx.x == 0) {
        carry = 0;
        scarry = 0;
    }
    __syncthreads();
    for (uint32_t c0 = 0; c0 < we; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        uint32_t nt = 0;
        uint64_t ns = 0, g0 = 0, ng = 0;
        uint32_t arr = 0;
        if (i < we) {
            const Sub sb = a.big[a.wb + i];
            const uint64_t t64 = a.T >= sb.m ? 1 : (sb.m + a.T - 1) / a.T;
            nt = (uint32_t)(t64 < 0xffffffffull ? t64 : 0xffffffffull);
            g0 = sb.o / B;                        // grid slots overlapping [o, o+m)
            ng = (sb.o + sb.m + B - 1) / B - g0;
            ns = (ng + 63) & ~63ull;               // segments start at multiples of 64
            arr = sb.arr;
        }
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<uint32_t>(nt, scan, &total);
        uint64_t stotal;
        const uint64_t sex = block_exclusive_scan<uint64_t>(ns, scan64, &stotal);
        const uint32_t begin = carry + ex;
        if (i < we) {
            a.sp_tile_begin[i] = begin;
            for (uint32_t t = 0; t < nt; ++t)
                if (begin + t < a.tile_cap) a.tiles[begin + t] = TileRef{a.wb + i, t};
            a.segs[i] = SegDesc{scarry + sex, g0, ng, arr, 0};
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry += total;
            scarry += stotal;
        }
        __syncthreads();
    }
    // the order classify takes the tiles in: all non-last tiles (full size) first, then every
    // subproblem's last, usually smaller, tile -- the short tiles fill the SMs that the long
    // ones leave idle when a wave has fewer subproblems than SMs
    if (carry <= a.tile_cap) {
        for (uint32_t i = threadIdx.x; i < we; i += blockDim.x) {
            const uint32_t begin = a.sp_tile_begin[i];
            const uint32_t end = i + 1 < we ? a.sp_tile_begin[i + 1] : carry;
            for (uint32_t t = begin; t + 1 < end; ++t) a.sched[t - i] = t;
            if (end > begin) a.sched[carry - we + i] = end - 1;
        }
    }
    if (threadIdx.x == 0) {
        bool ok = true;
        if (carry > a.tile_cap) {
            report(a.status, RIP_EWORKSPACE, 0x6101, carry);
            ok = false;
        }
        if (scarry > a.slot_cap) {  // the wave's segments do not fit the table: skip the wave
            report(a.status, RIP_EWORKSPACE, 0x6103, scarry);
            ok = false;
        }
        a.counters[0] = ok ? carry : 0u;
        for (int c = 1; c <= 6; ++c) a.counters[c] = 0;
        a.counters[7] = ok ? we : 0u;
        a.counters[8] = ok ? (uint32_t)(scarry / 64u) : 0u;
        *a.pool_used = 0;
        if (a.wb == 0 && nbig > a.wend) report(a.status, RIP_EWORKSPACE, 0x6104, nbig);  // more than planned
        if (a.wb == 0) {  // the next level's lists fill over all waves of this one
            *a.next_big_count = 0;
            *a.small_count = 0;
            *a.medium_count = 0;
        }
    }
}

// ------------------------------------------------------------------ scan

__global__ void scan_kernel(LevelArgs a, uint32_t small_max_m) {
    __shared__ uint64_t start[kMaxK];
    __shared__ uint64_t scan64[32];
    if (block_call_failed(a.status)) return;
    const uint32_t k = a.k, B = a.B;
    const uint32_t we = a.counters[7];
    for (uint32_t wi = blockIdx.x; wi < we; wi += gridDim.x) {
        const uint32_t sp = a.wb + wi;
        const Sub S = a.big[sp];
        const SegDesc seg = a.segs[wi];
        const uint32_t nt = (uint32_t)(a.T >= S.m ? 1 : (S.m + a.T - 1) / a.T);
        const uint32_t tb = a.sp_tile_begin[wi];
        if ((uint64_t)tb + nt > a.counters[0]) {  // tile list overflowed (reported by tiles_kernel)
            if (threadIdx.x == 0) report(a.status, RIP_EWORKSPACE, 0x6102, tb);
            continue;
        }
        for (uint32_t b = threadIdx.x; b < k; b += blockDim.x) {
            uint64_t size = 0;
            uint32_t fsum = 0, rsum = 0;
            for (uint32_t t = 0; t < nt; ++t) {
                const uint64_t ci = (uint64_t)(tb + t) * k + b;
                const uint32_t c = a.C[ci];
                a.FBc[ci] = fsum;
                a.TLc[ci] = rsum;
                fsum += c / B;
                rsum += c % B;
                size += c;
            }
            start[b] = size;
            ChildInfo ci{};
            ci.Fb = fsum;
            ci.placed = rsum;  // tails, temporarily
            a.child[(uint64_t)wi * k + b] = ci;
        }
        __syncthreads();
        {
            const uint32_t i0 = 2 * threadIdx.x, i1 = 2 * threadIdx.x + 1;
            const uint64_t v0 = i0 < k ? start[i0] : 0, v1 = i1 < k ? start[i1] : 0;
            const uint64_t ex = block_exclusive_scan<uint64_t>(v0 + v1, scan64, nullptr);
            if (i0 < k) start[i0] = ex;
            if (i1 < k) start[i1] = ex + v0;
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < k; b += blockDim.x) {
            ChildInfo ci = a.child[(uint64_t)wi * k + b];
            const uint32_t tails = ci.placed;
            const uint64_t sb = start[b];
            const uint64_t se = b + 1 < k ? start[b + 1] : S.m;
            ci.o = S.o + sb;
            ci.m = se - sb;
            const uint32_t e0 = (uint32_t)((B - ci.o % B) % B);
            ci.eps = ci.m > e0 ? e0 : 0;
            ci.placed = ci.Fb >= 1 ? (e0 <= tails ? ci.Fb : ci.Fb - 1) : 0;
            ci.slot_base = seg.base + ((ci.o + e0) / B - seg.orig);
            a.child[(uint64_t)wi * k + b] = ci;
            const Sub c{ci.o, ci.m, S.arr, S.level + 1, ci.eps, 0};
            route_sub(c, a.plan, small_max_m, a.next_big, a.next_big_count, a.big_cap, a.small, a.small_count,
                      a.medium, a.medium_count, a.small_cap, a.medium_cap, a.bigfy, a.bigfy_count, a.bigfy_cap, a.status);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ resolve

__global__ void resolve_kernel(LevelArgs a) {
    if (block_call_failed(a.status)) return;
    const uint32_t ntiles = a.counters[0];
    const uint32_t k = a.k, B = a.B;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileRef tr = a.tiles[tile];
        const TileInfo ti = a.tinfo[tile];
        for (uint32_t h = threadIdx.x; h < ti.home_used; h += blockDim.x) {
            const uint32_t w = a.words[ti.hs0 + h];
            if ((w & (kWordOcc | kWordTaken)) != kWordOcc) continue;  // empty: held a part of a tail only
            const uint32_t b = (w >> kBlkBits) & (kMaxK - 1u);
            const uint32_t blk = w & ((1u << kBlkBits) - 1u);
            const ChildInfo ci = a.child[(uint64_t)(tr.sp - a.wb) * k + b];
            const uint32_t J = a.FBc[(uint64_t)tile * k + b] + blk;
            uint32_t nw;
            if (J < ci.placed) {
                const uint64_t d = ci.slot_base + J;
                if (d > kWordDestMask) report(a.status, RIP_EINVAL, 0x6301, d);
                nw = kWordOcc | (uint32_t)d;
            } else {
                const uint64_t alloc = ((uint64_t)B + a.pool_align - 1) / a.pool_align * a.pool_align;
                const uint64_t off = atomicAdd((unsigned long long*)a.pool_used, (unsigned long long)alloc);
                if (off + B > a.pool_cap) report(a.status, RIP_EWORKSPACE, 0x6302, off);
                const uint32_t rec = atomicAdd(&a.counters[2], 1u);
                if (rec < a.dem_cap)
                    a.dem[rec] = DemRec{tr.sp, tile, b, blk, off};
                else
                    report(a.status, RIP_EWORKSPACE, 0x6303, rec);
                nw = kWordOcc | kWordDem | rec;
            }
            a.words[ti.hs0 + h] = nw;
        }
    }
}

// ------------------------------------------------------------------ permute

template <typename U>
__global__ void __launch_bounds__(kPermuteThreads, 4) permute_kernel(LevelArgs a, uint32_t w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t units = a.B * w / (uint32_t)sizeof(U);
    const uint32_t tid = threadIdx.x;
    const uint32_t g = tid / kGroup, lg = tid % kGroup;
    const uint32_t gmask = 0xFFu << ((tid & 31u) & ~(kGroup - 1u));
    const uint32_t leader_lane = (tid & 31u) & ~(kGroup - 1u);
    const bool leader = lg == 0;
    U* slots = reinterpret_cast<U*>(smem_raw) + (size_t)g * 2u * units;  // carried block, incoming block
    uint32_t cs = 0;  // slot of the carried block
    const uint64_t slot_bytes = (uint64_t)a.B * w;

    bool carrying = false;
    uint32_t dw = 0;
    char* abase = nullptr;
    uint64_t aslot = 0, anslots = 0;
    uint64_t chunk = ~0ull;   // current 64-slot chunk of start candidates
    uint32_t cpos = 64;       // next candidate inside the chunk
    uint32_t cw[8];           // the chunk's words, 8 per lane of the group (lane lg holds slots lg*8 ..)
    uint32_t steps = 0;       // swaps of the current chain

    for (;;) {
        if (!carrying) {
            if (cpos >= 64) {
                uint64_t c0 = ~0ull;  // stays past the end once the call has failed
                if (leader && !call_failed(a.status)) c0 = atomicAdd((unsigned long long*)&a.counters[4], 1ull);
                chunk = __shfl_sync(gmask, c0, leader_lane);
                if (chunk >= a.counters[8]) break;
                const uint64_t s0 = chunk * 64u + lg * 8u;
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) cw[j] = ld_relaxed(&a.words[s0 + j]);
                cpos = 0;
                // the segment holding this chunk (segments start at multiples of 64)
                uint32_t lo = 0, hi = a.counters[7];
                if (leader) {
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (a.segs[mid].base <= chunk * 64u) lo = mid; else hi = mid;
                    }
                }
                lo = __shfl_sync(gmask, lo, leader_lane);
                const SegDesc sg = a.segs[lo];
                const ArrayDesc ad = a.arrays[sg.arr];
                aslot = sg.base;
                // whole grid slots of the array inside the segment
                const uint64_t whole = ad.n / a.B > sg.orig ? ad.n / a.B - sg.orig : 0;
                anslots = sg.nslots < whole ? sg.nslots : whole;
                abase = ad.data + sg.orig * slot_bytes;
            }
            // next candidate holding an unmoved block
            const uint32_t owner = cpos >> 3;
            uint32_t w0 = 0;
#pragma unroll
            for (uint32_t j = 0; j < 8; ++j)
                if ((cpos & 7u) == j) w0 = cw[j];
            w0 = __shfl_sync(gmask, w0, leader_lane + owner);
            const uint64_t s = chunk * 64u + cpos;
            ++cpos;
            if ((w0 >> 30) != 1u) continue;
            uint32_t ok = 0;
            if (leader) ok = atomicCAS(&a.words[s], w0, w0 | kWordTaken) == w0;
            ok = __shfl_sync(gmask, ok, leader_lane);
            if (!ok) continue;
            if (s < aslot || s - aslot >= anslots) {
                if (leader) report(a.status, RIP_EINTERNAL, 0x6403, s);
                continue;
            }
            const U* sp = reinterpret_cast<const U*>(abase + (s - aslot) * slot_bytes);
            if (reinterpret_cast<uintptr_t>(sp) % sizeof(U)) {  // claimed but unmovable: report
                if (leader) report(a.status, RIP_EINTERNAL, 0x6407, s);
                continue;
            }
            U* buf = slots + cs * units;
            for (uint32_t u = lg; u < units; u += kGroup) buf[u] = ld_cg(sp + u);
            __syncwarp(gmask);  // every lane's read of slot s has returned
            if (leader) st_release(&a.words[s], 0u);
            carrying = true;
            dw = w0;
            steps = 0;
            continue;
        }

        if (dw & kWordDem) {
            if ((dw & kWordDestMask) >= min(a.counters[2], a.dem_cap)) {
                if (leader) report(a.status, RIP_EINTERNAL, 0x6404, dw);
                carrying = false;
                continue;
            }
            const DemRec rec = a.dem[dw & kWordDestMask];
            if (rec.pool_off + a.B > a.pool_cap || ((rec.pool_off * w) % sizeof(U)) != 0) {
                if (leader) report(a.status, RIP_EINTERNAL, 0x6405, rec.pool_off);
                carrying = false;
                continue;
            }
            U* dst = reinterpret_cast<U*>(a.pool + rec.pool_off * w);
            const U* buf = slots + cs * units;
            for (uint32_t u = lg; u < units; u += kGroup) dst[u] = buf[u];
            __syncwarp(gmask);
            carrying = false;
            continue;
        }
        const uint64_t d = dw & kWordDestMask;
        if (d < aslot || d - aslot >= anslots) {  // never write outside the array
            if (leader) report(a.status, RIP_EINTERNAL, 0x6402, d);
            carrying = false;
            continue;
        }
        U* dp = reinterpret_cast<U*>(abase + (d - aslot) * slot_bytes);
        if (reinterpret_cast<uintptr_t>(dp) % sizeof(U)) {
            if (leader) report(a.status, RIP_EINTERNAL, 0x6406, d);
            carrying = false;
            continue;
        }
        if (steps >= a.park_after) {
            // long chain: put the block aside (the destination keeps its unmoved block,
            // which a chain start will read out later); placed after this kernel
            uint32_t ok = 0;
            uint64_t off = 0;
            if (leader) {
                const uint32_t rec = atomicAdd(&a.counters[6], 1u);
                if (rec < a.park_cap) {
                    const uint64_t alloc = ((uint64_t)a.B + a.pool_align - 1) / a.pool_align * a.pool_align;
                    off = atomicAdd((unsigned long long*)a.pool_used, (unsigned long long)alloc);
                    ok = off + a.B <= a.pool_cap && ((off * w) % sizeof(U)) == 0;
                    a.parks[rec] = ParkRec{ok ? off : ~0ull, reinterpret_cast<uint64_t>(dp)};
                }
            }
            ok = __shfl_sync(gmask, ok, leader_lane);
            if (ok) {
                off = __shfl_sync(gmask, off, leader_lane);
                U* dst = reinterpret_cast<U*>(a.pool + off * w);
                const U* buf = slots + cs * units;
                for (uint32_t u = lg; u < units; u += kGroup) dst[u] = buf[u];
                __syncwarp(gmask);
                carrying = false;
                continue;
            }
            steps = 0x80000000u;  // no room: finish this chain without parking
        }
        // the block at d, read ahead of the claim into the incoming slot (only this group writes d)
        U* buf = slots + cs * units;
        U* inc = slots + (cs ^ 1u) * units;
        for (uint32_t u = lg; u < units; u += kGroup) cp_async_unit(inc + u, dp + u);
        cp_async_commit();
        uint32_t old = 0;
        if (leader) old = atom_or_acquire(&a.words[d], kWordTaken);
        old = __shfl_sync(gmask, old, leader_lane);
        __syncwarp(gmask);  // order the group's accesses to d after the leader's acquire
        if (old & kWordTaken) {
            // a chain start holds the slot: wait (bounded) until it has read it out
            const uint32_t limit = a.wait_polls ? a.wait_polls : (1u << 24);
            uint32_t spins = 0;
            if (leader) {
                while (ld_acquire(&a.words[d]) != 0u) {
                    if (++spins > limit) {
                        report(a.status, RIP_ETIMEOUT, 0x6401, d);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            spins = __shfl_sync(gmask, spins, leader_lane);
            cp_async_wait_all();  // the incoming slot is reloaded on the next try
            if (spins > limit) {
                carrying = false;  // give up; the error is reported
                continue;
            }
            __syncwarp(gmask);
            continue;
        }
        cp_async_wait_all();  // this lane's units of the block at d are in the incoming slot
        if (old & kWordOcc) {
            // swap: write ours to d, carry the block read from it
            for (uint32_t u = lg; u < units; u += kGroup) dp[u] = buf[u];
            __syncwarp(gmask);
            cs ^= 1u;
            dw = old;
            ++steps;
        } else {
            for (uint32_t u = lg; u < units; u += kGroup) dp[u] = buf[u];
            __syncwarp(gmask);
            carrying = false;
        }
    }
}

// ------------------------------------------------------------------ tails

template <int W>
__global__ void tails_kernel(LevelArgs a) {
    using T = typename Elem<W>::T;
    __shared__ uint32_t pre[kMaxK];
    __shared__ uint32_t scan[32];
    if (block_call_failed(a.status)) return;
    const uint32_t ntiles = a.counters[0];
    const uint32_t k = a.k, B = a.B;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const T* pool = reinterpret_cast<const T*>(a.pool);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileRef tr = a.tiles[tile];
        const TileInfo ti = a.tinfo[tile];
        const Sub S = a.big[tr.sp];
        T* base = reinterpret_cast<T*>(a.arrays[S.arr].data);
        const uint32_t i0 = 2 * threadIdx.x, i1 = 2 * threadIdx.x + 1;
        const uint32_t r0 = i0 < k ? a.C[(uint64_t)tile * k + i0] % B : 0;
        const uint32_t r1 = i1 < k ? a.C[(uint64_t)tile * k + i1] % B : 0;
        const uint32_t ex = block_exclusive_scan<uint32_t>(r0 + r1, scan, nullptr);
        if (i0 < k) pre[i0] = ex;
        if (i1 < k) pre[i1] = ex + r0;
        __syncthreads();
        for (uint32_t b = warp; b < k; b += nwarps) {
            const uint64_t ci_idx = (uint64_t)tile * k + b;
            const uint32_t R = a.C[ci_idx] % B;
            if (R == 0) continue;
            const ChildInfo ci = a.child[(uint64_t)(tr.sp - a.wb) * k + b];
            const uint64_t x0 = (uint64_t)B * ci.Fb + a.TLc[ci_idx];
            const T* src = pool + ti.pool_base + pre[b];
            const uint64_t n_arr = a.arrays[S.arr].n;
            if (ti.pool_base + pre[b] + R > a.pool_cap || x0 + R > ci.m || ci.o + ci.m > n_arr) {
                if (lane == 0) report(a.status, RIP_EINTERNAL, 0x6601, x0);
                continue;
            }
            for (uint32_t j = lane; j < R; j += 32u) {
                uint64_t xe = x0 + j + ci.eps;
                if (xe >= ci.m) xe -= ci.m;
                base[ci.o + xe] = src[j];
            }
        }
        __syncthreads();
    }
}

// Parked blocks go to their destination slots, all of which were read out by
// the permutation kernel.
template <typename U>
__global__ void parked_kernel(LevelArgs a, uint32_t w) {
    if (call_failed(a.status)) return;
    const uint32_t n = min(a.counters[6], a.park_cap);
    const uint32_t units = a.B * w / (uint32_t)sizeof(U);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < n; i += nw) {
        const ParkRec r = a.parks[i];
        if (r.pool_off == ~0ull) continue;
        const U* src = reinterpret_cast<const U*>(a.pool + r.pool_off * w);
        U* dst = reinterpret_cast<U*>(r.dst);
        for (uint32_t u = lane; u < units; u += 32u) dst[u] = src[u];
    }
}

template <int W>
__global__ void demoted_kernel(LevelArgs a) {
    using T = typename Elem<W>::T;
    if (call_failed(a.status)) return;
    const uint32_t ndem = min(a.counters[2], a.dem_cap);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const T* pool = reinterpret_cast<const T*>(a.pool);
    for (uint32_t i = gw; i < ndem; i += nw) {
        const DemRec rec = a.dem[i];
        const ChildInfo ci = a.child[(uint64_t)(rec.sp - a.wb) * a.k + rec.b];
        const uint64_t J = (uint64_t)a.FBc[(uint64_t)rec.tile * a.k + rec.b] + rec.blk;
        const ArrayDesc ad = a.arrays[a.big[rec.sp].arr];
        T* base = reinterpret_cast<T*>(ad.data);
        if ((J + 1) * a.B > ci.m || ci.o + ci.m > ad.n || rec.pool_off + a.B > a.pool_cap) {
            if (lane == 0) report(a.status, RIP_EINTERNAL, 0x6701, J);
            continue;
        }
        for (uint32_t j = lane; j < a.B; j += 32u) {
            uint64_t xe = J * a.B + j + ci.eps;
            if (xe >= ci.m) xe -= ci.m;
            base[ci.o + xe] = pool[rec.pool_off + j];
        }
    }
}

// ------------------------------------------------------------------ large leaves

// Leaves too large for one SM (only with plans whose base or level cap
// exceeds the on-SM limit): undo the rotation in place, then a plain
// sequential Fisher-Yates in global memory, one thread per leaf.
template <int W>
__global__ void bigfy_kernel(const Sub* list, const uint32_t* count, uint32_t cap, const ArrayDesc* arrays,
                             DevPlan plan, const uint32_t* leftover, Status* call, Status* status) {
    using T = typename Elem<W>::T;
    // every earlier kernel of the call is complete: its status goes to the device's word
    const Status cs = *call;
    if (blockIdx.x == 0 && threadIdx.x == 0 && cs.code) report(status, cs.code, cs.where, cs.detail);
    if (cs.code) return;
    const uint32_t n = min(*count, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && *leftover != 0)  // deeper recursion than the host planned
        report(status, RIP_EWORKSPACE, 0x6501, *leftover);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Sub s = list[i];
        const ArrayDesc ad = arrays[s.arr];
        T* x = reinterpret_cast<T*>(ad.data) + s.o;
        const uint64_t m = s.m;
        if (m > (1ull << 32)) {  // Fisher-Yates draws are 32-bit (Lemire with 32-bit words)
            report(status, RIP_EINVAL, 0x6502, m);
            continue;
        }
        auto rev = [&](uint64_t l, uint64_t r) {  // reverse x[l..r)
            while (l + 1 < r) {
                --r;
                const T t = x[l];
                x[l] = x[r];
                x[r] = t;
                ++l;
            }
        };
        if (s.eps) {  // physical = rotate-left of logical by (m - eps): three reversals
            const uint64_t e = s.eps;
            rev(0, e);
            rev(e, m);
            rev(0, m);
            // now logical i sits at physical i
        }
        FyStream fs;
        fs.init(make_key(ad.seed), s.level, s.o);
        for (uint64_t j = m - 1; j >= 1; --j) {
            const uint64_t p = fs.draw(j);
            const T t = x[j];
            x[j] = x[p];
            x[p] = t;
        }
    }
}

}  // namespace

// Threads of a permutation CTA: every kGroup lanes move one block and hold two B-element slots
// in shared memory (the carried block and the next one, read ahead); large blocks get fewer
// groups per CTA.  0: a single group's slots do not fit.
uint32_t permute_threads(uint32_t B, uint32_t w) {
    const size_t per_group = 2ull * B * w;
    const size_t groups = per_group ? kSmemOptin / per_group : 0;
    const size_t threads = std::min<size_t>(kPermuteThreads, groups * kGroup) / 32u * 32u;
    return (uint32_t)threads;
}

size_t permute_smem_bytes(uint32_t B, uint32_t w) {
    return (size_t)(permute_threads(B, w) / kGroup) * 2u * B * w;
}

cudaError_t launch_descs(const DescChunk& c, cudaStream_t s) {
    ProfScope p("descs", s);
    descs_kernel<<<1, 160, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_init(const InitArgs& a, cudaStream_t s) {
    ProfScope p("init", s);
    init_kernel<<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_level_w(const LevelArgs& a, uint32_t num_sms, cudaStream_t s, uint32_t* launches) {
    cudaError_t err;
    {
        ProfScope p("tiles", s);
        tiles_kernel<<<1, 1024, 0, s>>>(a);
    }
    err = launch_classify(a, W, num_sms, s);
    if (err != cudaSuccess) return err;
    {
        ProfScope p("scan", s);
        scan_kernel<<<num_sms * 2, 512, 0, s>>>(a, a.small_max_m);
    }
    {
        ProfScope p("resolve", s);
        resolve_kernel<<<num_sms * 4, 256, 0, s>>>(a);
    }
    const uint32_t pthreads = permute_threads(a.B, W);
    if (pthreads == 0) return cudaErrorInvalidConfiguration;  // a block of more than 113 KB
    const size_t psm = permute_smem_bytes(a.B, W);
    const uint32_t pgrid = num_sms * 8u * (kPermuteThreads / pthreads);
    if (a.vec16) {
        err = ensure_dyn_smem(reinterpret_cast<const void*>(permute_kernel<uint4>), (int)psm);
        if (err != cudaSuccess) return err;
        ProfScope p("permute", s);
        permute_kernel<uint4><<<pgrid, pthreads, psm, s>>>(a, W);
    } else {
        using T = typename Elem<W>::T;
        err = ensure_dyn_smem(reinterpret_cast<const void*>(permute_kernel<T>), (int)psm);
        if (err != cudaSuccess) return err;
        ProfScope p("permute", s);
        permute_kernel<T><<<pgrid, pthreads, psm, s>>>(a, W);
    }
    {
        ProfScope p("parked", s);
        if (a.vec16)
            parked_kernel<uint4><<<num_sms * 2, 256, 0, s>>>(a, W);
        else
            parked_kernel<typename Elem<W>::T><<<num_sms * 2, 256, 0, s>>>(a, W);
    }
    {
        ProfScope p("tails", s);
        tails_kernel<W><<<num_sms * 4, 512, 0, s>>>(a);
    }
    {
        ProfScope p("demoted", s);
        demoted_kernel<W><<<num_sms, 256, 0, s>>>(a);
    }
    if (launches) *launches += 8;
    return cudaGetLastError();
}

cudaError_t launch_level(const LevelArgs& a, uint32_t w, uint32_t num_sms, cudaStream_t s, uint32_t* launches) {
    switch (w) {
        case 4: return launch_level_w<4>(a, num_sms, s, launches);
        case 8: return launch_level_w<8>(a, num_sms, s, launches);
        default: return launch_level_w<16>(a, num_sms, s, launches);
    }
}

cudaError_t launch_bigfy(const Sub* list, const uint32_t* count, uint32_t cap, const ArrayDesc* arrays,
                         DevPlan plan, uint32_t w, const uint32_t* leftover, Status* status, Status* global,
                         cudaStream_t s) {
    ProfScope p("bigfy", s);
    switch (w) {
        case 4: bigfy_kernel<4><<<8, 32, 0, s>>>(list, count, cap, arrays, plan, leftover, status, global); break;
        case 8: bigfy_kernel<8><<<8, 32, 0, s>>>(list, count, cap, arrays, plan, leftover, status, global); break;
        default: bigfy_kernel<16><<<8, 32, 0, s>>>(list, count, cap, arrays, plan, leftover, status, global); break;
    }
    return cudaGetLastError();
}

}  // namespace rip
