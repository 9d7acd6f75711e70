// rip_classify.cu -- the classify step of one in-place scatter level.
//
// One CTA streams one tile of T elements (Sec. 3.1: every element draws its
// bucket, Sec. 2.2; elements of one bucket keep their input order inside the
// tile).  Bucket b's elements form a stream; its j-th B-element block is the
// stream's elements [jB, (j+1)B).  Every completed block is written back into
// the tile's own front, which has already been read ("home slots", the
// in-place block buffers of Sec. 3.5), or, while no read home slot is free,
// into a small pool; the remainder of every stream (fewer than B elements) is
// the tile's tail for that bucket and goes to the pool at the end of the tile.
//
// Per round of nwr*128 consecutive positions:
//   load     the round's elements arrive in a shared-memory buffer by bulk
//            (TMA) copies one or two rounds ahead, completing on an mbarrier;
//            ragged edges (unaligned ends, the rotation's wrap piece) are
//            copied by the threads.  The I/O warp does nothing else: with the
//            chunk stores also on the copy engine, a round's load queued behind
//            them and the compute warps waited for their input
//   rank     Philox bucket draws (a1), stable ranks per bucket: the lanes of a
//            step with the same bucket come from a 32-entry shared-memory mask
//            row per warp (indexed by the low five bucket bits) and one ballot
//            per higher bit; the warp's running count per bucket lives in a
//            (bucket, warp) table of 16-bit counters (a2)
//   book     per bucket: exclusive prefix over the ranking warps (one lane
//            per bucket, 32 buckets per warp), blocks completed, home slots or
//            pool blocks for blocks that receive data, slot words
//            -- meanwhile the other warps write the chunks completed by the
//               previous round to their blocks with 16-byte stores (with fewer
//               ranking warps than compute warps, the warps that do not rank
//               do so during the ranking instead)
//   place    every element goes to its bucket's shared-memory chunk (Bs
//            elements, Bs divides B), straight to its block in global memory
//            when its whole chunk lies inside this round, or is carried into
//            the next round when it starts a chunk that completes later
//
// Pipelined rounds (k = 64 or 256 with 4- or 8-byte elements, the common
// plans): the k/32 bookkeeping warps do nothing else, and book round i-1 while
// the other warps write out round i-2's completed chunks and rank round i; the
// rank warps then place round i-1.  The (bucket, warp) table has two copies, so
// round i's counts do not disturb round i-1's offsets; elements carried into
// the next round wait in registers, so a round's buffer is free as soon as it
// is placed.  With one barrier per phase the bookkeeping (latency-bound, k
// lanes) hides behind the ranking (throughput-bound) instead of following it.
// Both groups then wait mostly on the shared-memory unit (loads, stores,
// atomics and shuffles share its queue), so these rounds spend few shared-memory
// operations: 64-entry mask rows, a lane's four buckets packed into one word
// (one shuffle per step), and a table stride that lets the bookkeeping scan two
// counts per 32-bit word.
//
// A block gets its location when its first chunk is written.  A home slot h
// may be used once the tile's elements [0, (h+1)B) have been read; otherwise
// (at the start of a tile, when chunks are smaller than blocks) the block goes
// to the pool.  At most k blocks per tile take the pool that way: every
// allocated block except the <= k open ones is complete, and the home slots
// only lag the consumed elements by less than one block.
#include "rip_internal.cuh"

namespace rip {

namespace {

template <bool V>
struct BoolC {
    static constexpr bool value = V;
};

constexpr uint64_t kLocPool = 1ull << 63;  // location in the pool (else: element index in the array)
constexpr uint32_t kNone = 0xffffffffu;
constexpr uint32_t kLoadPiece = 4096u;  // bytes per bulk copy of a round's input (a multiple of 16)

struct ClsMisc {
    uint64_t full[3];      // input buffer loaded (transaction count of the bulk copy)
    uint64_t flush_ready;  // the compute warps have placed a round
    uint64_t pool_base;
    uint32_t tile;
    uint32_t home_next;
    uint32_t nflush[2];
    uint32_t fail;   // a wait of this CTA expired (either role)
    uint32_t cfail;  // the compute warps' verdict for the current round (written by thread 0 before
                     // a compute barrier, read by every compute thread after it)
    uint32_t scan[32];
};

// Lanes of the warp whose buckets agree with the calling lane's in the bits above the low
// five (the low five are matched through a shared-memory mask row): one ballot per bit;
// KB > 0 fixes the bit count at compile time.
template <int KB, int LO = 5>
__device__ __forceinline__ uint32_t bucket_peers_hi(uint32_t b, uint32_t kbits) {
    uint32_t peers = 0xffffffffu;
    if constexpr (KB > 0) {
#pragma unroll
        for (int i = LO; i < KB; ++i) {
            const bool bit = (b >> i) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
    } else {
        for (uint32_t i = 5; i < kbits; ++i) {
            const bool bit = (b >> i) & 1u;
            const uint32_t m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
    }
    return peers;
}

// Geometry that depends on k only (the same formulas as classify_config): warp 31 does the
// bulk copies, warps 0..30 compute; nwr of them rank (the table holds k * nwr counters).
constexpr uint32_t kIoWarp = kClassifyThreads / 32u - 1u;
constexpr uint32_t kComputeThreads = kIoWarp * 32u;
// 16-byte records rank with 16 warps: rounds half as long keep whole blocks staged.  k = 1024
// ranks with 16 warps, not 8: rounds of 2048 positions halve the per-element share of the
// bookkeeping over 1024 buckets (measured at 2^34: classify 1.42 -> 1.19 s for u32, 2.20 -> 1.78 s
// for u64; 31 warps measured slower, its staged chunks shrink to 32 or 16 bytes)
// Pipelined rounds (k = 64 or 256, elements of 4 or 8 bytes): warps 0 .. k/32-1 do the
// bookkeeping only, the others rank and place, and the bookkeeping of a round runs while the next
// round is ranked (the table of counts is double-buffered).
__host__ __device__ constexpr bool cls_pipe(uint32_t k, uint32_t w) { return (k == 64u || k == 256u) && w <= 8u; }
__host__ __device__ constexpr uint32_t cls_nwr(uint32_t k, uint32_t w) {
    return cls_pipe(k, w) ? kIoWarp - k / 32u
           : (k >= 1024u ? 16384u / k : 8192u / k) < (w >= 16 ? 16u : kIoWarp)
               ? (k >= 1024u ? 16384u / k : 8192u / k)
               : (w >= 16 ? 16u : kIoWarp);
}
// Table stride per bucket (16-bit entries, more than nwr): odd, or for pipelined rounds twice an
// odd number -- a warp's entries of 32 buckets still fall in distinct banks, and every column starts
// on a 4-byte boundary, so the bookkeeping reads and writes it two entries at a time.
__host__ __device__ constexpr uint32_t cls_stride(uint32_t k, uint32_t w) {
    return cls_pipe(k, w) ? ((cls_nwr(k, w) + 1u) / 2u | 1u) * 2u : (cls_nwr(k, w) + 1u) | 1u;
}

__device__ __forceinline__ void compute_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(kComputeThreads) : "memory");
}

// A flush entry: bucket in bits 48..57, the chunk's destination location in the rest.
constexpr uint64_t kEntLoc = ~(0x3FFull << 48);

// KB = log2 k for the specialised kernels, 0: k from the arguments.
template <int W, int KB>
__global__ void __launch_bounds__(kClassifyThreads, 1) classify_kernel(LevelArgs a) {
    using T = typename Elem<W>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ClsCfg g = a.cls;
    constexpr uint32_t KC = KB > 0 ? (1u << KB) : 0u;
    constexpr bool PIPE = KB > 0 && cls_pipe(KC, W);
    ClsMisc& ms = *reinterpret_cast<ClsMisc*>(smem_raw);
    uint16_t* tbl = reinterpret_cast<uint16_t*>(smem_raw + g.off_tbl);
    uint32_t* run = reinterpret_cast<uint32_t*>(smem_raw + g.off_u32);
    const uint32_t k = KB > 0 ? KC : a.k;
    const uint32_t nwr = KB > 0 ? cls_nwr(KC, W) : g.nwr;
    const uint32_t S = KB > 0 ? cls_stride(KC, W) : g.S;
    const uint32_t B = a.B, L = a.level, Bs = g.Bs, cpb = g.cpb;
    uint32_t* rb = run + k;      // stream length before the current round
    uint32_t* oblk = rb + k;     // block index of the open block (kNone: none)
    uint32_t* jnew = oblk + k;   // first block allocated this round
    uint32_t* take = jnew + k;   // of which this many got home slots
    uint32_t* hbase = take + k;  // first of those home slots
    uint64_t* optr = reinterpret_cast<uint64_t*>(smem_raw + g.off_u64);  // location of the open block
    uint64_t* jloc = optr + k;   // location of the block holding the round's first chunk
    uint64_t* pbase = jloc + k;  // pool location of the round's first pool block
    uint64_t* flist = reinterpret_cast<uint64_t*>(smem_raw + g.off_flist);  // 2 x k flush entries
    uint32_t* masks = reinterpret_cast<uint32_t*>(smem_raw + g.off_mask);  // per ranking warp: 32 lane masks
    T* stage = reinterpret_cast<T*>(smem_raw + g.off_stage);
    T* bufs = reinterpret_cast<T*>(smem_raw + g.off_buf);

    const uint32_t kbits = KB > 0 ? (uint32_t)KB : log2_pow2(k);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const bool io = warp == kIoWarp;
    const uint32_t round = nwr * 128u, q = g.q, nbuf = g.nbuf;
    const uint32_t ntiles = a.counters[0];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const bool bs_pow2 = (Bs & (Bs - 1u)) == 0;
    const uint32_t bs_shift = log2_pow2(Bs);
    const bool b_pow2 = (B & (B - 1u)) == 0;
    const uint32_t b_shift = log2_pow2(B);
    const bool flush_vec = a.vec16 && (Bs * W) % 16u == 0;
    T* pool = reinterpret_cast<T*>(a.pool);
    const uint32_t polls = a.wait_polls ? a.wait_polls : kMbarPolls;  // hand-off waits

    for (uint32_t j = tid; j < nwr * (PIPE ? 64u : 32u); j += blockDim.x) masks[j] = 0;  // kept zero after every step
    if (tid == 0) {
        for (uint32_t i = 0; i < nbuf; ++i) mbar_init(&ms.full[i], 1);
        mbar_init(&ms.flush_ready, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ms.fail = 0;
    }
    __syncthreads();

    // completions so far of the input buffers and of flush_ready (one each per round); every
    // thread counts the same way
    uint32_t grc = 0, frc = 0;
    for (;;) {
        if (tid == 0) {
            const uint32_t c = atomicAdd(&a.counters[1], 1u);
            ms.tile = c < ntiles && !call_failed(a.status) ? a.sched[c] : 0xffffffffu;
            ms.cfail = 0;
        }
        __syncthreads();
        const uint32_t tile = ms.tile;
        if (tile >= ntiles || ms.fail) break;
        const TileRef tr = a.tiles[tile];
        const Sub Sp = a.big[tr.sp];
        const ArrayDesc ad = a.arrays[Sp.arr];
        T* base = reinterpret_cast<T*>(ad.data);
        const PhiloxKey pk = make_key(ad.seed);
        const uint64_t lo = (uint64_t)tr.t * a.T;
        const uint32_t r = (uint32_t)(min(lo + a.T, Sp.m) - lo);
        const uint64_t alo = Sp.o + Sp.eps + lo;  // physical start of the tile's aligned piece
        const uint32_t avail = Sp.m > Sp.eps + lo ? (uint32_t)min((uint64_t)r, Sp.m - Sp.eps - lo) : 0u;
        const uint32_t H = avail / B;
        const SegDesc seg = a.segs[tr.sp - a.wb];
        const uint64_t hs0 = seg.base + (alo / B - seg.orig);  // table entry of home slot 0
        const uint64_t P0 = Sp.o + lo;  // logical global position of the tile's first element
        const uint32_t delta = (uint32_t)(P0 & 3u);
        const uint64_t Q0 = P0 >> 2;
        const uint32_t rv = r + delta;  // positions covered, counted from 4*Q0
        const uint32_t nrounds = (rv + round - 1) / round;
        if (alo % B != 0 && tid == 0) report(a.status, RIP_EINTERNAL, 0x6201, alo);

        // Slots of this level's grid inside the leading wrap piece [o, o+eps) lie in the
        // region but in no tile's home range (only when B is smaller than the parent's):
        // mark them empty so the permutation may fill them.
        if (tr.t == 0 && Sp.eps >= B) {
            const uint64_t first = (Sp.o + B - 1) / B, last = (Sp.o + Sp.eps) / B;
            for (uint64_t x = first + tid; x < last; x += blockDim.x) a.words[seg.base + (x - seg.orig)] = 0u;
        }
        for (uint32_t b = tid; b < k; b += blockDim.x) {
            run[b] = 0;
            oblk[b] = kNone;
        }
        // every home slot starts empty; completed blocks fill in their words
        for (uint32_t h = tid; h < H; h += blockDim.x) a.words[hs0 + h] = 0u;
        for (uint32_t j = tid; j < k * S * (PIPE ? 2u : 1u); j += blockDim.x) tbl[j] = 0;
        if (tid == 0) {
            ms.home_next = 0;
            ms.nflush[0] = ms.nflush[1] = 0;
        }
        __syncthreads();

        // round rr holds tile elements [R - delta, R - delta + round) at buffer index
        // (element - (R - delta) + shift), shift chosen so bulk copies start 16-byte aligned
        auto shift_of = [&](uint32_t rr) -> uint32_t {
            return (uint32_t)((alo + (uint64_t)rr * round - delta) & (uint64_t)(q - 1u));
        };
        auto loc_ptr = [&](uint64_t loc) -> T* {
            return (loc & kLocPool) ? pool + (loc & ~kLocPool) : base + loc;
        };
        uint32_t carried[4] = {kNone, kNone, kNone, kNone};
        uint32_t carried_buf = 0;  // buffer of the carried elements
        uint32_t loads_issued = 0;  // I/O warp: rounds whose load has been issued

            // bookkeeping of round q: one lane per bucket; the (bucket, warp) counts in tb become
            // offsets from the start of the bucket's current chunk (below Bs: the staged chunk)
            auto book = [&](uint32_t q, uint16_t* tb) {
                const uint32_t R = q * round;
                const uint32_t par = q & 1u;
                const int64_t e_rd = (int64_t)R + round - delta;  // elements read through this round
                const uint32_t e_end = min(e_rd < (int64_t)r ? (uint32_t)e_rd : r, avail);
                const uint32_t F = min(H, b_pow2 ? e_end >> b_shift : a.fdB.div(e_end));
                for (uint32_t b0 = warp * 32u; b0 < k; b0 += kComputeThreads) {
                    const uint32_t b = b0 + lane;
                    const bool mine = b < k;
                    const uint32_t cur = mine ? run[b] : 0u;
                    // the open block's index and location, loaded beside the run length (the
                    // shared-memory round trips are the bookkeeping's latency)
                    const uint32_t ob_ld = mine ? oblk[b] : kNone;
                    const uint64_t oloc_ld = mine ? optr[b] : 0ull;
                    const uint32_t fill = bs_pow2 ? cur & (Bs - 1u) : cur % Bs;
                    uint32_t acc = fill;
                    if (mine) {
                        uint16_t* col = tb + b * S;
                        if constexpr (PIPE) {
                            // two entries per 32-bit word (the column starts 4-byte aligned), all
                            // loads first; with an odd count the last word's upper entry is padding
                            // that stays zero
                            constexpr uint32_t NW = cls_nwr(KC, W), NW2 = (NW + 1u) / 2u;
                            static_assert(cls_stride(KC, W) % 4u == 2u, "4-byte aligned columns");
                            uint32_t* col32 = reinterpret_cast<uint32_t*>(col);
                            uint32_t cv[NW2];
#pragma unroll
                            for (uint32_t j = 0; j < NW2; ++j) cv[j] = col32[j];
#pragma unroll
                            for (uint32_t j = 0; j < NW2; ++j) {
                                const uint32_t lo = cv[j] & 0xFFFFu;
                                const uint32_t hi = (2u * j + 1u < NW) ? cv[j] >> 16 : 0u;
                                const uint32_t a1 = acc + lo;
                                col32[j] = (acc & 0xFFFFu) | ((2u * j + 1u < NW ? a1 & 0xFFFFu : 0u) << 16);
                                acc = a1 + hi;
                            }
                        } else if constexpr (KB > 0) {
                            // loads first, in batches of eight: the stores cannot alias them,
                            // but the compiler cannot tell, and would wait for each load in turn
                            constexpr uint32_t NW = cls_nwr(KC, W);
#pragma unroll
                            for (uint32_t j0 = 0; j0 < NW; j0 += 8) {
                                uint32_t cv[8];
#pragma unroll
                                for (uint32_t j = 0; j < 8; ++j)
                                    if (j0 + j < NW) cv[j] = col[j0 + j];
#pragma unroll
                                for (uint32_t j = 0; j < 8; ++j)
                                    if (j0 + j < NW) {
                                        col[j0 + j] = (uint16_t)acc;
                                        acc += cv[j];
                                    }
                            }
                        } else {
                            for (uint32_t j = 0; j < nwr; ++j) {
                                const uint32_t c = col[j];
                                col[j] = (uint16_t)acc;
                                acc += c;
                            }
                        }
                    }
                    const uint32_t t = acc - fill, nr = cur + t;
                    const uint32_t c0 = bs_pow2 ? cur >> bs_shift : cur / Bs;
                    const uint32_t c1 = bs_pow2 ? nr >> bs_shift : nr / Bs;
                    const bool moves = mine && c1 > c0;  // a chunk completes: blocks receive data
                    uint32_t jlo = 0, jhi = 0, ob = kNone, jn = 0, nb = 0;
                    uint64_t oloc = 0;
                    if (moves) {
                        jlo = c0 / cpb;
                        jhi = (c1 - 1u) / cpb;
                        ob = ob_ld;
                        oloc = oloc_ld;
                        jn = ob == jlo ? jlo + 1u : jlo;
                        nb = jhi + 1u - jn;
                    }
                    // exclusive prefix of nb over the warp's buckets: nb is almost always 0 or 1, so
                    // ballots give it (their bits need no trip through the shared-memory unit, which
                    // the ranking warps keep busy); a shuffle scan where some bucket opened more
                    uint32_t ex, wtotal;
                    if (!__any_sync(0xffffffffu, nb > 2u)) {
                        const uint32_t m1 = __ballot_sync(0xffffffffu, nb >= 1u);
                        const uint32_t m2 = __ballot_sync(0xffffffffu, nb >= 2u);
                        ex = (uint32_t)__popc(m1 & lt_mask) + (uint32_t)__popc(m2 & lt_mask);
                        wtotal = (uint32_t)__popc(m1) + (uint32_t)__popc(m2);
                    } else {
                        ex = nb;
#pragma unroll
                        for (uint32_t d = 1; d < 32u; d <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xffffffffu, ex, d);
                            if (lane >= d) ex += y;
                        }
                        wtotal = __shfl_sync(0xffffffffu, ex, 31);
                        ex -= nb;
                    }
                    // whole blocks staged: completed blocks never outrun the read elements, so
                    // the frontier binds only past H (wrap piece) and a plain add is exact;
                    // chunks: a block is placed at its first chunk, so claim no slot past F
                    // the warp's flush-list entries and home slots: lane 0 issues both claims at
                    // once and one round of shuffles hands the bases out
                    const unsigned fl_mask = __ballot_sync(0xffffffffu, moves);
                    uint32_t hb0 = 0, lim = F, fl0 = 0;
                    if (lane == 0 && fl_mask) fl0 = atomicAdd(&ms.nflush[par], (uint32_t)__popc(fl_mask));
                    if (lane == 0 && wtotal) {
                        if (cpb == 1) {
                            hb0 = atomicAdd(&ms.home_next, wtotal);
                        } else {
                            uint32_t old = *reinterpret_cast<volatile uint32_t*>(&ms.home_next), tk = 0;
                            for (;;) {
                                tk = old < F ? min(wtotal, F - old) : 0u;
                                if (tk == 0) break;
                                const uint32_t prev = atomicCAS(&ms.home_next, old, old + tk);
                                if (prev == old) break;
                                old = prev;
                            }
                            hb0 = old;
                            lim = old + tk;
                        }
                    }
                    hb0 = __shfl_sync(0xffffffffu, hb0, 0);
                    lim = __shfl_sync(0xffffffffu, lim, 0);
                    fl0 = __shfl_sync(0xffffffffu, fl0, 0);
                    if (mine && t) {
                        rb[b] = cur;
                        run[b] = nr;
                    }
                    if (moves) {
                        const uint32_t hb = hb0 + ex;
                        const uint32_t tk = lim > hb ? min(nb, lim - hb) : 0u;
                        uint64_t pb = 0;
                        if (nb > tk) {
                            const uint64_t need = (uint64_t)(nb - tk) * B;
                            const uint64_t alloc = (need + a.pool_align - 1) / a.pool_align * a.pool_align;
                            pb = atomicAdd((unsigned long long*)a.pool_used, (unsigned long long)alloc);
                            if (pb + need > a.pool_cap) report(a.status, RIP_EWORKSPACE, 0x6202, pb);
                        }
                        auto locf = [&](uint32_t j) -> uint64_t {
                            if (j == ob) return oloc;
                            const uint32_t x = j - jn;
                            if (x < tk) return alo + (uint64_t)(hb + x) * B;
                            return kLocPool | (pb + (uint64_t)(x - tk) * B);
                        };
                        const uint64_t l0 = locf(jlo);
                        // the placement reads these only for a chunk that lies wholly inside the
                        // round (x >= Bs and c < c1): never unless the round crosses two chunk
                        // boundaries of the bucket (rare), so the stores are skipped otherwise
                        if (c1 >= c0 + 2u) {
                            jnew[b] = jn;
                            take[b] = tk;
                            hbase[b] = hb;
                            pbase[b] = pb;
                            jloc[b] = l0;
                        }
                        // the staged chunk c0 completes: its flush entry
                        flist[par * k + fl0 + (uint32_t)__popc(fl_mask & lt_mask)] =
                            (l0 + (uint64_t)(c0 % cpb) * Bs) | ((uint64_t)b << 48);
                        // blocks completed this round: slot words (home) or demoted records (pool)
                        const uint32_t jc0 = b_pow2 ? cur >> b_shift : a.fdB.div(cur);
                        const uint32_t jc1 = b_pow2 ? nr >> b_shift : a.fdB.div(nr);
                        for (uint32_t j = jc0; j < jc1; ++j) {
                            if (j >= (1u << kBlkBits)) report(a.status, RIP_EINVAL, 0x6203, j);
                            const uint64_t l = locf(j);
                            if (!(l & kLocPool)) {
                                const uint32_t h = b_pow2 ? (uint32_t)((l - alo) >> b_shift)
                                                          : a.fdB.div((uint32_t)(l - alo));
                                a.words[hs0 + h] = kWordOcc | (b << kBlkBits) | j;
                            } else {
                                if ((l & ~kLocPool) + B > a.pool_cap) continue;  // allocation failure, reported
                                const uint32_t rec = atomicAdd(&a.counters[2], 1u);
                                if (rec < a.dem_cap)
                                    a.dem[rec] = DemRec{tr.sp, tile, b, j, l & ~kLocPool};
                                else
                                    report(a.status, RIP_EWORKSPACE, 0x6204, rec);
                            }
                        }
                        if ((uint64_t)(jhi + 1u) * B > nr) {
                            oblk[b] = jhi;
                            optr[b] = locf(jhi);
                        } else {
                            oblk[b] = kNone;
                        }
                    }
                }
            };

            // the chunks that round pp's bookkeeping listed as complete go to their blocks, 16 bytes
            // (or one element) per thread, spread over many warps instead of queueing behind one
            // copy engine. The flushing warps are those on no critical path: with fewer ranking
            // warps than compute warps (k >= 512, 16-byte records) the warps that do not rank, while
            // the others rank; else the warps that do not book (one lane per bucket, on the round's
            // critical path) while the others book, or all warps when every warp books.
            const bool flush_early = !PIPE && nwr < kIoWarp;
            const uint32_t fw0 = flush_early ? nwr : (k < kComputeThreads ? k / 32u : 0u);  // first flushing warp
            const uint32_t fth = kComputeThreads - fw0 * 32u;  // flushing threads
            const uint32_t ftid = tid - fw0 * 32u;             // (wraps for the others)
            auto flush_chunks = [&](uint32_t pp) {
                if (warp < fw0) return;
                const uint32_t nf = ms.nflush[pp];
                const uint64_t* fl = flist + pp * k;
                if (flush_vec) {
                    const uint32_t vpc = Bs * (uint32_t)W / 16u;  // 16-byte words per chunk
                    const bool vpc_pow2 = (vpc & (vpc - 1u)) == 0;
                    const uint32_t vsh = log2_pow2(vpc);
                    for (uint32_t i = ftid; i < nf * vpc; i += fth) {
                        const uint32_t f = vpc_pow2 ? i >> vsh : i / vpc;
                        const uint32_t u = i - f * vpc;
                        const uint64_t e = fl[f];
                        const uint32_t b = (uint32_t)(e >> 48) & 0x3FFu;
                        const uint64_t loc = e & kEntLoc;
                        if ((loc & kLocPool) && (loc & ~kLocPool) + Bs > a.pool_cap) continue;  // reported
                        reinterpret_cast<uint4*>(loc_ptr(loc))[u] =
                            reinterpret_cast<const uint4*>(stage + (size_t)b * Bs)[u];
                    }
                } else {
                    for (uint32_t i = ftid; i < nf * Bs; i += fth) {
                        const uint32_t f = bs_pow2 ? i >> bs_shift : i / Bs;
                        const uint32_t u = i - f * Bs;
                        const uint64_t e = fl[f];
                        const uint32_t b = (uint32_t)(e >> 48) & 0x3FFu;
                        const uint64_t loc = e & kEntLoc;
                        if ((loc & kLocPool) && (loc & ~kLocPool) + Bs > a.pool_cap) continue;  // reported
                        loc_ptr(loc)[u] = stage[(size_t)b * Bs + u];
                    }
                }
            };

        if (io) {
            // ---------------------------------------------------------------- I/O warp
            // load of round rr into buffer (grc + rr) % nbuf: bulk copy for the aligned inside,
            // the lanes copy ragged ends and the rotation's wrap piece
            auto load = [&](uint32_t rr) {
                const uint32_t gr = grc + rr;
                loads_issued = rr + 1u;
                T* buf = bufs + (size_t)(gr % nbuf) * g.bufstride;
                const uint32_t R = rr * round;
                const uint32_t sh = shift_of(rr);
                const int64_t e0 = (int64_t)R - (int64_t)delta;  // element of buffer index `sh`
                const uint32_t e_lo = e0 > 0 ? (uint32_t)e0 : 0u;
                const int64_t e_end = e0 + (int64_t)round;
                const uint32_t e_hi = e_end < (int64_t)r ? (uint32_t)e_end : r;
                const uint32_t a_hi = min(e_hi, avail);
                uint32_t b_lo = e_lo, b_hi = e_lo;  // bulk part [b_lo, b_hi), inside the aligned piece
                if (a_hi > e_lo) {
                    const uint32_t mis = (uint32_t)((alo + e_lo) & (uint64_t)(q - 1u));
                    b_lo = e_lo + (mis ? q - mis : 0u);
                    b_hi = a_hi - (uint32_t)((alo + a_hi) & (uint64_t)(q - 1u));
                    if (b_hi <= b_lo || !a.vec16) b_lo = b_hi = e_lo;
                }
                for (uint32_t e = e_lo + lane; e < b_lo; e += 32u)
                    buf[(uint32_t)((int64_t)e - e0) + sh] = base[alo + e];
                for (uint32_t e = b_hi + lane; e < e_hi; e += 32u)
                    buf[(uint32_t)((int64_t)e - e0) + sh] = e < avail ? base[alo + e] : base[phys_index(Sp, lo + e)];
                __syncwarp();
                if (b_hi > b_lo) {
                    // pieces of kLoadPiece bytes, one per lane: several copies in flight fetch a round
                    // sooner than one long copy
                    const uint32_t bytes = (b_hi - b_lo) * (uint32_t)W;
                    if (lane == 0) mbar_arrive_expect_tx(&ms.full[gr % nbuf], bytes);
                    __syncwarp();
                    unsigned char* d0 = reinterpret_cast<unsigned char*>(buf + ((uint32_t)((int64_t)b_lo - e0) + sh));
                    const unsigned char* s0 = reinterpret_cast<const unsigned char*>(base + alo + b_lo);
                    for (uint32_t off = lane * kLoadPiece; off < bytes; off += 32u * kLoadPiece)
                        bulk_g2s(d0 + off, s0 + off, min(kLoadPiece, bytes - off), &ms.full[gr % nbuf]);
                } else if (lane == 0) {
                    mbar_arrive(&ms.full[gr % nbuf]);
                }
            };
            if constexpr (PIPE) {
                // pipelined rounds: after round rr is placed its buffer is free (the elements it
                // carries into the next round wait in registers), so round rr + nbuf loads into it.
                // (The chunk stores stay off this warp: a bulk copy issued after this thread's own
                // global stores was measured to wait for them.)
                for (uint32_t rr = 0; rr < nbuf && rr < nrounds; ++rr) load(rr);
                for (uint32_t rr = 0; rr < nrounds; ++rr) {
                    uint32_t ok = 1;
                    if (lane == 0) {
                        ok = mbar_wait(&ms.flush_ready, (frc + rr) & 1u, polls);
                        if (!ok) {
                            report(a.status, RIP_ETIMEOUT, 0x6208, rr);
                            ms.fail = 1;
                        } else if (ms.fail) {
                            ok = 0;
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    __syncwarp();  // lane 0's acquire covers the whole warp
                    if (!ok) break;
                    if (rr + nbuf < nrounds) load(rr + nbuf);
                }
            } else {
                for (uint32_t rr = 0; rr + 1 < nbuf && rr < nrounds; ++rr) load(rr);
                for (uint32_t rr = 0; rr < nrounds; ++rr) {
                    // round rr is placed: the buffer of round rr-1 is free (its carried elements are placed)
                    // (lane 0 decides for the warp: its wait, or a failure the compute warps recorded)
                    uint32_t ok = 1;
                    if (lane == 0) {
                        ok = mbar_wait(&ms.flush_ready, (frc + rr) & 1u, polls);
                        if (!ok) {
                            report(a.status, RIP_ETIMEOUT, 0x6208, rr);
                            ms.fail = 1;
                        } else if (ms.fail) {
                            ok = 0;
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    __syncwarp();  // lane 0's acquire covers the whole warp
                    if (!ok) break;
                    if (rr + nbuf - 1 < nrounds) load(rr + nbuf - 1);
                }
            }
            // after a failure: the loads still in flight land in this CTA's shared memory, so they
            // complete before the CTA leaves (the last load of each buffer; earlier ones were
            // consumed)
            if (ms.fail && lane == 0) {
                for (uint32_t j = loads_issued > nbuf ? loads_issued - nbuf : 0u; j < loads_issued; ++j) {
                    const uint32_t gr = grc + j;
                    mbar_wait(&ms.full[gr % nbuf], (gr / nbuf) & 1u);
                }
            }
            __syncwarp();
        } else if constexpr (PIPE) {
            // ---------------------------------------------------------------- compute warps, pipelined
            // iteration it: the rank warps rank round it while the bookkeeping warps book round it-1
            // (barrier X); then the rank warps place round it-1 (barrier Y).  The table of counts
            // alternates between two copies, so a round's offsets survive until it is placed.
            constexpr uint32_t NB = KC / 32u;  // bookkeeping warps: one lane per bucket
            const bool bookw = warp < NB;
            const uint32_t rw = warp - NB;  // rank index of a rank warp
            if (bookw) {
                for (uint32_t it = 0; it <= nrounds; ++it) {
                    if (it >= 1) book(it - 1, tbl + ((it - 1) & 1u) * k * S);
                    if (tid == 0) ms.cfail = ms.fail;  // one verdict for all compute warps
                    compute_sync();  // X
                    if (ms.cfail) {
                        if (tid == 0) mbar_arrive(&ms.flush_ready);  // lets the I/O warp see the failure
                        break;
                    }
                    // round it's flush list starts empty: the list of the same parity (round it-2)
                    // was written out before barrier X
                    if (tid == 0 && it < nrounds) ms.nflush[it & 1u] = 0;
                    // round it's input, placed after the next barrier X: thread 0 waits for it now,
                    // while the bookkeeping warps have nothing else to do (a failure reaches all
                    // compute warps through the verdict taken before that barrier)
                    if (tid == 0 && it < nrounds) {
                        const uint32_t gq = grc + it;
                        if (!mbar_wait(&ms.full[gq % nbuf], (gq / nbuf) & 1u, polls)) {
                            report(a.status, RIP_ETIMEOUT, 0x6207, gq);
                            ms.fail = 1;
                        }
                    }
                    if (it >= 1) {
                        compute_sync();  // Y
                        if (tid == 0) mbar_arrive(&ms.flush_ready);  // round it-1 is placed
                    }
                }
                // end of the tile: the rank warps write the last round's chunks out, then put the
                // carried elements in the stage (ms.cfail: the last verdict at X)
                if (!ms.cfail) compute_sync();
            } else {
                // a round's ranks (bucket | rank << 8, 0xffff: no position), two per word
                uint32_t pk_cur[2] = {0xffffffffu, 0xffffffffu}, pk_nxt[2] = {0xffffffffu, 0xffffffffu};
                uint32_t cmeta[4] = {kNone, kNone, kNone, kNone};  // carried element: bucket | position << 10
                T cval[4];                                          // and its value
                for (uint32_t it = 0; it <= nrounds; ++it) {
                    // round it-2's completed chunks (placed before the last barrier Y) leave the
                    // stage before round it-1 is placed
                    if (it >= 2) flush_chunks((it - 2u) & 1u);
                    if (it < nrounds) {
                        const uint32_t R = it * round;
                        uint16_t* tb = tbl + (it & 1u) * k * S;
                        uint32_t* mrow = masks + rw * 64u;  // 64 entries: the low six bucket bits
                        auto rankp = [&](auto in_c) {
                            constexpr bool IN = decltype(in_c)::value;
                            const uint4 words = group_philox(pk, L, Sp.o, Q0 + (R >> 2) + rw * 32u);
                            // the lane's four buckets (k <= 256: the top KB bits of each word) in one
                            // word, so a step needs one shuffle instead of four
                            const uint32_t pb = bucket_of(words.x, k) | (bucket_of(words.y, k) << 8) |
                                                (bucket_of(words.z, k) << 16) | (bucket_of(words.w, k) << 24);
                            const uint32_t v0 = R + rw * 128u + lane;
                            uint32_t e[4];
#pragma unroll
                            for (uint32_t s = 0; s < 4; ++s) {
                                const uint32_t v = v0 + 32u * s;
                                const bool valid = IN || (v >= delta && v - delta < r);
                                const uint32_t src = __shfl_sync(0xffffffffu, pb, (int)(8u * s + (lane >> 2)));
                                const uint32_t b = (src >> (8u * (lane & 3u))) & 0xFFu;
                                uint32_t* mk = mrow + (b & 63u);
                                if (valid) atomicOr(mk, 1u << lane);
                                uint32_t peers = bucket_peers_hi<KB, 6>(b, kbits);
                                __syncwarp();
                                uint16_t* c = tb + b * S + rw;
                                peers &= valid ? *mk : 0u;
                                const uint32_t pre = valid ? (uint32_t)*c : 0u;
                                __syncwarp();
                                if (valid && (peers & lt_mask) == 0) {
                                    *c = (uint16_t)(pre + (uint32_t)__popc(peers));
                                    *mk = 0u;
                                }
                                __syncwarp();
                                e[s] = valid ? (b | ((pre + (uint32_t)__popc(peers & lt_mask)) << 8)) : 0xffffu;
                            }
                            pk_nxt[0] = e[0] | (e[1] << 16);
                            pk_nxt[1] = e[2] | (e[3] << 16);
                        };
                        if (R >= delta && R + round <= rv)
                            rankp(BoolC<true>{});
                        else
                            rankp(BoolC<false>{});
                    }
                    compute_sync();  // X
                    if (ms.cfail) break;
                    if (it >= 1) {
                        // place round q = it-1, the elements carried from round q-1 first
                        const uint32_t q = it - 1u, gq = grc + q;
                        const T* vb = bufs + (size_t)(gq % nbuf) * g.bufstride;
                        const uint32_t sh = shift_of(q);
                        uint16_t* tb = tbl + (q & 1u) * k * S;
#pragma unroll
                        for (uint32_t s = 0; s < 4; ++s)
                            if (cmeta[s] != kNone) stage[(size_t)(cmeta[s] & 0x3FFu) * Bs + (cmeta[s] >> 10)] = cval[s];
#pragma unroll
                        for (uint32_t s = 0; s < 4; ++s) {
                            const uint32_t e = (pk_cur[s >> 1] >> (16u * (s & 1u))) & 0xffffu;
                            cmeta[s] = kNone;
                            if (e == 0xffffu) continue;
                            const uint32_t b = e & 0xFFu, rk = e >> 8;
                            const uint32_t x = tb[b * S + rw] + rk;  // offset from the current chunk's start
                            const uint32_t bi = rw * 128u + 32u * s + lane + sh;
                            if (x < Bs) {
                                stage[(size_t)b * Bs + x] = vb[bi];
                                continue;
                            }
                            const uint32_t qx = bs_pow2 ? x >> bs_shift : x / Bs;  // chunks past the current one
                            const uint32_t pos = x - qx * Bs;
                            const uint32_t rbb = rb[b], run_b = run[b];
                            const uint32_t c0 = bs_pow2 ? rbb >> bs_shift : rbb / Bs;
                            const uint32_t c1 = bs_pow2 ? run_b >> bs_shift : run_b / Bs;
                            const uint32_t c = c0 + qx;
                            if (c < c1) {  // the whole chunk lies in this round: straight to its block
                                const uint32_t j = c / cpb, jlo = c0 / cpb;
                                uint64_t l;
                                if (j == jlo) {
                                    l = jloc[b];
                                } else {
                                    const uint32_t xj = j - jnew[b], tk = take[b];
                                    l = xj < tk ? alo + (uint64_t)(hbase[b] + xj) * B
                                                : kLocPool | (pbase[b] + (uint64_t)(xj - tk) * B);
                                }
                                if ((l & kLocPool) && (l & ~kLocPool) + B > a.pool_cap) continue;  // reported at allocation
                                loc_ptr(l + (uint64_t)(c % cpb) * Bs)[pos] = vb[bi];
                            } else {
                                cmeta[s] = b | (pos << 10);
                                cval[s] = vb[bi];
                            }
                        }
                        // the warp's column of this copy of the table is read only by the warp itself
                        __syncwarp();
                        for (uint32_t b = lane; b < k; b += 32u) tb[b * S + rw] = 0;
                        compute_sync();  // Y
                    }
                    pk_cur[0] = pk_nxt[0];
                    pk_cur[1] = pk_nxt[1];
                }
                if (!ms.cfail) {
                    flush_chunks((nrounds - 1u) & 1u);
                    compute_sync();
#pragma unroll
                    for (uint32_t s = 0; s < 4; ++s)
                        if (cmeta[s] != kNone) stage[(size_t)(cmeta[s] & 0x3FFu) * Bs + (cmeta[s] >> 10)] = cval[s];
                }
            }
        } else {
            // ---------------------------------------------------------------- compute warps
            for (uint32_t rr = 0; rr < nrounds; ++rr) {
                const uint32_t R = rr * round;
                const uint32_t gr = grc + rr;
                const uint32_t par = rr & 1u;
                if (tid == 0) ms.nflush[par] = 0;
                // the previous round's completed chunks leave the stage before this round places
                // (barriers A and B lie between)
                if (flush_early && rr > 0) flush_chunks(par ^ 1u);

                // rank: lanes of a step with the same bucket read the warp's running count
                // together, the lowest of them writes it back advanced by their number
                uint32_t packed[4] = {kNone, kNone, kNone, kNone};
                // IN: every position of the round is valid (all rounds but a tile's first and last)
                auto rank4 = [&](auto in_c) {
                    constexpr bool IN = decltype(in_c)::value;
                    const uint4 words = group_philox(pk, L, Sp.o, Q0 + (R >> 2) + warp * 32u);
                    const uint32_t v0 = R + warp * 128u + lane;
#pragma unroll
                    for (uint32_t s = 0; s < 4; ++s) {
                        const uint32_t v = v0 + 32u * s;
                        const bool valid = IN || (v >= delta && v - delta < r);
                        const uint32_t b = bucket_of(group_step_word(words, s), k);
                        // lanes with the same bucket: the low five bits through the warp's mask
                        // row (one shared atomic OR per lane), the higher ones by ballot -- on
                        // GB300 a ballot costs more issue time than the shared-memory round trip
                        uint32_t* mk = masks + warp * 32u + (b & 31u);
                        if (valid) atomicOr(mk, 1u << lane);
                        uint32_t peers = bucket_peers_hi<KB>(b, kbits);
                        __syncwarp();
                        uint16_t* c = tbl + b * S + warp;
                        peers &= valid ? *mk : 0u;
                        const uint32_t pre = valid ? (uint32_t)*c : 0u;
                        __syncwarp();
                        if (valid && (peers & lt_mask) == 0) {
                            *c = (uint16_t)(pre + (uint32_t)__popc(peers));
                            *mk = 0u;  // every bucket sharing the entry clears it: same value
                        }
                        __syncwarp();
                        if (valid) packed[s] = b | ((pre + (uint32_t)__popc(peers & lt_mask)) << 10);
                    }
                };
                if (warp < nwr) {
                    if (R >= delta && R + round <= rv)
                        rank4(BoolC<true>{});
                    else
                        rank4(BoolC<false>{});
                }
                compute_sync();  // A
                // the previous round's completed chunks leave the stage before this round places
                // (barrier B lies between), while the bookkeeping warps work
                if (!flush_early && rr > 0) flush_chunks(par ^ 1u);

                book(rr, tbl);
                // this round's input is loaded
                if (tid == 0) {
                    if (!mbar_wait(&ms.full[gr % nbuf], (gr / nbuf) & 1u, polls)) {
                        report(a.status, RIP_ETIMEOUT, 0x6207, gr);
                        ms.fail = 1;
                    }
                    ms.cfail = ms.fail;  // one verdict for all compute warps (ms.fail may change later)
                }
                compute_sync();  // B
                if (ms.cfail) {
                    if (tid == 0) mbar_arrive(&ms.flush_ready);  // lets the I/O warp see the failure
                    break;
                }

                // place: carried elements of the previous round, then this round's
                {
                    const T* cb = bufs + (size_t)carried_buf * g.bufstride;
#pragma unroll
                    for (uint32_t s = 0; s < 4; ++s) {
                        const uint32_t cv = carried[s];
                        if (cv == kNone) continue;
                        const uint32_t bi = cv & 0x1FFFu, b = (cv >> 13) & 0x3FFu, pos = cv >> 23;
                        stage[(size_t)b * Bs + pos] = cb[bi];
                    }
                }
                const T* vb = bufs + (size_t)(gr % nbuf) * g.bufstride;
                const uint32_t sh = shift_of(rr);
#pragma unroll
                for (uint32_t s = 0; s < 4; ++s) {
                    const uint32_t p = packed[s];
                    carried[s] = kNone;
                    if (p == kNone) continue;
                    const uint32_t b = p & 0x3FFu, rk = p >> 10;
                    const uint32_t x = tbl[b * S + warp] + rk;  // offset from the current chunk's start
                    const uint32_t bi = warp * 128u + 32u * s + lane + sh;
                    if (x < Bs) {
                        stage[(size_t)b * Bs + x] = vb[bi];
                        continue;
                    }
                    const uint32_t qx = bs_pow2 ? x >> bs_shift : x / Bs;  // chunks past the current one
                    const uint32_t pos = x - qx * Bs;
                    const uint32_t rbb = rb[b], run_b = run[b];
                    const uint32_t c0 = bs_pow2 ? rbb >> bs_shift : rbb / Bs;
                    const uint32_t c1 = bs_pow2 ? run_b >> bs_shift : run_b / Bs;
                    const uint32_t c = c0 + qx;
                    if (c < c1) {  // the whole chunk lies in this round: straight to its block
                        const uint32_t j = c / cpb, jlo = c0 / cpb;
                        uint64_t l;
                        if (j == jlo) {
                            l = jloc[b];
                        } else {
                            const uint32_t xj = j - jnew[b], tk = take[b];
                            l = xj < tk ? alo + (uint64_t)(hbase[b] + xj) * B
                                        : kLocPool | (pbase[b] + (uint64_t)(xj - tk) * B);
                        }
                        if ((l & kLocPool) && (l & ~kLocPool) + B > a.pool_cap) continue;  // reported at allocation
                        loc_ptr(l + (uint64_t)(c % cpb) * Bs)[pos] = vb[bi];
                    } else {
                        carried[s] = bi | (b << 13) | (pos << 23);
                    }
                }
                carried_buf = gr % nbuf;
                // the warp's column of the table is read only by the warp itself: clear it
                __syncwarp();
                if (warp < nwr)
                    for (uint32_t b = lane; b < k; b += 32u) tbl[b * S + warp] = 0;
                compute_sync();  // C
                if (tid == 0) mbar_arrive(&ms.flush_ready);
            }
            // end of the tile: the last round's chunks go out, then the carried elements take the
            // stage (ms.cfail is the verdict every compute thread saw at the last barrier B)
            if (!ms.cfail) {
                if (nrounds > 0) flush_chunks((nrounds - 1u) & 1u);
                compute_sync();
                const T* cb = bufs + (size_t)carried_buf * g.bufstride;
#pragma unroll
                for (uint32_t s = 0; s < 4; ++s) {
                    const uint32_t cv = carried[s];
                    if (cv == kNone) continue;
                    const uint32_t bi = cv & 0x1FFFu, b = (cv >> 13) & 0x3FFu, pos = cv >> 23;
                    stage[(size_t)b * Bs + pos] = cb[bi];
                }
            }
        }
        grc += nrounds;
        frc += nrounds;
        __syncthreads();
        if (ms.fail) break;  // a copy or a hand-off did not arrive: reported, the level's output is void
        {
            // tails of every bucket -> pool, in bucket order; k <= 2 * blockDim.x
            const uint32_t i0 = 2 * tid, i1 = 2 * tid + 1;
            const uint32_t r0 = i0 < k ? a.fdB.mod(run[i0]) : 0, r1 = i1 < k ? a.fdB.mod(run[i1]) : 0;
            uint32_t total;
            const uint32_t ex = block_exclusive_scan<uint32_t>(r0 + r1, ms.scan, &total);
            if (i0 < k) jnew[i0] = ex;  // reused: tail offset of the bucket
            if (i1 < k) jnew[i1] = ex + r0;
            if (tid == 0) {
                const uint64_t alloc = ((uint64_t)total + a.pool_align - 1) / a.pool_align * a.pool_align;
                const uint64_t pb = atomicAdd((unsigned long long*)a.pool_used, (unsigned long long)alloc);
                if (pb + total > a.pool_cap) report(a.status, RIP_EWORKSPACE, 0x6205, pb);
                ms.pool_base = pb;
            }
            __syncthreads();
            const uint64_t pb = ms.pool_base;
            const uint32_t nwarps = blockDim.x >> 5;
            for (uint32_t b = warp; b < k; b += nwarps) {
                const uint32_t nr = run[b];
                const uint32_t Rt = a.fdB.mod(nr);
                const uint32_t in_stage = bs_pow2 ? nr & (Bs - 1u) : nr % Bs;
                const uint32_t in_block = Rt - in_stage;  // elements already in the open block
                const uint64_t ol = optr[b];
                const bool ob_ok = !in_block || !(ol & kLocPool) || (ol & ~kLocPool) + B <= a.pool_cap;
                if (pb + total <= a.pool_cap && ob_ok) {
                    const T* obp = in_block ? loc_ptr(ol) : nullptr;
                    for (uint32_t j = lane; j < Rt; j += 32u)
                        pool[pb + jnew[b] + j] = j < in_block ? obp[j] : stage[(size_t)b * Bs + (j - in_block)];
                }
                if (lane == 0 && oblk[b] != kNone && !(optr[b] & kLocPool)) {
                    // an open block in a home slot held a part of the tail only: that slot is empty
                    const uint64_t l = optr[b];
                    const uint32_t h = b_pow2 ? (uint32_t)((l - alo) >> b_shift) : a.fdB.div((uint32_t)(l - alo));
                    a.words[hs0 + h] = 0u;
                }
            }
            for (uint32_t b = tid; b < k; b += blockDim.x) a.C[(uint64_t)tile * k + b] = run[b];
            const uint32_t used = min(ms.home_next, H);
            if (tid == 0) a.tinfo[tile] = TileInfo{hs0, pb, used, H};
            __syncthreads();
        }
    }
}

}  // namespace

bool classify_config(uint32_t k, uint32_t B, uint32_t w, ClsCfg* out) {
    if (k < 2 || k > kMaxK || (k & (k - 1)) || B < 1) return false;
    ClsCfg c{};
    c.nwr = cls_nwr(k, w);
    c.S = cls_stride(k, w);
    c.round = c.nwr * 128u;
    c.q = w >= 16 ? 1u : 16u / w;
    c.bufstride = (c.round + c.q + 15u) / 16u * 16u;  // elements; keeps every buffer 16-byte aligned
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    size_t off = a16(sizeof(ClsMisc));
    c.off_tbl = (uint32_t)off;
    off = a16(off + (size_t)k * c.S * 2 * (cls_pipe(k, w) ? 2u : 1u));
    c.off_u32 = (uint32_t)off;
    off = a16(off + (size_t)k * 6 * 4);
    c.off_u64 = (uint32_t)off;
    off = a16(off + (size_t)k * 3 * 8);
    c.off_flist = (uint32_t)off;
    off = a16(off + (size_t)k * 2 * 8);
    c.off_mask = (uint32_t)off;
    off = a16(off + (size_t)c.nwr * (cls_pipe(k, w) ? 64 : 32) * 4);  // mask rows
    const size_t fixed = off;
    const size_t buf_bytes = a16((size_t)c.bufstride * w);
    uint32_t best_d = 0, best_nbuf = 0;
    for (uint32_t nbuf = cls_pipe(k, w) ? 2u : 3u; nbuf >= 2; --nbuf) {  // pipelined: two (see the kernel)
        if (fixed + nbuf * buf_bytes >= kSmemOptin) continue;
        const size_t rem = kSmemOptin - fixed - nbuf * buf_bytes;
        uint32_t d = 0;
        for (uint32_t x = std::min<uint32_t>(B, 512u); x >= 1; --x)
            if (B % x == 0 && (size_t)k * x * w <= rem) {
                d = x;
                break;
            }
        // prefer whole blocks in shared memory (no pool blocks for open blocks), then more buffers
        if (d > best_d) {
            best_d = d;
            best_nbuf = nbuf;
        }
    }
    if (!best_d) return false;
    c.Bs = best_d;
    c.cpb = B / best_d;
    c.nbuf = best_nbuf;
    c.off_stage = (uint32_t)fixed;
    c.off_buf = (uint32_t)a16(fixed + (size_t)k * c.Bs * w);
    c.bytes = (uint32_t)(c.off_buf + c.nbuf * buf_bytes);
    if (c.bytes > kSmemOptin) return false;
    *out = c;
    return true;
}

template <int W, int KB>
static cudaError_t launch_cls(const LevelArgs& a, uint32_t num_sms, cudaStream_t s) {
    const int smem = (int)a.cls.bytes;
    cudaError_t err = ensure_dyn_smem(reinterpret_cast<const void*>(classify_kernel<W, KB>), smem);
    if (err != cudaSuccess) return err;
    classify_kernel<W, KB><<<num_sms, kClassifyThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_cls_w(const LevelArgs& a, uint32_t num_sms, cudaStream_t s) {
    switch (a.k) {  // the common bucket counts get kernels with k fixed at compile time
        case 64: return launch_cls<W, 6>(a, num_sms, s);
        case 256: return launch_cls<W, 8>(a, num_sms, s);
        case 1024: return launch_cls<W, 10>(a, num_sms, s);
        default: return launch_cls<W, 0>(a, num_sms, s);
    }
}

cudaError_t launch_classify(const LevelArgs& a, uint32_t w, uint32_t num_sms, cudaStream_t s) {
    ProfScope p("classify", s);
    switch (w) {
        case 4: return launch_cls_w<4>(a, num_sms, s);
        case 8: return launch_cls_w<8>(a, num_sms, s);
        default: return launch_cls_w<16>(a, num_sms, s);
    }
}

}  // namespace rip
