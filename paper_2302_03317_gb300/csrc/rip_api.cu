// rip_api.cu -- host side of the C ABI: argument and plan validation, the
// device workspace layout, and the level-synchronous driver of the recursion
// (Sec. 3.2: scatter, then recurse into every bucket; Sec. 4: the buckets of a
// level are independent, so one launch processes all of them).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rip_internal.cuh"

namespace rip {

__device__ Status g_status;  // device status word of this library, per device

// ----------------------------------------------------------------- kernel timing
namespace {
struct ProfRec {
    const char* name;
    cudaEvent_t start, stop;
};
struct Profiler {
    bool on = false;
    std::vector<ProfRec> open;  // recorded, not yet folded into totals
    std::vector<cudaEvent_t> spare;
    std::vector<const char*> stack;
    std::vector<cudaEvent_t> start_stack;
    struct Tot {
        std::string name;
        uint64_t launches = 0;
        double ms = 0;
    };
    std::vector<Tot> totals;
    cudaEvent_t get() {
        if (!spare.empty()) {
            cudaEvent_t e = spare.back();
            spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void fold() {
        for (ProfRec& r : open) {
            float ms = 0;
            if (cudaEventSynchronize(r.stop) == cudaSuccess && cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
                auto it = std::find_if(totals.begin(), totals.end(), [&](const Tot& t) { return t.name == r.name; });
                if (it == totals.end()) {
                    totals.push_back(Tot{r.name, 0, 0});
                    it = totals.end() - 1;
                }
                it->launches += 1;
                it->ms += ms;
            }
            spare.push_back(r.start);
            spare.push_back(r.stop);
        }
        open.clear();
        std::sort(totals.begin(), totals.end(), [](const Tot& x, const Tot& y) { return x.name < y.name; });
    }
};
Profiler g_prof;
}  // namespace

cudaError_t ensure_dyn_smem(const void* func, int bytes) {
    static std::mutex m;
    static std::vector<std::pair<std::pair<int, const void*>, int>> set;  // (device, kernel) -> bytes
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(m);
    for (auto& e : set)
        if (e.first.first == dev && e.first.second == func) {
            if (e.second >= bytes) return cudaSuccess;
            err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (err == cudaSuccess) e.second = bytes;
            return err;
        }
    err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (err == cudaSuccess) set.push_back({{dev, func}, bytes});
    return err;
}

void prof_begin(const char* name, cudaStream_t s) {
    if (!g_prof.on) return;
    cudaEvent_t e = g_prof.get();
    cudaEventRecord(e, s);
    g_prof.stack.push_back(name);
    g_prof.start_stack.push_back(e);
}

void prof_end(cudaStream_t s) {
    if (!g_prof.on || g_prof.stack.empty()) return;
    cudaEvent_t e = g_prof.get();
    cudaEventRecord(e, s);
    g_prof.open.push_back(ProfRec{g_prof.stack.back(), g_prof.start_stack.back(), e});
    g_prof.stack.pop_back();
    g_prof.start_stack.pop_back();
    if (g_prof.open.size() > 4096) g_prof.fold();  // bounded event count
}

namespace {

constexpr uint32_t kMediumGrid = 16;  // CTAs of the medium solver when medium subproblems are expected
constexpr uint32_t kParkAfter = 256;  // chain steps before the permutation parks a block

struct LevelCaps {
    uint32_t big = 0;       // subproblems that may run in place
    uint32_t wave = 0;      // of which one wave holds at most this many
    uint32_t waves = 0;
    uint64_t tiles = 0;     // per wave
    uint64_t pairs = 0;     // tiles x k
    uint64_t pool = 0;      // elements, per wave
    uint64_t dem = 0;
};

struct Layout {
    size_t total = 0;
    size_t cstatus, arrays, lists_big0, lists_big1, small, medium, bigfy, counts, counters, pool_used;
    size_t tiles, sched, sp_tile_begin, segs, C, FBc, TLc, tinfo, child, words, pool, dem, parks, mscratch;
    uint32_t big_cap, small_cap, medium_cap, bigfy_cap, tile_cap, dem_cap, park_cap, levels, wave_cap;
    uint32_t medium_grid;
    uint64_t pair_cap, child_cap, pool_cap, slot_cap;
    uint32_t wave[64], waves[64];  // per level: subproblems per wave, waves
    uint32_t small_max_m;
    uint64_t aux_bytes;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t small_max_m_for(uint32_t w) {
    const size_t fixed = small_fixed_smem();
    const size_t m = (kSmemOptin - fixed - 16) / (4 + w);  // 16: alignment slack of D
    return (uint32_t)std::min<size_t>(m & ~size_t(7), kMediumMaxM);
}

DevPlan to_dev(const rip_plan& p) {
    DevPlan d{};
    d.num_levels = p.num_levels;
    d.cap = p.max_levels ? p.max_levels : kDepthCap;
    d.base = p.base;
    for (uint32_t l = 0; l < p.num_levels; ++l) {
        d.k[l] = p.level[l].k;
        d.B[l] = p.level[l].block;
        d.T[l] = p.level[l].tile;
    }
    return d;
}

bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

int validate_plan(const rip_plan& p, uint32_t w) {
    if (p.num_levels < 1 || p.num_levels > RIP_MAX_LEVEL_PARAMS) return RIP_EINVAL;
    if (p.base < 1 || p.base > 0xFFFFFFFFull) return RIP_EINVAL;
    if (p.max_levels > kDepthCap) return RIP_EINVAL;
    for (uint32_t l = 0; l < p.num_levels; ++l) {
        const rip_level_params& q = p.level[l];
        if (!pow2(q.k) || q.k < 2 || q.k > kMaxK) return RIP_EINVAL;
        if (q.block < 1 || q.tile < q.block || q.tile % q.block) return RIP_EINVAL;
        ClsCfg cc;
        if (!classify_config(q.k, q.block, w, &cc)) return RIP_EINVAL;
        if (permute_threads(q.block, w) == 0) return RIP_EINVAL;  // two block slots per group must fit
        if (l > 0 && p.level[l - 1].block % q.block) return RIP_EINVAL;  // slot grids must nest
    }
    return RIP_OK;
}

bool valid_w(uint32_t w) { return w == 4 || w == 8 || w == 16; }

// Host check of the invariant-division constants against plain division.
bool fastdiv_ok(const FastDiv& f) {
    const uint32_t d = f.d;
    const uint32_t ns[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d - 1u, 2u * d, 12345678u, 0x7fffffffu,
                           0x80000000u, 0xfffffffeu, 0xffffffffu, d * 1000u + 7u};
    for (uint32_t n : ns) {
        const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
        const uint32_t q = (t + ((n - t) >> f.s1)) >> f.s2;
        if (q != n / d) return false;
    }
    return true;
}

// Expected-size model of the recursion used to size the workspace.  A level
// can hold subproblems too large for one SM when mu_L + 10 sqrt(mu_L) + 64
// reaches the smallest size that must run in place (mu_L = n / prod k; a
// subproblem size is Binomial(n, 1/prod k), so larger deviations have
// probability below e^-50 each).
// Device-side capacity checks report RIP_EWORKSPACE if the model is exceeded.
Layout make_layout(const std::vector<uint64_t>& ns, uint32_t w, const rip_plan& p) {
    Layout L{};
    const DevPlan dp = to_dev(p);
    L.small_max_m = small_max_m_for(w);
    uint64_t nmax = 0, nsum = 0;
    for (uint64_t n : ns) {
        nmax = std::max(nmax, n);
        nsum += n;
    }
    const uint32_t narr = (uint32_t)ns.size();

    // smallest subproblem that runs in place at level lev
    auto inplace_min_at = [&](uint32_t lev) -> uint64_t {
        uint64_t im = (uint64_t)kMediumMaxM + 1;
        if (!small_solver_can_scatter(dp, kMediumMaxM, lev)) {  // eligibility is monotone in m
            uint64_t lo = 1, hi = kMediumMaxM;                    // can(lo) or lo == 1, !can(hi)
            while (hi - lo > 1) {
                const uint64_t mid = (lo + hi) / 2;
                if (small_solver_can_scatter(dp, mid, lev)) lo = mid; else hi = mid;
            }
            im = hi;
        }
        return std::max<uint64_t>(im, dp.base + 1);
    };
    // The slot table holds the segments of one wave.  Level 0 runs every root at once; deeper
    // levels run their subproblems in waves that fit the same table.
    uint64_t slot_cap = 64;
    {
        const uint64_t B0 = p.level[dp.idx(0)].block, im0 = inplace_min_at(0);
        uint64_t s0 = 0;
        for (uint64_t n : ns)
            if (n >= im0) s0 += align_up((n + B0 - 1) / B0 + 1, 64);
        slot_cap = std::max<uint64_t>(slot_cap, s0);
    }

    // Subproblems above the shared-memory limit (medium solver) or the on-SM limit (large
    // leaves) are rare: a child size is Binomial(m, 1/k), whose upper tail beyond t = mu + d
    // is at most exp(-d^2 / (2 (mu + d/3))) (Bernstein).  Their lists are sized by the
    // expected count with a wide margin, never beyond the count that fits the input.
    auto tail = [](double mu, double t) {
        if (t <= mu) return 1.0;
        const double d = t - mu;
        return std::exp(-d * d / (2.0 * (mu + d / 3.0)));
    };
    // lower tail: P(size <= t) for t below the mean mu is at most exp(-(mu - t)^2 / (2 mu)) (Chernoff)
    auto lower = [](double mu, double t) {
        if (t >= mu) return 1.0;
        const double d = mu - t;
        return std::exp(-d * d / (2.0 * mu));
    };
    double e_med = 0, e_big = 0;
    for (uint64_t n : ns) {
        if (n > L.small_max_m && n <= kMediumMaxM) e_med += 1;
        if (n > kMediumMaxM) e_big += 1;
    }
    std::vector<LevelCaps> caps;
    uint64_t prodk = 1;
    uint64_t small_children = narr, bigfy_total = narr, max_children = 0;
    for (uint32_t lev = 0; lev < dp.cap && lev < 64; ++lev) {
        const uint32_t li = dp.idx(lev);
        const uint32_t k = p.level[li].k, B = p.level[li].block;
        const uint64_t T = p.level[li].tile;
        const uint64_t inplace_min = inplace_min_at(lev);
        // per array: expected size at this level; count subproblems that may run in place
        uint64_t big = 0, tiles_all = 0;
        for (uint64_t n : ns) {
            if (n < inplace_min) continue;
            // a subproblem size at level L is Binomial(n, 1/prod k): mean mu, sd <= sqrt(mu)
            const double mu = (double)n / (double)prodk;
            if (mu + 10.0 * std::sqrt(mu) + 64.0 < (double)inplace_min) continue;
            const uint64_t cnt = std::min<uint64_t>(prodk, n / inplace_min);
            big += std::max<uint64_t>(cnt, 1);
            tiles_all += n / T + std::max<uint64_t>(cnt, 1);
        }
        if (big == 0) break;
        const double mu = (double)nmax / (double)prodk;
        const double m_sub = lev == 0 ? (double)nmax : std::min((double)nmax, mu + 10.0 * std::sqrt(mu) + 64.0);
        const uint64_t per_sub = align_up((uint64_t)(m_sub / B) + 3, 64);  // slots of one subproblem
        LevelCaps c;
        c.big = (uint32_t)std::min<uint64_t>(big + 16, 0xffffffffull);
        if (lev == 0) {
            c.wave = c.big;
        } else {
            slot_cap = std::max(slot_cap, per_sub);
            const uint64_t wmax = std::max<uint64_t>(1, std::min<uint64_t>(c.big, slot_cap / per_sub));
            const uint64_t nw = (c.big + wmax - 1) / wmax;
            c.wave = (uint32_t)((c.big + nw - 1) / nw);  // balanced waves
        }
        c.waves = (c.big + c.wave - 1) / c.wave;
        const uint64_t tiles_per_sub = (uint64_t)std::ceil(m_sub / (double)T);  // m_sub bounds every size
        c.tiles = std::min<uint64_t>(tiles_all, (uint64_t)c.wave * tiles_per_sub) + 16;
        c.pairs = c.tiles * k;
        // tails: (B-1)/2 per (tile, bucket) on average when counts are >> B, with a
        // Hoeffding margin; otherwise every tile-bucket may be a tail
        const double mu_tile = std::min<double>((double)T, m_sub);
        const double mu_c = mu_tile / k;
        const double pairs = (double)c.pairs;
        const double wave_elems = std::min((double)nsum, m_sub * c.wave);
        double tails;
        if (mu_c >= 4.0 * B)
            tails = pairs * (B - 1) / 2.0 * 1.05 + 20.0 * B * std::sqrt(pairs) + 4.0 * B * k;
        else
            tails = std::min<double>(pairs * (B - 1), wave_elems + B);
        // demoted blocks: at most one per (subproblem, bucket) plus two per subproblem.
        // With counts >> B the tail total of a bucket is (close to) uniform mod B, so a
        // bucket's last block is demoted with probability <= 1/2: Hoeffding margin.
        const double dem_worst = std::min<double>((double)c.wave * (k + 2), wave_elems / B + c.wave * 2.0);
        const double pairs_sp = (double)c.wave * k;
        const double dem_blocks = mu_c >= 4.0 * B
                                      ? std::min(dem_worst, pairs_sp / 2.0 + 20.0 * std::sqrt(pairs_sp) + 2.0 * c.wave)
                                      : dem_worst;
        c.dem = (uint64_t)dem_worst + 16;
        c.pool = (uint64_t)(tails + dem_blocks * B) + 64;
        // chunked staging: a block's location is taken at its first chunk, from the pool while
        // no read home slot is free -- at most k (1 - Bs/B) + 1 such blocks per tile
        ClsCfg cc{};
        if (classify_config(k, B, w, &cc) && cc.cpb > 1) {
            const uint64_t per_tile = (uint64_t)k * (cc.cpb - 1) / cc.cpb + 1;
            c.pool += c.tiles * per_tile * B;
            c.dem += c.tiles * per_tile;
        }
        max_children = std::max<uint64_t>(max_children, (uint64_t)c.big * k);
        const double mu_child = (double)nmax / ((double)prodk * k);
        // medium children: above the on-SM limit and at most kMediumMaxM (larger ones run in place)
        e_med += (double)c.big * k * std::min(tail(mu_child, (double)L.small_max_m), lower(mu_child, (double)kMediumMaxM));
        e_big += (double)c.big * k * tail(mu_child, (double)kMediumMaxM);
        caps.push_back(c);
        small_children += (uint64_t)c.big * k;
        bigfy_total += (uint64_t)c.big * k;
        prodk = std::min<uint64_t>(prodk * k, (uint64_t)1 << 62);
    }
    L.slot_cap = slot_cap;
    L.levels = (uint32_t)caps.size();
    uint32_t kmax = 2;
    for (uint32_t l = 0; l < p.num_levels; ++l) kmax = std::max(kmax, p.level[l].k);
    for (uint32_t l = 0; l < L.levels; ++l) {
        const LevelCaps& c = caps[l];
        L.wave[l] = c.wave;
        L.waves[l] = c.waves;
        L.big_cap = std::max(L.big_cap, c.big);
        L.wave_cap = std::max(L.wave_cap, c.wave);
        L.tile_cap = (uint32_t)std::max<uint64_t>(L.tile_cap, c.tiles);
        // each tile's tails and each demoted block are separate 16-byte-rounded allocations
        L.pool_cap = std::max(L.pool_cap, c.pool + (c.tiles + c.dem) * (16 / std::min<uint32_t>(w, 16)));
        L.dem_cap = (uint32_t)std::max<uint64_t>(L.dem_cap, c.dem);
    }
    const uint64_t per_level_small = std::max<uint64_t>(narr, max_children);
    L.small_cap = (uint32_t)std::min<uint64_t>(per_level_small + 16, 0x7fffffffull);
    const double det_med = (double)nsum / (L.small_max_m + 1.0) + narr + 16.0;
    const double det_big = (double)nsum / (kMediumMaxM + 1.0) + narr + 16.0;
    L.medium_cap = (uint32_t)std::min<double>({det_med, e_med + 10.0 * std::sqrt(e_med) + 64.0, (double)L.small_cap});
    L.bigfy_cap = (uint32_t)std::min<double>({det_big, e_big + 10.0 * std::sqrt(e_big) + 64.0, (double)bigfy_total + 16.0});
    L.medium_grid = e_med < 4.0 ? 2u : kMediumGrid;
    if (L.big_cap == 0) L.big_cap = 1;
    if (L.wave_cap == 0) L.wave_cap = 1;
    if (L.tile_cap == 0) L.tile_cap = 1;
    // any level may index (tile, bucket) and (subproblem, bucket) tables with the largest k
    L.pair_cap = (uint64_t)L.tile_cap * kmax;
    L.child_cap = (uint64_t)L.wave_cap * kmax;

    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return o;
    };
    L.cstatus = take(sizeof(Status));
    L.arrays = take(sizeof(ArrayDesc) * narr);
    L.lists_big0 = take(sizeof(Sub) * L.big_cap);
    L.lists_big1 = take(sizeof(Sub) * L.big_cap);
    L.small = take(sizeof(Sub) * L.small_cap);
    L.medium = take(sizeof(Sub) * L.medium_cap);
    L.bigfy = take(sizeof(Sub) * L.bigfy_cap);
    L.counts = take(sizeof(uint32_t) * 8);
    L.counters = take(sizeof(uint32_t) * 16);
    L.pool_used = take(sizeof(uint64_t));
    const size_t meta_start = off;
    L.tiles = take(sizeof(TileRef) * L.tile_cap);
    L.sched = take(sizeof(uint32_t) * L.tile_cap);
    L.sp_tile_begin = take(sizeof(uint32_t) * L.wave_cap);
    L.segs = take(sizeof(SegDesc) * L.wave_cap);
    L.C = take(sizeof(uint32_t) * L.pair_cap);
    L.FBc = take(sizeof(uint32_t) * L.pair_cap);
    L.TLc = take(sizeof(uint32_t) * L.pair_cap);
    L.tinfo = take(sizeof(TileInfo) * L.tile_cap);
    L.child = take(sizeof(ChildInfo) * L.child_cap);
    L.words = take(L.levels ? sizeof(uint32_t) * L.slot_cap : 0);
    L.pool = take(L.levels ? (size_t)w * L.pool_cap : 0);
    L.dem = take(sizeof(DemRec) * L.dem_cap);
    L.park_cap = L.levels ? (uint32_t)std::min<uint64_t>(65536, L.slot_cap / 16 + 64) : 0;
    L.parks = take(sizeof(ParkRec) * L.park_cap);
    // the medium solver (data in global scratch) runs only for subproblems above the
    // shared-memory limit: children of in-place levels, or a root in that range
    bool need_medium = L.levels > 0;
    for (uint64_t n : ns) need_medium |= n > L.small_max_m && n <= kMediumMaxM;
    L.mscratch = take(need_medium ? (size_t)L.medium_grid * kMediumMaxM * w : 0);
    L.total = off;
    (void)meta_start;
    L.aux_bytes = off;
    return L;
}

// Plans are a function of (n, w) alone: the root is always cut into kRootSplit tiles, whatever
// GPU runs the call (152 is GB300's SM count, so there the root has one tile per SM).  The tile
// split is part of the canonical output (Sec. 5: the result is reproducible from the seed);
// the SM count of the device changes only the schedule, never (k, T, B).
constexpr uint32_t kRootSplit = 152;

bool default_plan_impl(uint64_t n, uint32_t w, rip_plan* p) {
    if (!valid_w(w) || !p) return false;
    std::memset(p, 0, sizeof(*p));
    const uint64_t bytes = n * w;
    const uint32_t k = bytes < (128ull << 20) ? 64 : 256;  // Sec. 5: k = 64 below 128 MiB, else 256
    uint32_t B = (uint32_t)((128u * 1024u) / (k * w));
    B = std::max<uint32_t>(1, std::min<uint32_t>(B, 1024));
    // level 0: kRootSplit tiles (rounded to a multiple of B); deeper levels: one tile per subproblem,
    // or, where level 1 runs in place, two: the first 4/5 of the expected subproblem and the rest.
    // Classify takes all first tiles before the short ones, so when a wave holds fewer
    // subproblems than SMs the idle SMs work through the short tiles meanwhile (measured on
    // GB300 at 2^30 u64, 128 subproblems per wave on 152 SMs: 4/5 best of 0.6 to 0.95)
    uint64_t T0 = (n + kRootSplit - 1) / kRootSplit;
    T0 = std::max<uint64_t>(T0, (uint64_t)B * 64);
    T0 = (T0 + B - 1) / B * B;
    T0 = std::min<uint64_t>(T0, (uint64_t)B << 20);
    T0 = T0 / B * B;
    // level 1 and below: where the root's children run in place (above ~32K elements), k is
    // chosen so that their children hold about 8K elements -- the on-SM solver then finishes
    // them with one more scatter or none (measured on GB300: 1.4-2.3x faster from 2^22 to
    // 2^28 elements than k = 256 at every level); smaller children keep the root's k
    const uint64_t m1 = n / k;
    uint32_t k1 = k;
    if (m1 > 32768) {
        k1 = 16;
        while (k1 < 256 && (uint64_t)k1 * 8192 < m1) k1 *= 2;
    }
    p->num_levels = 2;
    p->level[0].k = k;
    p->level[0].block = B;
    p->level[0].tile = T0;
    p->level[1].k = k1;
    p->level[1].block = B;
    p->level[1].tile = std::min<uint64_t>((uint64_t)B << 20, (uint64_t)1 << 40) / B * B;
    if (m1 > 32768) p->level[1].tile = std::max<uint64_t>((uint64_t)B * 64, (4 * m1 / 5 + B - 1) / B * B);
    p->base = 4096;
    p->max_levels = 0;
    return true;
}

// Plan for inputs that fill most of the device (the near-capacity case): k = 1024 buckets
// over two levels, then Fisher-Yates; blocks of 1 KiB at the root (the slot table costs 4
// bytes per block) and 32 elements below (the tails of the 2^20 deeper tiles cost about
// B/2 elements each); kRootSplit root tiles, one tile per level-1 subproblem.
bool capacity_plan_impl(uint64_t n, uint32_t w, rip_plan* p) {
    if (!valid_w(w) || !p) return false;
    std::memset(p, 0, sizeof(*p));
    const uint32_t k = 1024;
    const uint32_t B0 = 1024u / w, B1 = 32;
    uint64_t T0 = (n + kRootSplit - 1) / kRootSplit;
    T0 = std::max<uint64_t>(T0, (uint64_t)B0 * 64);
    T0 = (T0 + B0 - 1) / B0 * B0;
    T0 = std::min<uint64_t>(T0, (uint64_t)B0 << 20) / B0 * B0;
    p->num_levels = 2;
    p->level[0].k = k;
    p->level[0].block = B0;
    p->level[0].tile = T0;
    p->level[1].k = k;
    p->level[1].block = B1;
    p->level[1].tile = (uint64_t)B1 << 20;
    p->base = 4096;
    p->max_levels = 2;
    return true;
}

constexpr uint32_t kAuxStreams = 8;   // plan groups of one batched call run concurrently on these
constexpr uint32_t kAuxSets = 32;     // caller streams with their own auxiliary streams, per device

// Auxiliary streams and fork/join events of one caller stream: batched calls issued on different
// caller streams never share them, so their plan groups overlap on the device as the callers'
// streams do, and calls from several host threads on different streams do not share events.
struct AuxSet {
    cudaStream_t caller = nullptr;
    cudaStream_t aux[kAuxStreams] = {};
    cudaEvent_t fork = nullptr, join[kAuxStreams] = {};
    uint64_t last_use = 0;
};

struct DevState {
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaEvent_t ws_done = nullptr;  // recorded after the last call that used the managed workspace
    bool ws_used = false;
    uint32_t num_sms = 0;
    Status* status = nullptr;
    unsigned long long* digest_buf = nullptr;
    uint64_t last_info[3] = {0, 0, 0};
    std::vector<AuxSet*> aux_sets;
    uint64_t aux_clock = 0;
};

std::mutex g_mutex;
std::vector<DevState> g_dev;

// Host-side fault injection for tests of the allocation-failure path (RIP_ENOMEM): while
// g_fail_allocs > 0, every workspace allocation the library would make fails instead (and
// decrements the counter).  Set through rip_test_fail_allocations.
uint32_t g_fail_allocs = 0;
// Limit of the device-side hand-off and chain waits (0: the built-in limits); set through
// rip_debug_set_wait_limit to test the RIP_ETIMEOUT path.
uint32_t g_wait_polls = 0;
bool alloc_allowed() {
    if (g_fail_allocs == 0) return true;
    --g_fail_allocs;
    return false;
}

DevState* dev_state(int* dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DevState& d = g_dev[dev];
    if (!d.num_sms) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return nullptr;
        d.num_sms = (uint32_t)sms;
        void* sp = nullptr;
        if (cudaGetSymbolAddress(&sp, g_status) != cudaSuccess) return nullptr;
        d.status = reinterpret_cast<Status*>(sp);
    }
    if (dev_out) *dev_out = dev;
    return &d;
}

// One level-synchronous run over arrays that share a plan: array i is shuffled with seeds[i].
// Adds to the device's last-call diagnostics (callers clear them).
int run_shuffle(const std::vector<char*>& ptrs, const std::vector<uint64_t>& ns, const std::vector<uint64_t>& seeds,
                uint32_t w, const rip_plan& plan, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!valid_w(w)) return RIP_EINVAL;
    for (size_t i = 0; i < ptrs.size(); ++i) {
        if (ns[i] > 1 && !ptrs[i]) return RIP_EINVAL;
        if (ns[i] > 1 && (reinterpret_cast<uintptr_t>(ptrs[i]) % w)) return RIP_EINVAL;
        if (ns[i] > (1ull << 40)) return RIP_EINVAL;
    }
    int dev = 0;
    DevState* ds = dev_state(&dev);
    if (!ds) return RIP_ECUDA;
    if (validate_plan(plan, w) != RIP_OK) return RIP_EINVAL;
    bool any = false;
    for (uint64_t n : ns) any |= n > 1;
    if (!any) return RIP_OK;

    const Layout lay = make_layout(ns, w, plan);
    char* wsp = static_cast<char*>(ws);  // resolved by the caller (run_groups)
    if (!wsp || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(wsp) & 255)) return RIP_EWORKSPACE;
    ds->last_info[0] = std::max<uint64_t>(ds->last_info[0], lay.aux_bytes);

    const DevPlan dplan = to_dev(plan);
    // tuning knob: chain steps before the permutation parks a block (RIP_PARK_AFTER)
    uint32_t park_after = kParkAfter;
    if (const char* env = std::getenv("RIP_PARK_AFTER")) park_after = (uint32_t)std::strtoul(env, nullptr, 10);
    // array table: device pointer, size, seed
    std::vector<ArrayDesc> arr(ptrs.size());
    bool aligned16 = true;
    for (size_t i = 0; i < ptrs.size(); ++i) {
        arr[i] = ArrayDesc{ptrs[i], ns[i] > 1 ? ns[i] : 0, seeds[i]};
        aligned16 &= (reinterpret_cast<uintptr_t>(ptrs[i]) % 16) == 0;
    }
    ArrayDesc* d_arr = reinterpret_cast<ArrayDesc*>(wsp + lay.arrays);
    uint32_t launches = 0;
    InitArgs ia{};
    // the table reaches the device in kernel parameters, never by a copy from host memory: no
    // stream sync, and a captured CUDA graph holds the table itself
    if (arr.size() <= kInlineArrays) {  // written by the init kernel
        ia.inline_count = (uint32_t)arr.size();
        for (size_t i = 0; i < arr.size(); ++i) ia.inline_arrays[i] = arr[i];
    } else {
        for (size_t i0 = 0; i0 < arr.size(); i0 += kDescsPerLaunch) {
            DescChunk c{};
            c.dst = d_arr + i0;
            c.n = (uint32_t)std::min<size_t>(kDescsPerLaunch, arr.size() - i0);
            for (uint32_t j = 0; j < c.n; ++j) c.a[j] = arr[i0 + j];
            if (launch_descs(c, stream) != cudaSuccess) return RIP_ECUDA;
            ++launches;
        }
    }

    uint32_t* counts = reinterpret_cast<uint32_t*>(wsp + lay.counts);
    Lists lists{};
    lists.big[0] = reinterpret_cast<Sub*>(wsp + lay.lists_big0);
    lists.big[1] = reinterpret_cast<Sub*>(wsp + lay.lists_big1);
    lists.big_count[0] = counts + 0;
    lists.big_count[1] = counts + 1;
    lists.big_cap = lay.big_cap;
    lists.small = reinterpret_cast<Sub*>(wsp + lay.small);
    lists.small_count = counts + 2;
    lists.medium = reinterpret_cast<Sub*>(wsp + lay.medium);
    lists.medium_count = counts + 3;
    lists.small_cap = lay.small_cap;
    lists.medium_cap = lay.medium_cap;
    lists.bigfy = reinterpret_cast<Sub*>(wsp + lay.bigfy);
    lists.bigfy_count = counts + 4;
    lists.bigfy_cap = lay.bigfy_cap;

    uint32_t* counters = reinterpret_cast<uint32_t*>(wsp + lay.counters);
    uint64_t* pool_used = reinterpret_cast<uint64_t*>(wsp + lay.pool_used);
    Status* cst = reinterpret_cast<Status*>(wsp + lay.cstatus);  // this call's status word

    ia.arrays = d_arr;
    ia.narrays = (uint32_t)arr.size();
    ia.plan = dplan;
    ia.status = cst;
    ia.lists = lists;
    ia.small_max_m = lay.small_max_m;
    ia.counters = counters;
    ia.pool_used = pool_used;
    if (launch_init(ia, stream) != cudaSuccess) return RIP_ECUDA;
    // chain starts scan the whole slot table for words in state 01: start from all zero
    if (lay.levels && cudaMemsetAsync(wsp + lay.words, 0, sizeof(uint32_t) * lay.slot_cap, stream) != cudaSuccess)
        return RIP_ECUDA;
    ++launches;

    auto run_small = [&]() -> int {
        SmallArgs sa{lists.small, lists.small_count, lists.small_cap, d_arr, dplan, cst, nullptr, 0, 0};
        const size_t smem = small_smem_bytes(lay.small_max_m, w, false);
        if (launch_small(sa, w, smem, ds->num_sms, stream) != cudaSuccess) return RIP_ECUDA;
        SmallArgs ma{lists.medium, lists.medium_count, lists.medium_cap, d_arr, dplan, cst,
                     wsp + lay.mscratch, (uint64_t)kMediumMaxM * w, 1};
        const size_t msmem = small_smem_bytes(kMediumMaxM, w, true);
        if (launch_small(ma, w, msmem, lay.medium_grid, stream) != cudaSuccess) return RIP_ECUDA;
        launches += 3;  // the on-SM solver, its index-path leaves, the medium solver
        return RIP_OK;
    };
    int rc = run_small();
    if (rc) return rc;

    for (uint32_t lev = 0; lev < lay.levels; ++lev) {
        const uint32_t li = dplan.idx(lev);
        LevelArgs a{};
        a.arrays = d_arr;
        a.plan = dplan;
        a.status = cst;
        a.wait_polls = g_wait_polls;
        a.level = lev;
        a.k = plan.level[li].k;
        a.B = plan.level[li].block;
        a.T = plan.level[li].tile;
        a.fdB = FastDiv::make(a.B);
        if (!fastdiv_ok(a.fdB)) return RIP_EINTERNAL;
        a.vec16 = aligned16 && ((a.B * w) % 16 == 0) ? 1u : 0u;
        if (!classify_config(a.k, a.B, w, &a.cls)) return RIP_EINVAL;
        a.big = lists.big[lev & 1];
        a.big_count = lists.big_count[lev & 1];
        a.next_big = lists.big[(lev + 1) & 1];
        a.next_big_count = lists.big_count[(lev + 1) & 1];
        a.big_cap = lay.big_cap;
        a.small = lists.small;
        a.small_count = lists.small_count;
        a.medium = lists.medium;
        a.medium_count = lists.medium_count;
        a.small_cap = lay.small_cap;
        a.medium_cap = lay.medium_cap;
        a.bigfy = lists.bigfy;
        a.bigfy_count = lists.bigfy_count;
        a.bigfy_cap = lay.bigfy_cap;
        a.small_max_m = lay.small_max_m;
        a.tiles = reinterpret_cast<TileRef*>(wsp + lay.tiles);
        a.sp_tile_begin = reinterpret_cast<uint32_t*>(wsp + lay.sp_tile_begin);
        a.sched = reinterpret_cast<uint32_t*>(wsp + lay.sched);
        a.counters = counters;
        a.pool_used = pool_used;
        a.tile_cap = lay.tile_cap;
        a.C = reinterpret_cast<uint32_t*>(wsp + lay.C);
        a.FBc = reinterpret_cast<uint32_t*>(wsp + lay.FBc);
        a.TLc = reinterpret_cast<uint32_t*>(wsp + lay.TLc);
        a.tinfo = reinterpret_cast<TileInfo*>(wsp + lay.tinfo);
        a.slot_cap = lay.slot_cap;
        a.segs = reinterpret_cast<SegDesc*>(wsp + lay.segs);
        a.child = reinterpret_cast<ChildInfo*>(wsp + lay.child);
        a.words = reinterpret_cast<uint32_t*>(wsp + lay.words);
        a.pool = wsp + lay.pool;
        a.pool_cap = lay.pool_cap;
        a.pool_align = 16 / std::min<uint32_t>(w, 16);
        a.dem = reinterpret_cast<DemRec*>(wsp + lay.dem);
        a.dem_cap = lay.dem_cap;
        a.parks = reinterpret_cast<ParkRec*>(wsp + lay.parks);
        a.park_cap = lay.park_cap;
        a.park_after = park_after;
        a.wcap = lay.wave[lev];
        a.wend = lay.wave[lev] * lay.waves[lev];
        for (uint32_t wv = 0; wv < lay.waves[lev]; ++wv) {  // the level's subproblems, one wave at a time
            a.wb = wv * lay.wave[lev];
            if (launch_level(a, w, ds->num_sms, stream, &launches) != cudaSuccess) return RIP_ECUDA;
        }
        rc = run_small();
        if (rc) return rc;
    }
    if (launch_bigfy(lists.bigfy, lists.bigfy_count, lists.bigfy_cap, d_arr, dplan, w,
                     lists.big_count[lay.levels & 1], cst, ds->status, stream) != cudaSuccess)
        return RIP_ECUDA;
    ++launches;
    ds->last_info[1] = std::max<uint64_t>(ds->last_info[1], lay.levels);
    ds->last_info[2] += launches;
    return RIP_OK;
}

// Arrays grouped by their plan (one run per group): `uniform` for every array if given,
// else plans[i] if given, else the default plan of each array's own size.
struct Group {
    rip_plan plan;
    std::vector<uint32_t> idx;
};

bool same_plan(const rip_plan& a, const rip_plan& b) {
    if (a.num_levels != b.num_levels || a.max_levels != b.max_levels || a.base != b.base) return false;
    for (uint32_t l = 0; l < a.num_levels && l < RIP_MAX_LEVEL_PARAMS; ++l)
        if (a.level[l].k != b.level[l].k || a.level[l].block != b.level[l].block || a.level[l].tile != b.level[l].tile)
            return false;
    return true;
}

std::vector<Group> group_arrays(const uint64_t* ns, uint32_t count, uint32_t w, const rip_plan* uniform,
                                const rip_plan* plans) {
    std::vector<Group> groups;
    for (uint32_t i = 0; i < count; ++i) {
        rip_plan p;
        if (uniform) p = *uniform;
        else if (plans) p = plans[i];
        else default_plan_impl(ns[i], w, &p);
        Group* g = nullptr;
        for (Group& x : groups)
            if (same_plan(x.plan, p)) {
                g = &x;
                break;
            }
        if (!g) {
            groups.push_back(Group{p, {}});
            g = &groups.back();
        }
        g->idx.push_back(i);
    }
    return groups;
}

// Workspace offsets of the groups (several groups run at once, each on its own slice);
// returns the total, 0 for an invalid plan.
size_t groups_workspace(const std::vector<Group>& groups, const uint64_t* ns, uint32_t w,
                        std::vector<size_t>* offsets = nullptr) {
    size_t need = 0;
    for (const Group& g : groups) {
        if (validate_plan(g.plan, w) != RIP_OK) return 0;
        std::vector<uint64_t> v;
        for (uint32_t i : g.idx) v.push_back(ns[i]);
        if (offsets) offsets->push_back(need);
        need += align_up(make_layout(v, w, g.plan).total, 256);
    }
    return need;
}

// The library-managed workspace of the current device, grown to `need` bytes.  The caller's
// stream is ordered after the previous call that used it (on whatever stream), so calls with the
// managed workspace never overlap on the device; callers that want concurrent shuffles pass
// their own workspaces.
char* managed_workspace(DevState* ds, size_t need, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!ds->ws_done && cudaEventCreateWithFlags(&ds->ws_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (ds->ws_bytes < need) {
        if (ds->ws) {
            cudaDeviceSynchronize();
            cudaFree(ds->ws);
            ds->ws = nullptr;
            ds->ws_bytes = 0;
        }
        if (!alloc_allowed() || cudaMalloc(&ds->ws, need) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ds->ws_bytes = need;
        ds->ws_used = false;
    } else if (ds->ws_used && cudaStreamWaitEvent(stream, ds->ws_done, 0) != cudaSuccess) {
        return nullptr;
    }
    return static_cast<char*>(ds->ws);
}

// Marks the end of a call that used the managed workspace (on `stream`).
bool managed_workspace_done(DevState* ds, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g_mutex);
    ds->ws_used = true;
    return cudaEventRecord(ds->ws_done, stream) == cudaSuccess;
}

// The auxiliary set of `caller` (created on first use; the least recently used set is reused
// for a new caller stream once kAuxSets exist -- that caller's earlier work is still ordered
// before, because every batched call joins its auxiliary streams back into its caller).
AuxSet* aux_set(DevState* ds, cudaStream_t caller) {
    std::lock_guard<std::mutex> lock(g_mutex);
    ++ds->aux_clock;
    for (AuxSet* a : ds->aux_sets)
        if (a->caller == caller) {
            a->last_use = ds->aux_clock;
            return a;
        }
    AuxSet* a = nullptr;
    if (ds->aux_sets.size() < kAuxSets) {
        a = new AuxSet();
        for (uint32_t i = 0; i < kAuxStreams; ++i) {
            if (cudaStreamCreateWithFlags(&a->aux[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
            if (cudaEventCreateWithFlags(&a->join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        }
        if (cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ds->aux_sets.push_back(a);
    } else {
        a = *std::min_element(ds->aux_sets.begin(), ds->aux_sets.end(),
                              [](const AuxSet* x, const AuxSet* y) { return x->last_use < y->last_use; });
    }
    a->caller = caller;
    a->last_use = ds->aux_clock;
    return a;
}

int run_groups(void* const* ptrs, const uint64_t* ns, uint32_t count, uint32_t w, uint64_t base_seed,
               const rip_plan* uniform, const rip_plan* plans, void* ws, size_t ws_bytes, cudaStream_t stream,
               const uint64_t* seeds_arg = nullptr) {
    if (!valid_w(w)) return RIP_EINVAL;
    if (count && (!ptrs || !ns)) return RIP_EINVAL;
    for (uint32_t i = 0; i < count; ++i) {  // argument errors come before any device work
        if (ns[i] > 1 && !ptrs[i]) return RIP_EINVAL;
        if (ns[i] > 1 && (reinterpret_cast<uintptr_t>(ptrs[i]) % w)) return RIP_EINVAL;
        if (ns[i] > (1ull << 40)) return RIP_EINVAL;
    }
    bool any = false;
    for (uint32_t i = 0; i < count; ++i) any |= ns[i] > 1;
    if (!any) return RIP_OK;
    DevState* ds = dev_state(nullptr);
    if (!ds) return RIP_ECUDA;
    ds->last_info[0] = ds->last_info[1] = ds->last_info[2] = 0;
    const std::vector<Group> groups = group_arrays(ns, count, w, uniform, plans);
    for (const Group& g : groups)
        if (validate_plan(g.plan, w) != RIP_OK) return RIP_EINVAL;
    std::vector<size_t> offs;
    const size_t need = groups_workspace(groups, ns, w, &offs);
    char* wsp = static_cast<char*>(ws);
    const bool managed = !wsp;
    if (wsp) {
        if (ws_bytes < need || (reinterpret_cast<uintptr_t>(wsp) & 255)) return RIP_EWORKSPACE;
    } else {
        wsp = managed_workspace(ds, need, stream);
        if (!wsp) return RIP_ENOMEM;
    }
    // one group runs on the caller's stream; several run concurrently, group g on auxiliary
    // stream g mod 8 of the caller stream's set, each group on its own workspace slice, forked
    // from and joined into the caller's stream
    const bool fan = groups.size() > 1;
    AuxSet* as = nullptr;
    if (fan) {
        as = aux_set(ds, stream);
        if (!as) return RIP_ECUDA;
        if (cudaEventRecord(as->fork, stream) != cudaSuccess) return RIP_ECUDA;
        for (uint32_t a = 0; a < kAuxStreams && a < groups.size(); ++a)
            if (cudaStreamWaitEvent(as->aux[a], as->fork, 0) != cudaSuccess) return RIP_ECUDA;
    }
    int rc = RIP_OK;
    for (size_t gi = 0; gi < groups.size() && rc == RIP_OK; ++gi) {
        const Group& g = groups[gi];
        std::vector<char*> p;
        std::vector<uint64_t> n, seeds;
        const uint64_t* seeds_in = seeds_arg;
        for (uint32_t i : g.idx) {
            p.push_back(static_cast<char*>(ptrs[i]));
            n.push_back(ns[i]);
            seeds.push_back(seeds_in ? seeds_in[i] : base_seed + i);
        }
        const cudaStream_t st = fan ? as->aux[gi % kAuxStreams] : stream;
        rc = run_shuffle(p, n, seeds, w, g.plan, wsp + offs[gi], need - offs[gi], st);
    }
    if (fan) {  // join even after an error, so the caller's stream orders everything enqueued
        for (uint32_t a = 0; a < kAuxStreams && a < groups.size(); ++a) {
            if (cudaEventRecord(as->join[a], as->aux[a]) != cudaSuccess) return RIP_ECUDA;
            if (cudaStreamWaitEvent(stream, as->join[a], 0) != cudaSuccess) return RIP_ECUDA;
        }
    }
    if (managed && !managed_workspace_done(ds, stream)) return RIP_ECUDA;
    return rc;
}

}  // namespace
}  // namespace rip

using namespace rip;

extern "C" {

int rip_default_plan(uint64_t n, uint32_t elem_bytes, rip_plan* plan) {
    if (!plan || !valid_w(elem_bytes)) return RIP_EINVAL;
    return default_plan_impl(n, elem_bytes, plan) ? RIP_OK : RIP_EINVAL;
}

int rip_capacity_plan(uint64_t n, uint32_t elem_bytes, rip_plan* plan) {
    if (!plan || !valid_w(elem_bytes)) return RIP_EINVAL;
    return capacity_plan_impl(n, elem_bytes, plan) ? RIP_OK : RIP_EINVAL;
}

size_t rip_shuffle_workspace_size(uint64_t n, uint32_t elem_bytes, const rip_plan* plan) {
    uint64_t one = n;
    return rip_shuffle_batched_workspace_size(&one, 1, elem_bytes, plan);
}

size_t rip_shuffle_batched_workspace_size(const uint64_t* ns, uint32_t count, uint32_t elem_bytes,
                                          const rip_plan* plan) {
    if (!valid_w(elem_bytes) || (count && !ns)) return 0;
    return groups_workspace(group_arrays(ns, count, elem_bytes, plan, nullptr), ns, elem_bytes);
}

size_t rip_shuffle_batched_ex_workspace_size(const uint64_t* ns, uint32_t count, uint32_t elem_bytes,
                                             const rip_plan* plans) {
    if (!valid_w(elem_bytes) || (count && !ns)) return 0;
    return groups_workspace(group_arrays(ns, count, elem_bytes, nullptr, plans), ns, elem_bytes);
}

size_t rip_shuffle_batched_plans_workspace_size(const uint64_t* ns, uint32_t count, uint32_t elem_bytes,
                                                const rip_plan* plans) {
    if (!valid_w(elem_bytes) || (count && (!ns || !plans))) return 0;
    return groups_workspace(group_arrays(ns, count, elem_bytes, nullptr, plans), ns, elem_bytes);
}

int rip_shuffle(void* data, uint64_t n, uint32_t elem_bytes, uint64_t seed, rip_stream_t stream) {
    return rip_shuffle_ex(data, n, elem_bytes, seed, nullptr, nullptr, 0, stream);
}

int rip_shuffle_ex(void* data, uint64_t n, uint32_t elem_bytes, uint64_t seed, const rip_plan* plan, void* ws,
                   size_t ws_bytes, rip_stream_t stream) {
    void* p[1] = {data};
    return run_groups(p, &n, 1, elem_bytes, seed, plan, nullptr, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int rip_shuffle_batched(void* const* ptrs, const uint64_t* ns, uint32_t count, uint32_t elem_bytes,
                        uint64_t base_seed, const rip_plan* plan, void* ws, size_t ws_bytes, rip_stream_t stream) {
    return run_groups(ptrs, ns, count, elem_bytes, base_seed, plan, nullptr, ws, ws_bytes,
                      reinterpret_cast<cudaStream_t>(stream));
}

int rip_shuffle_batched_ex(void* const* ptrs, const uint64_t* ns, const uint64_t* seeds, uint32_t count,
                           uint32_t elem_bytes, const rip_plan* plans, void* ws, size_t ws_bytes,
                           rip_stream_t stream) {
    if (count && !seeds) return RIP_EINVAL;
    return run_groups(ptrs, ns, count, elem_bytes, 0, nullptr, plans, ws, ws_bytes,
                      reinterpret_cast<cudaStream_t>(stream), seeds);
}

int rip_shuffle_batched_plans(void* const* ptrs, const uint64_t* ns, uint32_t count, uint32_t elem_bytes,
                              uint64_t base_seed, const rip_plan* plans, void* ws, size_t ws_bytes,
                              rip_stream_t stream) {
    if (count && !plans) return RIP_EINVAL;
    return run_groups(ptrs, ns, count, elem_bytes, base_seed, nullptr, plans, ws, ws_bytes,
                      reinterpret_cast<cudaStream_t>(stream));
}

int rip_digest(const void* data, uint64_t n, uint32_t elem_bytes, uint64_t* out, rip_stream_t stream) {
    if (!out || !valid_w(elem_bytes) || (n && !data)) return RIP_EINVAL;
    DevState* ds = dev_state(nullptr);
    if (!ds) return RIP_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!ds->digest_buf && cudaMalloc(&ds->digest_buf, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return RIP_ENOMEM;
        }
    }
    if (cudaMemsetAsync(ds->digest_buf, 0, sizeof(unsigned long long), s) != cudaSuccess) return RIP_ECUDA;
    if (n && launch_digest(data, n, elem_bytes, ds->digest_buf, s) != cudaSuccess) return RIP_ECUDA;
    unsigned long long h = 0;
    if (cudaMemcpyAsync(&h, ds->digest_buf, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RIP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RIP_ECUDA;
    *out = h;
    return RIP_OK;
}

int rip_get_device_status(rip_stream_t stream) {
    DevState* ds = dev_state(nullptr);
    if (!ds) return RIP_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return RIP_ECUDA;
    Status st{};
    if (cudaMemcpy(&st, ds->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return RIP_ECUDA;
    if (st.code) {
        Status zero{};
        if (cudaMemcpy(ds->status, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) return RIP_ECUDA;
    }
    return (int)st.code;
}

int rip_release_workspace(void) {
    DevState* ds = dev_state(nullptr);
    if (!ds) return RIP_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (ds->ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) return RIP_ECUDA;
        cudaFree(ds->ws);
        ds->ws = nullptr;
        ds->ws_bytes = 0;
        ds->ws_used = false;
    }
    return RIP_OK;
}

int rip_debug_fail_allocations(uint32_t count) {
    std::lock_guard<std::mutex> lock(g_mutex);
    g_fail_allocs = count;
    return RIP_OK;
}

int rip_debug_set_wait_limit(uint32_t polls) {
    std::lock_guard<std::mutex> lock(g_mutex);
    g_wait_polls = polls;
    return RIP_OK;
}

const char* rip_strerror(int code) {
    switch (code) {
        case RIP_OK: return "ok";
        case RIP_EINVAL: return "invalid argument or plan";
        case RIP_ENOMEM: return "device workspace allocation failed";
        case RIP_EWORKSPACE: return "workspace too small or device pool exhausted";
        case RIP_ECUDA: return "CUDA runtime error";
        case RIP_ETIMEOUT: return "device-side wait limit expired";
        case RIP_EINTERNAL: return "device-side consistency check failed";
        case RIP_ETOOLARGE: return "input too large for the fixed workspace of rip_shuffle_noalloc";
        default: return "unknown error";
    }
}

int rip_profile_enable(int on) {
    g_prof.on = on != 0;
    return RIP_OK;
}

int rip_profile_reset(void) {
    g_prof.fold();
    g_prof.totals.clear();
    return RIP_OK;
}

int rip_profile_get(uint32_t idx, const char** name, uint64_t* launches, double* total_ms) {
    g_prof.fold();
    if (idx >= g_prof.totals.size()) return RIP_EINVAL;
    if (name) *name = g_prof.totals[idx].name.c_str();
    if (launches) *launches = g_prof.totals[idx].launches;
    if (total_ms) *total_ms = g_prof.totals[idx].ms;
    return RIP_OK;
}

int rip_last_call_info(uint64_t out[3]) {
    if (!out) return RIP_EINVAL;
    DevState* ds = dev_state(nullptr);
    if (!ds) return RIP_ECUDA;
    for (int i = 0; i < 3; ++i) out[i] = ds->last_info[i];
    return RIP_OK;
}

}  // extern "C"
