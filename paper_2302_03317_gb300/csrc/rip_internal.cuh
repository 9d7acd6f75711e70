// rip_internal.cuh -- kernel argument blocks and launch entry points shared
// by the translation units of the library.
#pragma once
#include "rip_device.cuh"

namespace rip {

constexpr uint32_t kMaxK = 1024;
constexpr uint32_t kSmallThreads = 512;
constexpr uint32_t kSmallCntCap = 512;    // (tile, bucket) counters of one in-SMEM scatter
constexpr uint32_t kSmallTbl = 4096;      // (ranking warp, bucket) entries
constexpr uint32_t kSmallStack = 256;     // pending scatter ranges inside one subproblem
constexpr uint32_t kMediumMaxM = 49152;   // largest subproblem finished on one SM
constexpr uint32_t kClassifyThreads = 1024;
constexpr uint32_t kPermuteThreads = 256;
constexpr uint32_t kGroup = 8;            // lanes moving one block in the permutation
constexpr size_t kSmemOptin = 232448;     // dynamic shared memory per block on sm_100/103

// Slot words (one per B-element slot of the subproblems of one wave; each subproblem's
// slots form a segment of the table, starting at a multiple of 64):
//   bits 31..30 state: 00 empty, 01 holds an unmoved block, 11 claimed, 10 filled
//   after classification: bits 29..20 bucket, 19..0 block index inside (tile, bucket)
//   after resolution:     bit 29 "goes to the pool", bits 28..0 destination slot
//                         (or demoted-record index when bit 29 is set)
constexpr uint32_t kWordOcc = 1u << 30;
constexpr uint32_t kWordTaken = 1u << 31;
constexpr uint32_t kWordDem = 1u << 29;
constexpr uint32_t kWordDestMask = (1u << 29) - 1u;
constexpr uint32_t kBlkBits = 20;

// The slot segment of one subproblem of the current wave: table entries [base, base + nslots)
// hold grid slots orig .. orig + nslots - 1 of the array (grid slot g = elements [gB, (g+1)B)).
struct SegDesc {
    uint64_t base;
    uint64_t orig;
    uint64_t nslots;
    uint32_t arr;
    uint32_t pad;
};

struct TileRef {
    uint32_t sp;  // index in the level's big list
    uint32_t t;   // tile index inside the subproblem
};

struct TileInfo {
    uint64_t hs0;        // slot-table index of the tile's first home slot
    uint64_t pool_base;  // element offset of the tile's tails in the pool
    uint32_t home_used;  // home slots holding a full block after classification
    uint32_t H;          // home slots available
};

struct ChildInfo {
    uint64_t o;          // region start (array-relative)
    uint64_t m;          // size
    uint64_t slot_base;  // slot-table index of full block 0 (in the parent's segment)
    uint32_t Fb;         // full blocks of the bucket
    uint32_t placed;     // full blocks that go to slots (Fb or Fb-1)
    uint32_t eps;        // rotation of the child region
    uint32_t pad;
};

struct DemRec {
    uint32_t sp, tile, b, blk;
    uint64_t pool_off;
};

// A block a chain put aside after too many steps; placed after the permutation.
struct ParkRec {
    uint64_t pool_off;  // element offset in the pool, ~0 when the park failed
    uint64_t dst;       // destination address (byte pointer)
};

struct Lists {
    Sub* big[2];
    uint32_t* big_count[2];
    uint32_t big_cap;
    Sub* small;
    uint32_t* small_count;
    Sub* medium;
    uint32_t* medium_count;
    uint32_t small_cap, medium_cap;
    Sub* bigfy;
    uint32_t* bigfy_count;
    uint32_t bigfy_cap;
};

// Shared-memory geometry of the classify kernel for one (k, B, w), chosen on the host.
struct ClsCfg {
    uint32_t Bs;         // elements per shared-memory chunk (divides B; == B: whole blocks staged)
    uint32_t cpb;        // chunks per block
    uint32_t nwr;        // ranking warps (the (bucket, warp) table holds k * nwr counters)
    uint32_t S;          // table stride per bucket (odd, > nwr: conflict-free columns)
    uint32_t round;      // positions per round (nwr * 128)
    uint32_t q;          // elements per 16 bytes
    uint32_t nbuf;       // input buffers (2 or 3)
    uint32_t bufstride;  // elements per input buffer
    uint32_t off_tbl, off_u32, off_u64, off_flist, off_mask, off_stage, off_buf, bytes;
};

struct LevelArgs {
    const ArrayDesc* arrays;
    DevPlan plan;
    Status* status;
    uint32_t level, k, B, vec16;
    uint64_t T;
    FastDiv fdB;  // division by B
    // this level's subproblems and the next level's
    const Sub* big;
    const uint32_t* big_count;
    Sub* next_big;
    uint32_t* next_big_count;
    uint32_t big_cap;
    Sub* small;
    uint32_t* small_count;
    Sub* medium;
    uint32_t* medium_count;
    uint32_t small_cap, medium_cap;
    Sub* bigfy;
    uint32_t* bigfy_count;
    uint32_t bigfy_cap;
    uint32_t small_max_m;  // largest m whose data fits in shared memory
    // tiles
    TileRef* tiles;
    uint32_t wb, wcap, wend;  // this wave: big-list entries [wb, wb + wcap); all waves: [0, wend)
    uint32_t* sp_tile_begin;  // per subproblem of the wave
    uint32_t* sched;          // classify order of the tiles: every subproblem's non-last tiles, then the last ones
    SegDesc* segs;            // per subproblem of the wave
    uint64_t slot_cap;        // entries of the slot-word table
    uint32_t* counters;       // [0] tiles, [1] tile cursor, [2] demoted count, [4..5] chunk cursor, [6] parks,
                              // [7] subproblems of the wave, [8] 64-entry chunks of the wave's segments
    uint64_t* pool_used;
    uint32_t tile_cap;
    uint32_t* C;    // tile_cap x k counts
    uint32_t* FBc;  // tile_cap x k full blocks of earlier tiles
    uint32_t* TLc;  // tile_cap x k tail elements of earlier tiles
    TileInfo* tinfo;
    ChildInfo* child;       // wcap x k, indexed by (subproblem - wb, bucket)
    uint32_t* words;
    char* pool;
    uint64_t pool_cap;    // elements
    uint32_t pool_align;  // elements per 16 bytes: every pool allocation is a multiple of this
    DemRec* dem;
    uint32_t dem_cap;
    ParkRec* parks;
    uint32_t park_cap;
    uint32_t park_after;  // chain steps before a carried block is parked
    uint32_t wait_polls;  // limit of the hand-off and chain waits (0: the built-in limits)
    ClsCfg cls;
};

struct SmallArgs {
    const Sub* list;
    const uint32_t* count;
    uint32_t capacity;
    const ArrayDesc* arrays;
    DevPlan plan;
    Status* status;
    char* gscratch;
    uint64_t gslot_bytes;
    uint32_t medium;
    uint32_t dyn_bytes;  // dynamic shared memory after SmallShared (set by launch_small)
};

constexpr uint32_t kInlineArrays = 4;
constexpr uint32_t kDescsPerLaunch = 160;  // array descriptors carried by one descs_kernel's parameters

// A piece of a call's array table, written to the workspace by a kernel that carries it in its
// parameters (no host copy: the call can be captured in a CUDA graph).
struct DescChunk {
    ArrayDesc* dst;
    uint32_t n;
    uint32_t pad;
    ArrayDesc a[kDescsPerLaunch];
};
static_assert(sizeof(DescChunk) <= 4096, "kernel parameters stay within the classic 4 KB limit");

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when the kernel's setting on the current
// device is below `bytes` (rip_api.cu): calls made while a stream is being captured into a CUDA
// graph then issue no attribute calls once the same shapes ran before.
cudaError_t ensure_dyn_smem(const void* func, int bytes);

struct InitArgs {
    ArrayDesc* arrays;
    ArrayDesc inline_arrays[kInlineArrays];  // copied to `arrays` by the init kernel when used
    uint32_t inline_count;
    uint32_t narrays;
    DevPlan plan;
    Status* status;
    Lists lists;
    uint32_t small_max_m;
    uint32_t* counters;
    uint64_t* pool_used;
};

// rip_api.cu: optional per-launch CUDA-event timing
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);
struct ProfScope {
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st) : s(st) { prof_begin(name, st); }
    ~ProfScope() { prof_end(s); }
};

// rip_small.cu
size_t small_fixed_smem();
size_t small_smem_bytes(uint64_t m, uint32_t w, bool medium);
// the on-SM solver (small_kernel) and, unless medium, the leaves it leaves to leaf_kernel
cudaError_t launch_small(const SmallArgs& args, uint32_t w, size_t smem, uint32_t grid, cudaStream_t stream);

// rip_classify.cu
bool classify_config(uint32_t k, uint32_t B, uint32_t w, ClsCfg* out);
cudaError_t launch_classify(const LevelArgs& a, uint32_t w, uint32_t num_sms, cudaStream_t s);

// rip_level.cu
size_t permute_smem_bytes(uint32_t B, uint32_t w);
uint32_t permute_threads(uint32_t B, uint32_t w);
cudaError_t launch_init(const InitArgs& a, cudaStream_t s);
cudaError_t launch_descs(const DescChunk& c, cudaStream_t s);
cudaError_t launch_level(const LevelArgs& a, uint32_t w, uint32_t num_sms, cudaStream_t s, uint32_t* launches);
// The call's last kernel: copies the call's status word into the device's (global) one, then
// finishes leaves too large for one SM.
cudaError_t launch_bigfy(const Sub* list, const uint32_t* count, uint32_t cap, const ArrayDesc* arrays,
                         DevPlan plan, uint32_t w, const uint32_t* leftover, Status* status, Status* global,
                         cudaStream_t s);

// rip_digest.cu
cudaError_t launch_digest(const void* data, uint64_t n, uint32_t w, unsigned long long* out, cudaStream_t s);

// device-side eligibility of a subproblem for the on-SM solver (same rule as the host's)
__device__ __host__ __forceinline__ bool small_solver_can_scatter(const DevPlan& plan, uint64_t m, uint32_t L) {
    for (uint32_t l = plan.idx(L); l < plan.num_levels; ++l) {
        const uint64_t T = plan.T[l];
        const uint64_t tiles = T >= m ? 1 : (m + T - 1) / T;
        if (tiles * plan.k[l] > kSmallCntCap || plan.k[l] > kMaxK) return false;
    }
    return true;
}

}  // namespace rip
