/*
 * rip_shuffle.h -- C ABI of the GB300 in-place scatter-shuffle library.
 *
 * Problem (Sec. 1, Sec. 2.2 of Penschuck, "Engineering Shared-Memory Parallel
 * Shuffling to Generate Random Permutations In-Place"): rearrange a sequence
 * of n elements in place so that every permutation is equally likely, using
 * only small auxiliary memory, reproducibly from a seed although the parallel
 * schedule is not deterministic (Sec. 5).
 *
 * Method (Sec. 2.2 ScatterShuffle, Sec. 3.1-3.2 IpScShuf, Sec. 4 PIpScShuf):
 * every element draws an independent uniform bucket among k; elements move
 * into their bucket's contiguous region; every bucket is shuffled recursively;
 * subproblems of at most `base` elements are finished by Fisher-Yates
 * (Sec. 2.2, Fig. 1).  The result is a fixed ("canonical") function of
 * (seed, n, plan): at each level, the elements of bucket b inside each tile of
 * T elements keep their input order; the first B*floor(c/B) of them (c = their
 * count) form "full blocks", the rest the "tail"; bucket b's region holds the
 * full blocks of all tiles in tile order, then the tails in tile order.  The
 * random draws come from Philox-4x32-10 keyed by the seed and counters built
 * from (level, subproblem start, position); Fisher-Yates partners and bucket
 * numbers use Lemire's bounded sampling (Sec. 2.3).  The exact keying is
 * documented next to the device code and in the project's design notes.
 *
 * Conventions for every call below
 *   - Pointers named `data`/`ptrs`/`ws` are DEVICE pointers on the current CUDA
 *     device; the caller owns them and keeps them alive until the stream has
 *     executed the work.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued asynchronously on it; host-side argument errors return before
 *     anything is enqueued.
 *   - elem_bytes is 4, 8 or 16; elements are opaque and only moved.
 *     `data` must be aligned to elem_bytes.
 *   - Return value: RIP_OK or a RIP_E* code below.  Errors detected on the
 *     device (a wait limit that expired, workspace exhausted, an internal
 *     consistency check) are recorded in a device status word; they are
 *     reported by rip_get_device_status() and by the next call that syncs.
 *   - n <= 1 is a no-op returning RIP_OK.
 *   - Library-managed workspace (ws == NULL): one per device, shared by every
 *     call that passes no workspace.  The library orders each such call after
 *     the previous one on the device (an event recorded on the previous call's
 *     stream), so calls on different streams do not overlap on the GPU and do
 *     not race on it; a call that needs a larger workspace synchronises the
 *     device and reallocates.  Callers that want shuffles to run concurrently
 *     on several streams pass their own workspaces.  Calls from several host
 *     threads on one device must still be serialised by the caller.
 */
#ifndef RIP_SHUFFLE_H
#define RIP_SHUFFLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rip_stream_t; /* same type as cudaStream_t */

enum {
    RIP_OK = 0,
    RIP_EINVAL = 1,     /* invalid argument or plan                          */
    RIP_ENOMEM = 2,     /* the library could not allocate its workspace      */
    RIP_EWORKSPACE = 3, /* caller workspace too small / device pool exhausted */
    RIP_ECUDA = 4,      /* a CUDA runtime call failed                         */
    RIP_ETIMEOUT = 5,   /* a bounded device-side wait expired                 */
    RIP_EINTERNAL = 6,  /* a device-side consistency check failed            */
    RIP_ETOOLARGE = 7   /* input needs more than rip_shuffle_noalloc's fixed workspace */
};

#define RIP_MAX_LEVEL_PARAMS 8

/* Parameters of one scatter level (Sec. 3.1 "k buckets"; T and B define the
 * canonical tile/block layout described above). */
typedef struct {
    uint32_t k;     /* buckets: power of two, 2 <= k <= 1024                   */
    uint32_t block; /* B >= 1 elements per full block; B * elem_bytes <= 29 KiB  */
    uint64_t tile;  /* T >= B, T % B == 0 (tiles start at each subproblem start) */
} rip_level_params;

/* A plan: level L uses level[min(L, num_levels - 1)].  A subproblem with
 * m <= base elements, or one reaching level max_levels (0 = no cap, which the
 * library treats as 64), is finished by Fisher-Yates (Sec. 3.2, "base case").
 * base must be in [1, 2^32 - 1]. */
typedef struct {
    uint32_t num_levels;
    uint32_t max_levels;
    uint64_t base;
    rip_level_params level[RIP_MAX_LEVEL_PARAMS];
} rip_plan;

/* Fills *plan with the library's default plan for n elements of elem_bytes:
 * k = 256 (k = 64 below 128 MiB of data, the paper's rule in Sec. 5), base
 * 4096, B sized so k*B*elem_bytes = 128 KiB, the root cut into 152 tiles (one
 * per SM on GB300; the plan depends on n and elem_bytes only, never on the
 * device, so a seed gives the same output on every GPU); where level 1 runs in place
 * (root children above 32K elements) its tile is 4/5 of the expected child, so
 * every child has a long and a short tile (the short ones keep the SMs busy
 * while a wave's long ones run), else one tile per subproblem.  Returns
 * RIP_EINVAL for a NULL plan or bad elem_bytes. */
int rip_default_plan(uint64_t n, uint32_t elem_bytes, rip_plan *plan);

/* Fills *plan with a plan for inputs that fill most of the device (the
 * in-place requirement of Sec. 3 at its largest): k = 1024 buckets over two
 * levels, then Fisher-Yates (max_levels 2, base 4096); root blocks of 1 KiB and
 * the root cut into 152 tiles (independent of the device); 32-element blocks and one tile
 * per subproblem at level 1.  For 2^34 elements its workspace is 0.86% of a
 * 4-byte input and 0.63% of an 8-byte one; the root level's fixed part (tails
 * and blocks of 152 tiles x 1024 buckets) makes the fraction larger for
 * smaller inputs.  Returns RIP_EINVAL for a NULL plan or bad elem_bytes. */
int rip_capacity_plan(uint64_t n, uint32_t elem_bytes, rip_plan *plan);

/* Bytes of device workspace rip_shuffle_ex needs for (n, elem_bytes, plan);
 * plan NULL = default plan.  Returns 0 if the arguments are invalid. */
size_t rip_shuffle_workspace_size(uint64_t n, uint32_t elem_bytes, const rip_plan *plan);

/* Shuffle data[0..n) in place with the default plan and the library-managed
 * workspace (allocated on first use per device, grown when a larger call
 * needs it, kept until rip_release_workspace / process exit). */
int rip_shuffle(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed, rip_stream_t stream);

/* Shuffle data[0..n) in place with an explicit plan (NULL = default).  If ws
 * is non-NULL it must hold at least rip_shuffle_workspace_size() bytes and be
 * 256-byte aligned; the call then allocates nothing.  If ws is NULL the
 * library-managed workspace is used. */
int rip_shuffle_ex(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                   const rip_plan *plan, void *ws, size_t ws_bytes, rip_stream_t stream);

/* Batched form (Sec. 6, many independent shuffles): array i (device pointer
 * ptrs[i], ns[i] elements) is shuffled with seed base_seed + i, positions
 * relative to its own start.  plan != NULL: every array uses it; plan ==
 * NULL: every array uses its own default plan (rip_default_plan(ns[i])), so an
 * array's result is the same alone and in any batch.  Arrays that share a plan
 * run together: one level-synchronous pass over all of them, the small ones on
 * one SM each.  Groups with different plans run concurrently: each on one of
 * eight auxiliary streams that belong to the caller's `stream` (forked from it
 * and joined back into it, so the call is still ordered on `stream`), each on
 * its own slice of the workspace; the workspace is the sum of the groups'
 * slices (ask the *_workspace_size function).  ptrs and ns are HOST arrays of
 * `count` entries; the arrays must not overlap.  ws as in rip_shuffle_ex. */
size_t rip_shuffle_batched_workspace_size(const uint64_t *ns, uint32_t count, uint32_t elem_bytes,
                                          const rip_plan *plan);
int rip_shuffle_batched(void *const *ptrs, const uint64_t *ns, uint32_t count, uint32_t elem_bytes,
                        uint64_t base_seed, const rip_plan *plan, void *ws, size_t ws_bytes,
                        rip_stream_t stream);

/* Batched form with one plan per array (plans: HOST array of `count` plans,
 * e.g. chosen per size class by a tuner); otherwise as rip_shuffle_batched. */
size_t rip_shuffle_batched_plans_workspace_size(const uint64_t *ns, uint32_t count, uint32_t elem_bytes,
                                                const rip_plan *plans);
int rip_shuffle_batched_plans(void *const *ptrs, const uint64_t *ns, uint32_t count, uint32_t elem_bytes,
                              uint64_t base_seed, const rip_plan *plans, void *ws, size_t ws_bytes,
                              rip_stream_t stream);

/* Batched form with one seed per array (seeds: HOST array of `count` seeds; array i
 * is shuffled with seeds[i]) and optionally one plan per array (plans NULL: every
 * array its own default plan) -- for callers that batch independent requests, each
 * of which keeps its own seed, e.g. a serving loop.  Otherwise as
 * rip_shuffle_batched; the workspace size depends on ns and plans only. */
size_t rip_shuffle_batched_ex_workspace_size(const uint64_t *ns, uint32_t count, uint32_t elem_bytes,
                                             const rip_plan *plans);
int rip_shuffle_batched_ex(void *const *ptrs, const uint64_t *ns, const uint64_t *seeds, uint32_t count,
                           uint32_t elem_bytes, const rip_plan *plans, void *ws, size_t ws_bytes,
                           rip_stream_t stream);

/* Position-dependent 64-bit digest of data[0..n), computed on the device:
 *   H = sum_p splitmix64(p * 0x9E3779B97F4A7C15 ^ v(p)) mod 2^64,
 * v(p) = splitmix64 chained over the element's 8-byte little-endian words.
 * Used to compare outputs too large for a second host copy.  Synchronises
 * `stream` and writes the digest to *out (host pointer). */
int rip_digest(const void *data, uint64_t n, uint32_t elem_bytes, uint64_t *out, rip_stream_t stream);

/* Synchronises `stream`, returns and clears the device status word of the
 * current device (RIP_OK when no device-side error was recorded). */
int rip_get_device_status(rip_stream_t stream);

/* Frees the library-managed workspace of the current device. */
int rip_release_workspace(void);

/* Testing hook for the allocation-failure path (Sec. 1 names failing
 * allocations as a reason for in-place shuffling): the next `count` device
 * allocations the library would make for its managed workspace fail as if
 * cudaMalloc had failed, so the call returns RIP_ENOMEM before enqueuing any
 * work (the data stay untouched).  count 0 turns it off. */
int rip_debug_fail_allocations(uint32_t count);

/* Testing hook for the bounded device-side waits: later calls give every
 * hand-off wait of the classify step (input arrived, chunks read out, round
 * placed) and every chain wait of the block permutation at most `polls`
 * polls (the first one non-blocking) instead of the built-in limits (2^20
 * mbarrier polls of up to 4 us each, 2^24 spins).  A wait that runs out records RIP_ETIMEOUT;
 * the kernel finishes its own copies in flight and returns, the call's later
 * kernels skip their work, and rip_get_device_status reports RIP_ETIMEOUT.
 * The data of that call are then not a valid shuffle.  polls 0 restores the
 * built-in limits. */
int rip_debug_set_wait_limit(uint32_t polls);

/* Static message for a return code. */
const char *rip_strerror(int code);

/* Diagnostics of the last call on the current device, written to *out:
 *   out[0] aux bytes the call's workspace layout uses,
 *   out[1] number of scatter levels launched in place,
 *   out[2] kernels launched by the call.
 * Returns RIP_EINVAL if out is NULL. */
int rip_last_call_info(uint64_t out[3]);

/* Allocation-free variant of rip_shuffle_ex (the paper has no counterpart: it
 * is an interface for callers that must not allocate device memory, such as
 * code running inside a framework's own allocator or memory pool, processes
 * whose device memory is reserved up front by a pool owner, or paths that
 * cannot afford cudaMalloc's implicit synchronisation).  Its workspace is a
 * fixed array of RIP_NOALLOC_WS_BYTES in the library's device image, which
 * every GPU that loads the library holds until the process exits; the call
 * performs no allocation.  Inputs whose workspace
 * (rip_shuffle_workspace_size) exceeds the array are rejected with
 * RIP_ETOOLARGE before anything is enqueued; with the default plans every
 * power-of-two size up to 2^27 4-byte, 2^26 8-byte and 2^20 16-byte elements
 * fits (the workspace is not monotone in n: ask rip_shuffle_workspace_size).  The first call
 * on a device looks up the array's device address (a one-time set-up); make
 * that first call before any stream capture.  All calls share the array and
 * each call clears what must start at zero; calls that overlap on the GPU race
 * on it and must be serialised by the caller.  Arguments and results as in
 * rip_shuffle_ex without ws / ws_bytes. */
#define RIP_NOALLOC_WS_BYTES (32u << 20)
int rip_shuffle_noalloc(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                        const rip_plan *plan, rip_stream_t stream);

/* Kernel timing (the measurement side of the library, no counterpart in the
 * paper, which reports wall-clock means only, Sec. 6): while enabled, every
 * kernel launch of later calls is bracketed by two CUDA events recorded on the
 * launching stream.  rip_profile_get (call after synchronising the stream)
 * returns, for the idx-th kernel name in alphabetical order, the launches and
 * the summed event time in milliseconds; RIP_EINVAL when idx is past the
 * last name.  Not thread-safe; intended for benchmarks. */
int rip_profile_enable(int on);
int rip_profile_reset(void);
int rip_profile_get(uint32_t idx, const char **name, uint64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* RIP_SHUFFLE_H */
