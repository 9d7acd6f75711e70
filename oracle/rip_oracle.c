/*
 * rip_oracle.c -- CPU oracle for the canonical in-place scatter shuffle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py do.  It shares no code, header, table or helper with the
 * CUDA library: every piece below is written out again from its published
 * definition.
 *
 * What it computes (plain, out-of-place, single-threaded loops):
 *
 *   shuffle(X, o, m, L)
 *     if m <= base or L >= max_levels:  fisher_yates(X[o:o+m], o, L)
 *     else:
 *       every element at logical position pos = o+i draws a bucket b in [0,k)
 *         (ScatterShuffle, Sec. 2.2 and Sec. 3.1: independent uniform bucket per
 *          element, buckets become independent subproblems);
 *       tiles are [tT, min((t+1)T, m)) relative to o; inside tile t the
 *       elements of bucket b in increasing position form the list Lst[t][b];
 *       bucket b's region holds, in order,
 *         the first B*floor(|Lst[t][b]|/B) elements of Lst[t][b] for t = 0,1,..
 *         (the "full blocks", tile order), then
 *         the last |Lst[t][b]| mod B elements of Lst[t][b] for t = 0,1,..
 *         (the "tails", tile order);
 *       regions are laid out for b = 0..k-1 from o on; recurse on every
 *       non-empty bucket at level L+1 (Sec. 3.2, the recursion of IpScShuf;
 *       the order inside a bucket is irrelevant for uniformity, Sec. 3.4).
 *
 *   fisher_yates(Y, o, L): for i = m-1 down to 1, swap Y[i] with Y[j],
 *     j uniform in [0, i] (Sec. 2.2, Fig. 1 "fisher_yates").
 *
 * Random numbers (Sec. 2.3; replayable counter-based generator, Sec. 3.1):
 *   Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed_lo, seed_hi).
 *   bucket of pos at level L in the subproblem starting at o:
 *     ctr = (q_lo, q_hi, L | 1<<8, o_lo), q = pos >> 2, word = pos & 3,
 *     b = (word * k) >> 32           (k a power of two: the top log2(k) bits)
 *   Fisher-Yates partner for step i (position p = o+i), Lemire's bounded
 *   rejection for s = i+1 (Sec. 2.3, read as [0,s)):
 *     first word: ctr = (q_lo, q_hi, L | 2<<8, o_lo), q = p >> 2, word p & 3
 *       (four consecutive positions share one Philox call, as bucket draws do);
 *     on rejection, attempts a = 1,2,..: ctr = (p_lo, p_hi, L | 3<<8 | a<<16,
 *       o_lo), words 0..3 tried in order.
 *
 * Parameters per level L: (k, T, B) = level[min(L, num_levels-1)].
 * max_levels = 0 means "no cap"; the recursion is then capped at 64 levels
 * (a subproblem at level 64 goes to Fisher-Yates), which keeps the function
 * total without changing any output of practical probability.
 *
 * Element values are opaque: w bytes each, moved with memcpy (Sec. 1: data
 * may be non-copyable, the algorithm only moves it).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_DEPTH_CAP 64u
#define ORACLE_MAX_LEVEL_PARAMS 32u

/* ---------------------------------------------------------------- Philox */

/* One Philox-4x32 round: two 32x32->64 products, hi/lo words xored with the
 * other counter words and the round key, then the key is bumped by the Weyl
 * constants.  Multipliers and Weyl constants are the ones the Philox paper
 * fixes for the 4x32 variant. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* ---------------------------------------------------------------- Lemire */

/* One attempt of Lemire's bounded sampling ("Fast random integer generation
 * in an interval", TOMACS 2019, cited in Sec. 2.3) at word width `bits`
 * (1..32): x is a uniform `bits`-bit word, s in [1, 2^bits].  Returns 1 and
 * stores the value in [0, s) when x is accepted, 0 when it must be redrawn.
 * The 32-bit sampler below is this function with bits = 32, so an exhaustive
 * check at a small width exercises the same code. */
int oracle_lemire_try(uint32_t bits, uint64_t s, uint32_t x, uint32_t *value)
{
    uint64_t full = (uint64_t)1 << bits;
    uint64_t mask = full - 1;
    uint64_t m = (uint64_t)(x & mask) * s;
    uint64_t low = m & mask;
    if (low < s) {
        uint64_t threshold = (full - s) % s;
        if (low < threshold) return 0;
    }
    *value = (uint32_t)(m >> bits);
    return 1;
}

/* ---------------------------------------------------------------- draws */

#define TAG_SCATTER 1u
#define TAG_FY 2u
#define TAG_FY_RETRY 3u

uint32_t oracle_bucket(uint64_t seed, uint32_t level, uint64_t o, uint64_t pos, uint32_t k)
{
    uint64_t q = pos >> 2;
    uint32_t out[4];
    philox_seeded(seed, (uint32_t)q, (uint32_t)(q >> 32), level | (TAG_SCATTER << 8), (uint32_t)o, out);
    uint32_t word = out[pos & 3];
    return (uint32_t)(((uint64_t)word * (uint64_t)k) >> 32);
}

/* Partner j in [0, i] for Fisher-Yates step i of the subproblem at o. */
uint64_t oracle_fy_draw(uint64_t seed, uint32_t level, uint64_t o, uint64_t i)
{
    uint64_t p = o + i;
    uint64_t s = i + 1;
    uint64_t q = p >> 2;
    uint32_t out[4];
    uint32_t v;
    philox_seeded(seed, (uint32_t)q, (uint32_t)(q >> 32), level | (TAG_FY << 8), (uint32_t)o, out);
    if (oracle_lemire_try(32, s, out[p & 3], &v)) return v;
    for (uint32_t attempt = 1; attempt < 65536u; ++attempt) {
        philox_seeded(seed, (uint32_t)p, (uint32_t)(p >> 32),
                      level | (TAG_FY_RETRY << 8) | (attempt << 16), (uint32_t)o, out);
        for (int wd = 0; wd < 4; ++wd)
            if (oracle_lemire_try(32, s, out[wd], &v)) return v;
    }
    return 0; /* unreachable in practice: 262141 consecutive rejections */
}

/* ---------------------------------------------------------------- FY */

static void swap_elems(unsigned char *a, unsigned char *b, uint32_t w, unsigned char *tmp)
{
    memcpy(tmp, a, w);
    memcpy(a, b, w);
    memcpy(b, tmp, w);
}

/* Returns 0 on success, -1 if the subproblem is too large for 32-bit draws. */
int oracle_fisher_yates(void *data, uint64_t m, uint32_t w, uint64_t seed, uint64_t o, uint32_t level)
{
    if (m > ((uint64_t)1 << 32)) return -1;
    unsigned char *y = (unsigned char *)data;
    unsigned char tmp[256];
    unsigned char *t = w <= sizeof(tmp) ? tmp : (unsigned char *)malloc(w);
    for (uint64_t i = m; i-- > 1;) {
        uint64_t j = oracle_fy_draw(seed, level, o, i);
        if (j != i) swap_elems(y + i * w, y + j * w, w, t);
    }
    if (t != tmp) free(t);
    return 0;
}

/* ---------------------------------------------------------------- one level */

/* One scatter level of the subproblem data[0..m) whose first element sits at
 * logical global position o.  Out-of-place into a temporary, then copied
 * back.  bucket_sizes (k entries) receives |bucket b|.  Returns 0 or -1 on
 * allocation failure. */
int oracle_scatter_level(void *data, uint64_t m, uint32_t w, uint64_t seed, uint64_t o,
                         uint32_t level, uint32_t k, uint64_t T, uint32_t B, uint64_t *bucket_sizes)
{
    unsigned char *x = (unsigned char *)data;
    uint64_t tiles = (m + T - 1) / T;
    uint32_t *bkt = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)calloc(tiles * k + 1, sizeof(uint64_t));      /* C[t][b]          */
    uint64_t *full_before = (uint64_t *)calloc(tiles * k + 1, sizeof(uint64_t)); /* sum_{t'<t} F    */
    uint64_t *tail_before = (uint64_t *)calloc(tiles * k + 1, sizeof(uint64_t)); /* sum_{t'<t} R    */
    uint64_t *rank = (uint64_t *)calloc(tiles * k + 1, sizeof(uint64_t));
    uint64_t *start = (uint64_t *)calloc((uint64_t)k + 1, sizeof(uint64_t));
    uint64_t *full_total = (uint64_t *)calloc((uint64_t)k + 1, sizeof(uint64_t));
    unsigned char *out = (unsigned char *)malloc((m ? m : 1) * w);
    if (!bkt || !cnt || !full_before || !tail_before || !rank || !start || !full_total || !out) {
        free(bkt); free(cnt); free(full_before); free(tail_before); free(rank);
        free(start); free(full_total); free(out);
        return -1;
    }

    /* draws and per-tile counts */
    for (uint64_t i = 0; i < m; ++i) {
        bkt[i] = oracle_bucket(seed, level, o, o + i, k);
        cnt[(i / T) * k + bkt[i]] += 1;
    }
    /* bucket sizes, region starts, per-bucket prefix over tiles */
    for (uint32_t b = 0; b < k; ++b) {
        uint64_t size = 0, fsum = 0, rsum = 0;
        for (uint64_t t = 0; t < tiles; ++t) {
            uint64_t c = cnt[t * k + b];
            full_before[t * k + b] = fsum;
            tail_before[t * k + b] = rsum;
            fsum += c / B;
            rsum += c % B;
            size += c;
        }
        full_total[b] = fsum;
        bucket_sizes[b] = size;
    }
    start[0] = 0;
    for (uint32_t b = 0; b < k; ++b) start[b + 1] = start[b] + bucket_sizes[b];

    /* place every element: stable within its tile and bucket */
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t t = i / T;
        uint32_t b = bkt[i];
        uint64_t idx = t * k + b;
        uint64_t r = rank[idx]++;
        uint64_t in_full = (cnt[idx] / B) * B;
        uint64_t dest;
        if (r < in_full)
            dest = start[b] + full_before[idx] * B + r;
        else
            dest = start[b] + full_total[b] * B + tail_before[idx] + (r - in_full);
        memcpy(out + dest * w, x + i * w, w);
    }
    memcpy(x, out, m * w);

    free(bkt); free(cnt); free(full_before); free(tail_before); free(rank);
    free(start); free(full_total); free(out);
    return 0;
}

/* ---------------------------------------------------------------- recursion */

typedef struct {
    uint32_t num_levels;
    uint32_t k[ORACLE_MAX_LEVEL_PARAMS];
    uint64_t T[ORACLE_MAX_LEVEL_PARAMS];
    uint32_t B[ORACLE_MAX_LEVEL_PARAMS];
    uint64_t base;
    uint32_t max_levels;
} oracle_plan_t;

static int shuffle_rec(unsigned char *x, uint64_t m, uint32_t w, uint64_t seed, uint64_t o,
                       uint32_t level, const oracle_plan_t *p)
{
    uint32_t cap = p->max_levels ? p->max_levels : ORACLE_DEPTH_CAP;
    if (m <= p->base || level >= cap)
        return oracle_fisher_yates(x, m, w, seed, o, level);
    uint32_t li = level < p->num_levels ? level : p->num_levels - 1;
    uint32_t k = p->k[li];
    uint64_t *sizes = (uint64_t *)malloc((uint64_t)k * sizeof(uint64_t));
    if (!sizes) return -1;
    if (oracle_scatter_level(x, m, w, seed, o, level, k, p->T[li], p->B[li], sizes)) {
        free(sizes);
        return -1;
    }
    uint64_t s = 0;
    int rc = 0;
    for (uint32_t b = 0; b < k && rc == 0; ++b) {
        if (sizes[b] > 0) rc = shuffle_rec(x + s * w, sizes[b], w, seed, o + s, level + 1, p);
        s += sizes[b];
    }
    free(sizes);
    return rc;
}

static int plan_ok(uint32_t num_levels, const uint32_t *ks, const uint64_t *Ts, const uint32_t *Bs,
                   uint64_t base)
{
    if (num_levels < 1 || num_levels > ORACLE_MAX_LEVEL_PARAMS || base < 1) return 0;
    for (uint32_t l = 0; l < num_levels; ++l) {
        uint32_t k = ks[l];
        if (k < 2 || (k & (k - 1)) != 0) return 0;
        if (Bs[l] < 1 || Ts[l] < 1 || Ts[l] % Bs[l] != 0) return 0;
    }
    return 1;
}

/* Shuffle data[0..n) (elements of w bytes) in the canonical order for
 * (seed, plan).  Returns 0, or -1 on invalid arguments / allocation failure. */
int oracle_shuffle(void *data, uint64_t n, uint32_t w, uint64_t seed, uint32_t num_levels,
                   const uint32_t *ks, const uint64_t *Ts, const uint32_t *Bs, uint64_t base,
                   uint32_t max_levels)
{
    if (w < 1 || (n > 0 && !data)) return -1;
    if (!plan_ok(num_levels, ks, Ts, Bs, base)) return -1;
    oracle_plan_t p;
    memset(&p, 0, sizeof(p));
    p.num_levels = num_levels;
    for (uint32_t l = 0; l < num_levels; ++l) {
        p.k[l] = ks[l];
        p.T[l] = Ts[l];
        p.B[l] = Bs[l];
    }
    p.base = base;
    p.max_levels = max_levels;
    if (n <= 1) return 0;
    return shuffle_rec((unsigned char *)data, n, w, seed, 0, 0, &p);
}

/* The remaining recursion of one subproblem: data[0..m) sits at logical
 * offset o and level L of its array (the children of a level are independent,
 * Sec. 4, so callers may run several of these concurrently). */
int oracle_shuffle_sub(void *data, uint64_t m, uint32_t w, uint64_t seed, uint64_t o, uint32_t level,
                       uint32_t num_levels, const uint32_t *ks, const uint64_t *Ts, const uint32_t *Bs,
                       uint64_t base, uint32_t max_levels)
{
    if (w < 1 || (m > 0 && !data)) return -1;
    if (!plan_ok(num_levels, ks, Ts, Bs, base)) return -1;
    oracle_plan_t p;
    memset(&p, 0, sizeof(p));
    p.num_levels = num_levels;
    for (uint32_t l = 0; l < num_levels; ++l) {
        p.k[l] = ks[l];
        p.T[l] = Ts[l];
        p.B[l] = Bs[l];
    }
    p.base = base;
    p.max_levels = max_levels;
    if (m <= 1) return 0;
    return shuffle_rec((unsigned char *)data, m, w, seed, o, level, &p);
}

/* Batched form: array i (ptrs[i], ns[i] elements) is shuffled with seed
 * base_seed + i and positions relative to its own start. */
int oracle_shuffle_batched(void *const *ptrs, const uint64_t *ns, uint32_t count, uint32_t w,
                           uint64_t base_seed, uint32_t num_levels, const uint32_t *ks,
                           const uint64_t *Ts, const uint32_t *Bs, uint64_t base, uint32_t max_levels)
{
    for (uint32_t i = 0; i < count; ++i) {
        int rc = oracle_shuffle(ptrs[i], ns[i], w, base_seed + i, num_levels, ks, Ts, Bs, base, max_levels);
        if (rc) return rc;
    }
    return 0;
}

/* ---------------------------------------------------------------- hash */

/* splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014). */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The finaliser above, exported so tests can pin it to published outputs. */
uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }

/* Position-dependent 64-bit digest of an array:
 *   H = sum_p splitmix64(p * 0x9E3779B97F4A7C15 ^ v(p))  (mod 2^64),
 *   v = chain of splitmix64 over the element's 8-byte little-endian words
 *   (a short last word is zero-padded). */
/* Digest of n elements that sit at positions p0 .. p0+n-1 of a longer array:
 * the position-dependent sum above restricted to those positions (the digest
 * of a whole array is the sum of the digests of its pieces, mod 2^64). */
uint64_t oracle_hash_at(const void *data, uint64_t n, uint32_t w, uint64_t p0)
{
    const unsigned char *x = (const unsigned char *)data;
    uint64_t h = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t p = p0 + i;
        uint64_t v = 0;
        for (uint32_t off = 0; off < w; off += 8) {
            uint64_t word = 0;
            uint32_t len = (w - off) < 8 ? (w - off) : 8;
            for (uint32_t c = 0; c < len; ++c) word |= (uint64_t)x[i * w + off + c] << (8 * c);
            v = splitmix64(v ^ word);
        }
        h += splitmix64(p * 0x9E3779B97F4A7C15ull ^ v);
    }
    return h;
}

uint64_t oracle_hash(const void *data, uint64_t n, uint32_t w)
{
    const unsigned char *x = (const unsigned char *)data;
    uint64_t h = 0;
    for (uint64_t p = 0; p < n; ++p) {
        uint64_t v = 0;
        for (uint32_t off = 0; off < w; off += 8) {
            uint64_t word = 0;
            uint32_t len = (w - off) < 8 ? (w - off) : 8;
            for (uint32_t c = 0; c < len; ++c) word |= (uint64_t)x[p * w + off + c] << (8 * c);
            v = splitmix64(v ^ word);
        }
        h += splitmix64(p * 0x9E3779B97F4A7C15ull ^ v);
    }
    return h;
}

/* Statistics helper: `count` independent shuffles of the same template, seed
 * seed0 + r for run r, written one after another to out (count*n*w bytes). */
int oracle_shuffle_many(const void *tmpl, uint64_t n, uint32_t w, uint64_t seed0, uint64_t count,
                        uint32_t num_levels, const uint32_t *ks, const uint64_t *Ts,
                        const uint32_t *Bs, uint64_t base, uint32_t max_levels, void *out)
{
    unsigned char *dst = (unsigned char *)out;
    for (uint64_t r = 0; r < count; ++r) {
        memcpy(dst + r * n * w, tmpl, n * w);
        int rc = oracle_shuffle(dst + r * n * w, n, w, seed0 + r, num_levels, ks, Ts, Bs, base, max_levels);
        if (rc) return rc;
    }
    return 0;
}

/* ---------------------------------------------------------------- streaming level */

/* The canonical layout of one scatter level (oracle_scatter_level) for an
 * input too large to hold twice, when element values are a function of their
 * position ("iota": the element at array position p has value p, truncated to
 * w bytes for w < 8, and p in its first 8 bytes otherwise).  The same
 * definitions, evaluated piecewise: counts for a range of tiles, then the
 * placement of the elements of a range of tiles whose buckets lie in a range
 * of buckets.  Used to check near-capacity runs by digest and sampled ranges
 * (the subproblems the level creates are then finished by oracle_shuffle_sub).
 * Four consecutive positions share one Philox call exactly as oracle_bucket
 * defines (word pos & 3 of the call for pos >> 2). */

static void quad_buckets(uint64_t seed, uint32_t level, uint64_t o, uint64_t q, uint32_t k, uint32_t b[4])
{
    uint32_t out[4];
    philox_seeded(seed, (uint32_t)q, (uint32_t)(q >> 32), level | (TAG_SCATTER << 8), (uint32_t)o, out);
    for (int j = 0; j < 4; ++j) b[j] = (uint32_t)(((uint64_t)out[j] * (uint64_t)k) >> 32);
}

/* cnt[(t - t_lo) * k + b] = number of elements of tile t in bucket b, t in [t_lo, t_hi);
 * the subproblem holds positions o .. o+m-1. */
int oracle_level_counts(uint64_t m, uint64_t seed, uint64_t o, uint32_t level, uint32_t k, uint64_t T,
                        uint64_t t_lo, uint64_t t_hi, uint64_t *cnt)
{
    if (T == 0 || k == 0) return -1;
    memset(cnt, 0, (t_hi - t_lo) * k * sizeof(uint64_t));
    for (uint64_t t = t_lo; t < t_hi; ++t) {
        uint64_t lo = t * T, hi = lo + T < m ? lo + T : m;
        uint64_t *c = cnt + (t - t_lo) * k;
        uint64_t i = lo;
        while (i < hi) {
            uint64_t pos = o + i;
            uint32_t b[4];
            quad_buckets(seed, level, o, pos >> 2, k, b);
            for (uint64_t j = pos & 3; j < 4 && i < hi; ++j, ++i) c[b[j]] += 1;
        }
    }
    return 0;
}

static void iota_value(uint64_t p, uint32_t w, unsigned char *dst)
{
    memset(dst, 0, w);
    for (uint32_t c = 0; c < 8 && c < w; ++c) dst[c] = (unsigned char)(p >> (8 * c));
}

/* Places the elements of tiles [t_lo, t_hi) whose bucket is in [b_lo, b_hi) at
 * their level output positions (relative to o), writing those in
 * [out_base, out_base + out_len) to out.  cnt, full_before and tail_before are
 * indexed by (tile, bucket) over all tiles of the subproblem; start and
 * full_total by bucket -- all as oracle_scatter_level defines them. */
int oracle_level_place_iota(uint64_t m, uint32_t w, uint64_t seed, uint64_t o, uint32_t level, uint32_t k,
                            uint64_t T, uint32_t B, uint64_t t_lo, uint64_t t_hi, uint32_t b_lo, uint32_t b_hi,
                            const uint64_t *cnt, const uint64_t *full_before, const uint64_t *tail_before,
                            const uint64_t *start, const uint64_t *full_total, void *out, uint64_t out_base,
                            uint64_t out_len)
{
    unsigned char *dst = (unsigned char *)out;
    uint64_t *rank = (uint64_t *)calloc((uint64_t)k + 1, sizeof(uint64_t));
    if (!rank || T == 0 || B == 0) {
        free(rank);
        return -1;
    }
    for (uint64_t t = t_lo; t < t_hi; ++t) {
        memset(rank, 0, (uint64_t)k * sizeof(uint64_t));
        uint64_t lo = t * T, hi = lo + T < m ? lo + T : m;
        uint64_t i = lo;
        while (i < hi) {
            uint64_t pos = o + i;
            uint32_t bq[4];
            quad_buckets(seed, level, o, pos >> 2, k, bq);
            for (uint64_t j = pos & 3; j < 4 && i < hi; ++j, ++i) {
                uint32_t b = bq[j];
                uint64_t r = rank[b]++;
                if (b < b_lo || b >= b_hi) continue;
                uint64_t idx = t * k + b;
                uint64_t in_full = (cnt[idx] / B) * B;
                uint64_t dest;
                if (r < in_full)
                    dest = start[b] + full_before[idx] * B + r;
                else
                    dest = start[b] + full_total[b] * B + tail_before[idx] + (r - in_full);
                if (dest >= out_base && dest - out_base < out_len) iota_value(o + i, w, dst + (dest - out_base) * w);
            }
        }
    }
    free(rank);
    return 0;
}
