/*
 * leysort oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the record sort
 * computes.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library; the product path never does.  It shares
 * no code, header or table with the CUDA implementation.
 *
 * What the sort computes (Leyenda, Section 3.1 and Algorithm 1; record geometry
 * from Section 4.1): records of rec_bytes bytes whose first key_bytes bytes are
 * the key.  Keys compare as unsigned byte strings, byte 0 most significant --
 * the reading under which Algorithm 1's 256 buckets per key byte, taken from
 * the most significant byte down, produce sorted output.  The paper does not
 * state how equal keys are ordered; this oracle takes the stable reading: the
 * output is out[j] = in[p(j)], where p is the unique permutation that makes
 * (K(p(j)), p(j)) strictly increasing.  Because (key, index) is a strict total
 * order, that permutation is unique, so any correct sort must match it byte
 * for byte.
 *
 * The key-pointer variant (Section 3.2, "(key, pointer) tuples"; the
 * AlphaSort-style prefix/pointer pairs of Section 2.1) sorts (u64 key,
 * u32 payload) pairs by (key, input position); the payload travels with its key.
 *
 * Every function below is pinned by a CPU test against something other than
 * itself: brute force over all permutations, numpy's stable lexsort, the
 * worked partition example of Section 2.2, planted mistakes and invariants.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ sort */

typedef struct {
    const uint8_t* base;
    uint64_t rec;
    uint32_t key;
} rec_ctx;

/* Order of Section 3.1 under the stable reading: key bytes as an unsigned
 * string (memcmp), then original index. */
static int cmp_record_index(const void* pa, const void* pb, void* arg) {
    const rec_ctx* c = (const rec_ctx*)arg;
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    int r = memcmp(c->base + a * c->rec, c->base + b * c->rec, c->key);
    if (r != 0) return r < 0 ? -1 : 1;
    return (a < b) ? -1 : (a > b ? 1 : 0);
}

/* Sorts n records: out[j] = in[perm[j]].  perm_out (may be NULL) receives
 * the permutation.  Returns 0, or -1 if memory runs out. */
ORACLE_API int oracle_sort_records(const uint8_t* in, uint8_t* out, uint64_t n,
                                   uint32_t rec_bytes, uint32_t key_bytes,
                                   uint64_t* perm_out) {
    uint64_t* idx = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; i++) idx[i] = i;
    rec_ctx c = {in, rec_bytes, key_bytes};
    qsort_r(idx, n, sizeof(uint64_t), cmp_record_index, &c);
    for (uint64_t j = 0; j < n; j++) {
        if (out) memcpy(out + j * rec_bytes, in + idx[j] * rec_bytes, rec_bytes);
        if (perm_out) perm_out[j] = idx[j];
    }
    free(idx);
    return 0;
}

typedef struct {
    const uint64_t* keys;
} pair_ctx;

static int cmp_pair_index(const void* pa, const void* pb, void* arg) {
    const pair_ctx* c = (const pair_ctx*)arg;
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    uint64_t ka = c->keys[a], kb = c->keys[b];
    if (ka != kb) return ka < kb ? -1 : 1;
    return (a < b) ? -1 : (a > b ? 1 : 0);
}

/* Key-pointer pairs: sort by (keys_in[i] as unsigned u64, i); the u32
 * payload idx_in[i] travels with its key. */
ORACLE_API int oracle_sort_keys_index(const uint64_t* keys_in, const uint32_t* idx_in,
                                      uint64_t* keys_out, uint32_t* idx_out,
                                      uint64_t n) {
    uint64_t* idx = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; i++) idx[i] = i;
    pair_ctx c = {keys_in};
    qsort_r(idx, n, sizeof(uint64_t), cmp_pair_index, &c);
    for (uint64_t j = 0; j < n; j++) {
        keys_out[j] = keys_in[idx[j]];
        idx_out[j] = idx_in[idx[j]];
    }
    free(idx);
    return 0;
}

/* ------------------------------------------------- one round of Alg. 1 */

/* Section 3.1, "Cache Aware Scattering Process": the histogram of the
 * current radix (key byte `digit`) gives each bucket's size. */
ORACLE_API void oracle_digit_histogram(const uint8_t* in, uint64_t n, uint32_t rec_bytes,
                                       uint32_t digit, uint64_t* hist256) {
    for (int b = 0; b < 256; b++) hist256[b] = 0;
    for (uint64_t i = 0; i < n; i++) hist256[in[i * rec_bytes + digit]]++;
}

/* One round of Algorithm 1 over the whole input: records go to the bucket of
 * their byte `digit`, buckets in increasing byte order, and inside a bucket
 * in input order (the stable reading).  order_out[j] = index of the record
 * placed at position j.  Written as the textbook counting sort: histogram,
 * exclusive offsets, then placement in input order. */
ORACLE_API void oracle_msd_partition(const uint8_t* in, uint64_t n, uint32_t rec_bytes,
                                     uint32_t digit, uint64_t* order_out) {
    uint64_t hist[256], next[256];
    oracle_digit_histogram(in, n, rec_bytes, digit, hist);
    uint64_t run = 0;
    for (int b = 0; b < 256; b++) {
        next[b] = run;
        run += hist[b];
    }
    for (uint64_t i = 0; i < n; i++) order_out[next[in[i * rec_bytes + digit]]++] = i;
}

/* ------------------------------------------------------ k-way merge */

/* Section 3.2, merge stage: k sorted runs, stored back to back in `runs`
 * (run r holds records run_start[r] .. run_start[r+1]-1), merged into `out`
 * by the textbook k-way selection: each output record is the smallest head
 * key, ties going to the lower-numbered run.  O(n k). */
ORACLE_API void oracle_kway_merge_records(const uint8_t* runs, const uint64_t* run_start,
                                          uint32_t k, uint32_t rec_bytes,
                                          uint32_t key_bytes, uint8_t* out) {
    uint64_t* head = (uint64_t*)malloc((k ? k : 1) * sizeof(uint64_t));
    for (uint32_t r = 0; r < k; r++) head[r] = run_start[r];
    uint64_t total = run_start[k] - run_start[0];
    for (uint64_t j = 0; j < total; j++) {
        int best = -1;
        for (uint32_t r = 0; r < k; r++) {
            if (head[r] >= run_start[r + 1]) continue;
            if (best < 0 || memcmp(runs + head[r] * rec_bytes,
                                   runs + head[best] * rec_bytes, key_bytes) < 0)
                best = (int)r;
        }
        memcpy(out + j * rec_bytes, runs + head[best] * rec_bytes, rec_bytes);
        head[best]++;
    }
    free(head);
}

/* ---------------------------------------------- checks at any size */

/* rank(i) = #{m : (K(m), m) < (K(i), i)}: the output position of input
 * record i, straight from the definition.  Each sample scans all n records. */
ORACLE_API void oracle_rank_records(const uint8_t* in, uint64_t n, uint32_t rec_bytes,
                                    uint32_t key_bytes, const uint64_t* samples,
                                    uint64_t n_samples, uint64_t* ranks) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < (int64_t)n_samples; s++) {
        uint64_t i = samples[s], r = 0;
        const uint8_t* ki = in + i * rec_bytes;
        for (uint64_t m = 0; m < n; m++) {
            int c = memcmp(in + m * rec_bytes, ki, key_bytes);
            if (c < 0 || (c == 0 && m < i)) r++;
        }
        ranks[s] = r;
    }
}

ORACLE_API void oracle_rank_pairs(const uint64_t* keys, uint64_t n,
                                  const uint64_t* samples, uint64_t n_samples,
                                  uint64_t* ranks) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < (int64_t)n_samples; s++) {
        uint64_t i = samples[s], r = 0, ki = keys[i];
        for (uint64_t m = 0; m < n; m++)
            if (keys[m] < ki || (keys[m] == ki && m < i)) r++;
        ranks[s] = r;
    }
}

/* First j with K(j) > K(j+1), or -1 when keys never decrease. */
ORACLE_API int64_t oracle_check_sorted(const uint8_t* buf, uint64_t n, uint32_t rec_bytes,
                                       uint32_t key_bytes) {
    for (uint64_t j = 0; j + 1 < n; j++)
        if (memcmp(buf + j * rec_bytes, buf + (j + 1) * rec_bytes, key_bytes) > 0)
            return (int64_t)j;
    return -1;
}

/* 64-bit hash of one record (FNV-1a over its bytes, then the SplitMix64
 * finaliser to spread the bits). */
static uint64_t record_hash(const uint8_t* p, uint32_t len) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (uint32_t b = 0; b < len; b++) {
        h ^= p[b];
        h *= 0x100000001b3ull;
    }
    h ^= h >> 30;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 27;
    h *= 0x94d049bb133111ebull;
    return h ^ (h >> 31);
}

/* Multiset fingerprint: sum over records of record_hash mod 2^64.  Equal for
 * a buffer and any permutation of its records. */
ORACLE_API uint64_t oracle_record_hash_sum(const uint8_t* buf, uint64_t n, uint32_t rec_bytes) {
    uint64_t sum = 0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
    for (int64_t j = 0; j < (int64_t)n; j++) sum += record_hash(buf + (uint64_t)j * rec_bytes, rec_bytes);
    return sum;
}

/* Complete check of a sorted output whose records carry their input index as
 * a little-endian u32 at byte tag_off (outside the key).  It holds exactly
 * when out equals the oracle's answer:
 *   (1) every tag t_j is < n and no tag repeats (out is a permutation),
 *   (2) out[j] is byte-equal to in[t_j],
 *   (3) (K(j), t_j) strictly increases with j.
 * Returns -1 on success, else the first failing position j (or n if the
 * bitmap cannot be allocated). */
ORACLE_API int64_t oracle_check_tagged(const uint8_t* out, const uint8_t* in, uint64_t n,
                                       uint32_t rec_bytes, uint32_t key_bytes,
                                       uint32_t tag_off) {
    uint8_t* seen = (uint8_t*)calloc(n ? n : 1, 1);
    if (!seen) return (int64_t)n;
    int64_t bad = -1;
    uint32_t prev_tag = 0;
    for (uint64_t j = 0; j < n && bad < 0; j++) {
        const uint8_t* o = out + j * rec_bytes;
        uint32_t t = (uint32_t)o[tag_off] | ((uint32_t)o[tag_off + 1] << 8) |
                     ((uint32_t)o[tag_off + 2] << 16) | ((uint32_t)o[tag_off + 3] << 24);
        if (t >= n || seen[t]) { bad = (int64_t)j; break; }
        seen[t] = 1;
        if (memcmp(o, in + (uint64_t)t * rec_bytes, rec_bytes) != 0) { bad = (int64_t)j; break; }
        if (j > 0) {
            int c = memcmp(out + (j - 1) * rec_bytes, o, key_bytes);
            if (c > 0 || (c == 0 && prev_tag >= t)) { bad = (int64_t)j; break; }
        }
        prev_tag = t;
    }
    free(seen);
    return bad;
}

/* Same complete check for pairs whose input payload is the input position:
 * idx_out[j] < n and distinct, keys_out[j] == keys_in[idx_out[j]], and
 * (keys_out[j], idx_out[j]) strictly increasing. */
ORACLE_API int64_t oracle_check_pairs_tagged(const uint64_t* keys_out, const uint32_t* idx_out,
                                             const uint64_t* keys_in, uint64_t n) {
    uint8_t* seen = (uint8_t*)calloc(n ? n : 1, 1);
    if (!seen) return (int64_t)n;
    int64_t bad = -1;
    for (uint64_t j = 0; j < n; j++) {
        uint32_t t = idx_out[j];
        if (t >= n || seen[t] || keys_out[j] != keys_in[t]) { bad = (int64_t)j; break; }
        seen[t] = 1;
        if (j > 0 && (keys_out[j - 1] > keys_out[j] ||
                      (keys_out[j - 1] == keys_out[j] && idx_out[j - 1] >= t))) {
            bad = (int64_t)j;
            break;
        }
    }
    free(seen);
    return bad;
}
