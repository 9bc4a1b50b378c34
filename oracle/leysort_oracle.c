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
#include <pthread.h>
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

/* ------------------------------------------ the same sort on T threads */

/* The sort of oracle_sort_records on T host threads, the multi-core form of
 * the CPU baseline (it is timed, never used to produce expected values).
 *  1. The input is cut into T contiguous index ranges ("chunks"); each thread
 *     sorts its chunk's (key, index) order with the same comparison.
 *  2. T-1 pivots split the merged order into T pieces: 32 evenly spaced
 *     elements of every sorted chunk are sorted together and every 32nd is
 *     taken (the classic sample split of a parallel merge).
 *  3. Thread t merges piece t: in every chunk, the elements from pivot t
 *     (inclusive) to pivot t+1 (exclusive), found by binary search, by a
 *     binary min-heap of sub-range heads (the textbook T-way merge), into the
 *     output positions that follow all elements below pivot t.
 *  4. T threads copy the records into place.
 * The chunks are contiguous and every comparison includes the index, so the
 * order is exactly the single-threaded one. */
#define SAMPLES_PER_CHUNK 32

typedef struct {
    const uint8_t* in;
    uint8_t* out;
    uint64_t* idx;          /* sorted chunks, in place */
    uint64_t* perm;         /* merged order */
    const uint64_t* cb;     /* chunk boundaries, T + 1 entries */
    const uint64_t* pivot;  /* T + 1 entries: pivot t is an element index; entries 0 and T
                               are unused (no lower, no upper bound) */
    uint64_t lo, hi;        /* this thread's chunk (step 1) or output range (step 4) */
    uint32_t t, T, rec, key;
} par_job;

static void* sort_chunk(void* arg) {
    par_job* j = (par_job*)arg;
    for (uint64_t i = j->lo; i < j->hi; i++) j->idx[i] = i;
    rec_ctx c = {j->in, j->rec, j->key};
    qsort_r(j->idx + j->lo, j->hi - j->lo, sizeof(uint64_t), cmp_record_index, &c);
    return NULL;
}

/* First position in sorted idx[lo, hi) whose element is not below element v. */
static uint64_t lower_bound_idx(const uint64_t* idx, uint64_t lo, uint64_t hi, uint64_t v,
                                rec_ctx* c) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (cmp_record_index(&idx[mid], &v, c) < 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static void sift_down(const uint64_t* idx, const uint64_t* pos, uint32_t* heap, uint32_t size,
                      uint32_t i, rec_ctx* c) {
    for (;;) {
        uint32_t m = i, l = 2 * i + 1, r = 2 * i + 2;
        if (l < size && cmp_record_index(&idx[pos[heap[l]]], &idx[pos[heap[m]]], c) < 0) m = l;
        if (r < size && cmp_record_index(&idx[pos[heap[r]]], &idx[pos[heap[m]]], c) < 0) m = r;
        if (m == i) return;
        uint32_t tmp = heap[i];
        heap[i] = heap[m];
        heap[m] = tmp;
        i = m;
    }
}

static void* merge_piece(void* arg) {
    par_job* j = (par_job*)arg;
    const uint32_t T = j->T, t = j->t;
    rec_ctx c = {j->in, j->rec, j->key};
    uint64_t* pos = (uint64_t*)malloc(T * sizeof(uint64_t));
    uint64_t* end = (uint64_t*)malloc(T * sizeof(uint64_t));
    uint32_t* heap = (uint32_t*)malloc(T * sizeof(uint32_t));
    if (!pos || !end || !heap) {
        free(pos);
        free(end);
        free(heap);
        j->lo = 1;  /* failure flag */
        return NULL;
    }
    uint64_t out = 0;  /* elements of all chunks below pivot t */
    for (uint32_t i = 0; i < T; i++) {
        const uint64_t a = j->cb[i], b = j->cb[i + 1];
        pos[i] = t == 0 ? a : lower_bound_idx(j->idx, a, b, j->pivot[t], &c);
        end[i] = t + 1 == T ? b : lower_bound_idx(j->idx, a, b, j->pivot[t + 1], &c);
        out += pos[i] - a;
    }
    uint32_t size = 0;
    for (uint32_t i = 0; i < T; i++)
        if (pos[i] < end[i]) heap[size++] = i;
    for (uint32_t i = size / 2; i-- > 0;) sift_down(j->idx, pos, heap, size, i, &c);
    while (size) {
        const uint32_t i = heap[0];
        j->perm[out++] = j->idx[pos[i]++];
        if (pos[i] == end[i]) heap[0] = heap[--size];
        if (size) sift_down(j->idx, pos, heap, size, 0, &c);
    }
    free(pos);
    free(end);
    free(heap);
    j->lo = 0;
    return NULL;
}

static void* copy_range(void* arg) {
    par_job* j = (par_job*)arg;
    for (uint64_t i = j->lo; i < j->hi; i++)
        memcpy(j->out + i * j->rec, j->in + j->perm[i] * j->rec, j->rec);
    return NULL;
}

/* Runs fn on jobs[0..T) in T threads; -2 if a thread cannot be started. */
static int run_threads(void* (*fn)(void*), par_job* jobs, pthread_t* th, uint32_t T) {
    for (uint32_t t = 0; t < T; t++)
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) {
            for (uint32_t u = 0; u < t; u++) pthread_join(th[u], NULL);
            return -2;
        }
    for (uint32_t t = 0; t < T; t++) pthread_join(th[t], NULL);
    return 0;
}

/* Sorts n records on T threads: out[j] = in[perm[j]] with the permutation of
 * oracle_sort_records.  Returns 0, -1 if memory runs out, -2 if a thread
 * cannot be started. */
ORACLE_API int oracle_sort_records_threads(const uint8_t* in, uint8_t* out, uint64_t n,
                                           uint32_t rec_bytes, uint32_t key_bytes,
                                           uint32_t threads) {
    uint32_t T = threads ? threads : 1;
    if ((uint64_t)T > n) T = n ? (uint32_t)n : 1;
    const uint64_t ns = (uint64_t)T * SAMPLES_PER_CHUNK;
    uint64_t* idx = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* perm = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* cb = (uint64_t*)malloc((T + 1) * sizeof(uint64_t));
    uint64_t* pivot = (uint64_t*)malloc((T + 1) * sizeof(uint64_t));
    uint64_t* samp = (uint64_t*)malloc(ns * sizeof(uint64_t));
    pthread_t* th = (pthread_t*)malloc(T * sizeof(pthread_t));
    par_job* jobs = (par_job*)malloc(T * sizeof(par_job));
    int rc = 0;
    if (!idx || !perm || !cb || !pivot || !samp || !th || !jobs) {
        rc = -1;
        goto done;
    }
    for (uint32_t t = 0; t <= T; t++) cb[t] = n * t / T;
    for (uint32_t t = 0; t < T; t++) {
        par_job j = {in, out, idx, perm, cb, pivot, cb[t], cb[t + 1], t, T, rec_bytes, key_bytes};
        jobs[t] = j;
    }
    /* 1. chunks sorted in parallel */
    if ((rc = run_threads(sort_chunk, jobs, th, T)) != 0) goto done;
    /* 2. pivots from evenly spaced samples of the sorted chunks */
    {
        uint64_t m = 0;
        for (uint32_t t = 0; t < T; t++) {
            const uint64_t len = cb[t + 1] - cb[t];
            for (uint32_t k = 0; k < SAMPLES_PER_CHUNK && len; k++)
                samp[m++] = idx[cb[t] + len * k / SAMPLES_PER_CHUNK];
        }
        rec_ctx c = {in, rec_bytes, key_bytes};
        qsort_r(samp, m, sizeof(uint64_t), cmp_record_index, &c);
        pivot[0] = pivot[T] = 0;
        for (uint32_t t = 1; t < T; t++) pivot[t] = samp[m * t / T];
    }
    /* 3. the T pieces of the merge, in parallel */
    if ((rc = run_threads(merge_piece, jobs, th, T)) != 0) goto done;
    for (uint32_t t = 0; t < T; t++)
        if (jobs[t].lo != 0) {
            rc = -1;
            goto done;
        }
    /* 4. the records copied into place in parallel */
    for (uint32_t t = 0; t < T; t++) {
        jobs[t].lo = cb[t];
        jobs[t].hi = cb[t + 1];
    }
    rc = run_threads(copy_range, jobs, th, T);
done:
    free(idx);
    free(perm);
    free(cb);
    free(pivot);
    free(samp);
    free(th);
    free(jobs);
    return rc;
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

/* The check of oracle_check_tagged on T host threads (for full-size
 * outputs): thread t checks output positions [n t / T, n (t + 1) / T), each
 * position against its predecessor (across range boundaries too), and marks
 * tags with an atomic exchange so that a tag seen twice is caught whichever
 * thread sees it second.  Returns -1 if the output is exact, else a bad
 * position (the first one a thread found; with a duplicated tag, either
 * occurrence). */
typedef struct {
    const uint8_t *out, *in;
    uint8_t* seen;
    uint64_t n, lo, hi;
    uint32_t rec, key, tag_off;
    int64_t bad;
} check_job;

static void* check_range(void* arg) {
    check_job* c = (check_job*)arg;
    c->bad = -1;
    for (uint64_t j = c->lo; j < c->hi; j++) {
        const uint8_t* o = c->out + j * c->rec;
        const uint8_t* q = o + c->tag_off;
        const uint32_t t = (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) |
                           ((uint32_t)q[3] << 24);
        if (t >= c->n || __atomic_exchange_n(&c->seen[t], (uint8_t)1, __ATOMIC_RELAXED)) {
            c->bad = (int64_t)j;
            return NULL;
        }
        if (memcmp(o, c->in + (uint64_t)t * c->rec, c->rec) != 0) {
            c->bad = (int64_t)j;
            return NULL;
        }
        if (j > 0) {
            const uint8_t* p = o - c->rec;
            const uint8_t* pq = p + c->tag_off;
            const uint32_t pt = (uint32_t)pq[0] | ((uint32_t)pq[1] << 8) |
                                ((uint32_t)pq[2] << 16) | ((uint32_t)pq[3] << 24);
            const int cm = memcmp(p, o, c->key);
            if (cm > 0 || (cm == 0 && pt >= t)) {
                c->bad = (int64_t)j;
                return NULL;
            }
        }
    }
    return NULL;
}

ORACLE_API int64_t oracle_check_tagged_threads(const uint8_t* out, const uint8_t* in, uint64_t n,
                                               uint32_t rec_bytes, uint32_t key_bytes,
                                               uint32_t tag_off, uint32_t threads) {
    uint32_t T = threads ? threads : 1;
    if ((uint64_t)T > n) T = n ? (uint32_t)n : 1;
    uint8_t* seen = (uint8_t*)calloc(n ? n : 1, 1);
    pthread_t* th = (pthread_t*)malloc(T * sizeof(pthread_t));
    check_job* jobs = (check_job*)malloc(T * sizeof(check_job));
    int64_t bad = -1;
    if (!seen || !th || !jobs) {
        bad = (int64_t)n;
        goto done;
    }
    uint32_t started = 0;
    for (uint32_t t = 0; t < T; t++) {
        check_job c = {out, in, seen, n, n * t / T, n * (t + 1) / T, rec_bytes, key_bytes,
                       tag_off, -1};
        jobs[t] = c;
    }
    for (; started < T; started++)
        if (pthread_create(&th[started], NULL, check_range, &jobs[started]) != 0) break;
    for (uint32_t t = 0; t < started; t++) pthread_join(th[t], NULL);
    if (started < T) {
        bad = (int64_t)n;  /* could not check everything */
        goto done;
    }
    for (uint32_t t = 0; t < T; t++)
        if (jobs[t].bad >= 0 && (bad < 0 || jobs[t].bad < bad)) bad = jobs[t].bad;
done:
    free(seen);
    free(th);
    free(jobs);
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
