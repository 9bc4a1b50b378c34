/*
 * leysort -- GPU record sort (C ABI).
 *
 * Sorts fixed-size records by a fixed-size key prefix, following the problem
 * statement of Leyenda (arXiv 1909.08006): Section 1 and Section 4.1 fix the
 * workload (100-byte records, a 10-byte key, 90-byte value; data sets that fit,
 * partly fit, or do not fit a memory limit), Section 3.1 / Algorithm 1 the
 * method (adaptive MSD radix partitioning with small- and tiny-bucket
 * finishing), Section 3.2 the (key, pointer) tuples, the record scatter and the
 * external sort-merge pipeline.
 *
 * Order: keys compare as unsigned byte strings, byte 0 most significant.  Equal
 * keys keep their input order (the sort is stable), so the output is unique:
 * out[j] = in[p(j)] with (key(p(j)), p(j)) strictly increasing.
 *
 * Conventions for every entry point:
 *  - Pointers are plain device or host addresses; sizes are element counts.
 *  - `stream` is a cudaStream_t (the CUstream handle) passed as void*; NULL is
 *    the legacy default stream.
 *  - Device buffers must be 16-byte aligned.  Inputs are never written.
 *    Output buffers must not overlap inputs.
 *  - The caller owns all buffers it passes.  The library allocates its own
 *    scratch stream-ordered on `stream` from a per-device memory pool of its
 *    own and frees it before the call's work ends; every scratch byte counts
 *    against `mem_budget` (0 = no cap).  The pool keeps freed memory mapped
 *    for later calls, and external sorts keep their pinned host scratch (the
 *    sorted runs), until ley_release_cache().
 *  - Errors found on the host are returned before any work is queued.  Errors
 *    found by a kernel (a bounded wait that gave up) are latched in a
 *    per-device status word read by ley_last_device_status().
 *  - The first call on a device sets that device's current context's L2
 *    fetch granularity limit (cudaLimitMaxL2FetchGranularity) to 32 bytes,
 *    because the key reads and record gathers touch scattered 32-byte
 *    sectors.  The limit is a performance hint of the caller's context and
 *    ends with it; the environment variable LEY_L2_FETCH_BYTES=<0..128> picks
 *    another value and LEY_L2_FETCH_BYTES=keep leaves the context's own.
 */
#ifndef LEYSORT_H
#define LEYSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LEY_OK = 0,
    LEY_EINVAL = 1,       /* bad argument: NULL, misaligned, overlap, mixed memory kinds */
    LEY_ENOMEM = 2,       /* scratch would exceed mem_budget, or an allocation failed */
    LEY_EUNSUPPORTED = 3, /* geometry outside the supported range */
    LEY_ECUDA = 4,        /* a CUDA runtime call failed */
    LEY_ETIMEOUT = 5      /* a kernel's bounded wait gave up (device-side status) */
} ley_status;

typedef void* ley_stream_t;

/*
 * Sort n records of rec_bytes bytes by their first key_bytes bytes.
 * (Algorithm 1 and Section 3.1; the (key, pointer) tuples and record scatter
 * of Section 3.2; geometry of Section 4.1.)
 *
 *   in, out     n * rec_bytes bytes each, records back to back (array of
 *               structs).  Both on the device: the internal sort, queued on
 *               `stream` and asynchronous.  Both in pinned host memory
 *               (cudaHostAlloc / cudaHostRegister): the partially in-memory
 *               sort when the input plus scratch fits mem_budget, else the
 *               external run-formation + k-way merge sort; these block until
 *               the sorted records are in `out`.  Any other combination
 *               (mixed, pageable host memory) is LEY_EINVAL.
 *   rec_bytes   key_bytes..4096, any size (100 takes the specialised kernels;
 *               sizes that are a multiple of 4 are gathered in words, others
 *               in bytes).
 *   key_bytes   1..rec_bytes; the key is at offset 0.  A (key, pointer) tuple
 *               holds 12 key bytes, so a longer key is sorted one 12-byte
 *               window at a time, least significant window first
 *               (ceil(key_bytes / 12) sorts, each stable on the order left by
 *               the windows after it); scratch grows by 12 bytes per record.
 *               In the external mode each run and each merge partition is
 *               sorted that way (a partition's slices, in run order, sorted
 *               stably give its merge).
 *   mem_budget  cap on the library's device allocations in bytes, 0 = none.
 *   n           < 2^32.  n == 0 returns LEY_OK without touching the buffers.
 */
ley_status ley_sort_records(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                            uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream);

/*
 * As ley_sort_records, but a sort of pinned host buffers in the partially
 * in-memory mode (Section 4.1) is only queued on `stream`: the call returns
 * once the copy in, the sort and the copy out are enqueued, and the caller
 * synchronises `stream` before reading `out`, changing `in` or freeing
 * either.  Calls on different streams run concurrently, so one sort's copy
 * out overlaps the next one's copy in on the two directions of the host
 * link.  Each call in flight holds its own device scratch (n * rec_bytes plus
 * the workspace, within mem_budget).  Where the input does not fit the
 * partial mode the external sort runs and the call blocks, as
 * ley_sort_records does.  Device buffers: identical to ley_sort_records.
 * Errors found after the call returned surface at the stream's
 * synchronisation (CUDA errors) or in ley_last_device_status (device-side
 * status).
 */
ley_status ley_sort_records_async(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                                  uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream);

/*
 * Sort (key, payload) pairs: keys_in[i] as unsigned 64-bit, ties by input
 * position i; idx_in[i] travels with its key.  This is the key-pointer sort of
 * Section 3.2 (and the prefix/pointer pairs of Section 2.1) without a record
 * gather.  All four arrays on the device, n elements each, asynchronous on
 * `stream`.  keys_out/idx_out must not overlap the inputs.
 */
ley_status ley_sort_keys_index(const uint64_t* keys_in, const uint32_t* idx_in,
                               uint64_t* keys_out, uint32_t* idx_out, uint64_t n,
                               uint64_t mem_budget, ley_stream_t stream);

/*
 * Batched sorts: many independent requests of uneven sizes sorted by one
 * sequence of launches, each request exactly as its own ley_sort_records /
 * ley_sort_keys_index call would sort it.  (The paper sorts one data set; a
 * batch is this library's form of many small sorts, the requests being the
 * top-level buckets of one MSD sort -- Algorithm 1 never moves a tuple out
 * of its bucket.)
 *
 *   reqs[count]  host array, read before the call returns; requests with
 *                n == 0 are skipped.  All buffers on the device, as for the
 *                single-request call (records 16-byte aligned; keys 8, payloads
 *                4); a request's outputs must not overlap its inputs, and no
 *                request's buffers may overlap another request's outputs.
 *   sum over requests of n rounded up to 4096 must be < 2^32.
 * Asynchronous on `stream`; scratch (about 36 B per record slot, plus 4 B for
 * record sizes other than 100) counts against mem_budget.  The call does no
 * host synchronisation and no pageable copies, so it can be captured in a
 * CUDA graph (the request array is copied into the launches' parameters).
 */
typedef struct {
    const void* in;  /* n * rec_bytes bytes */
    void* out;       /* n * rec_bytes bytes */
    uint64_t n;
} ley_records_request;

ley_status ley_sort_records_batch(const ley_records_request* reqs, uint32_t count,
                                  uint32_t rec_bytes, uint32_t key_bytes, uint64_t mem_budget,
                                  ley_stream_t stream);

typedef struct {
    const uint64_t* keys_in;
    const uint32_t* idx_in;
    uint64_t* keys_out;
    uint32_t* idx_out;
    uint64_t n;
} ley_pairs_request;

ley_status ley_sort_keys_index_batch(const ley_pairs_request* reqs, uint32_t count,
                                     uint64_t mem_budget, ley_stream_t stream);

/*
 * Sort server: continuous batching of sort requests on the current device.
 * The paper has no counterpart (it sorts one data set per run); this is the
 * serving form of the batched sorts above.
 *
 * Requests are submitted from any host thread with their device buffers
 * already allocated (same rules as the single-request calls); submission
 * never blocks on the GPU.  A scheduler thread admits pending requests in
 * arrival order into a batch while one of `slots` launch streams is free and
 * the request's device memory -- its input and output plus its share of the
 * sort scratch -- fits `mem_budget` together with everything already in
 * flight (a single request larger than the budget runs alone).  Requests that
 * arrive while batches run join the next batch as soon as a slot and memory
 * free up, so batches on different slots overlap on the device.  At most
 * `max_batch` requests go into one batch.  Every request is sorted exactly as
 * its own ley_sort_records / ley_sort_keys_index call would sort it.
 *
 * Submission checks the request's arguments like the single-request call
 * (a rejected request gets no ticket).  ley_server_wait blocks until the
 * request is done, returns its status (as ley_last_device_status would report
 * it for the batch that carried it), its submit / launch / completion times
 * on the host clock in seconds since the server was created, and its batch's
 * interval on the device clock; a ticket can be waited for once.
 * ley_server_destroy finishes all submitted work, then stops the server's
 * threads.
 */
typedef struct ley_server ley_server;

typedef struct {
    double submit_s;     /* submission (host clock) */
    double start_s;      /* its batch was launched (host clock) */
    double done_s;       /* its batch's completion was observed on the host */
    double dev_start_s;  /* device clock, seconds after an event recorded at server
                            creation: a timing event on the batch's launch stream
                            just before its first kernel, i.e. when the stream
                            reached the batch's work */
    double dev_done_s;   /* device clock: the event after the batch's last kernel
                            (negative if the batch could not be timed) */
    uint64_t batch;      /* the batch that carried the request: 1, 2, ... in launch order */
} ley_server_times;

typedef struct {
    uint64_t pending;           /* submitted, not yet admitted */
    uint64_t inflight_batches;  /* launched, not yet completed */
    uint64_t launched_batches;  /* since creation */
    uint64_t bytes_in_use;      /* device bytes charged to admitted requests */
} ley_server_counters;

ley_status ley_server_create(ley_server** server, uint64_t mem_budget, uint32_t max_batch,
                             uint32_t slots);
ley_status ley_server_submit_records(ley_server* server, const void* in, void* out, uint64_t n,
                                     uint32_t rec_bytes, uint32_t key_bytes, uint64_t* ticket);
ley_status ley_server_submit_pairs(ley_server* server, const uint64_t* keys_in,
                                   const uint32_t* idx_in, uint64_t* keys_out, uint32_t* idx_out,
                                   uint64_t n, uint64_t* ticket);
ley_status ley_server_wait(ley_server* server, uint64_t ticket, ley_server_times* times);
ley_status ley_server_stats(ley_server* server, ley_server_counters* counters);
ley_status ley_server_destroy(ley_server* server);

/*
 * One round of Algorithm 1 (Section 3.1, "Cache Aware Scattering Process"):
 * the histogram of key byte `digit` and the stable partition of the records
 * into the 256 buckets of that byte.
 *   order_out  device, n x u32: order_out[j] = input index of the record that
 *              the partition places at position j (buckets in byte order,
 *              input order inside a bucket).
 *   hist_out   device, 256 x u64: bucket sizes.
 * digit < key_bytes.  Device `in` only.  Asynchronous on `stream`.
 */
ley_status ley_partition_records(const void* in, uint64_t n, uint32_t rec_bytes,
                                 uint32_t key_bytes, uint32_t digit, uint32_t* order_out,
                                 uint64_t* hist_out, ley_stream_t stream);

/*
 * Partition planning of the external sort's merge (Section 3.2: the merge is
 * cut into independent pieces for load balance): the merged order of k
 * sorted runs, in the order (key, run, position) -- equal keys of a lower
 * run first -- is cut into partitions of at most `cap` records by an exact
 * k-way co-rank.  Host-only: no device work, and no GPU is needed.
 *   runs[i]    host pointer to run i: run_len[i] records of rec_bytes bytes,
 *              sorted stably by their first key_bytes bytes.
 *   k          1..4096 runs (empty runs allowed).
 *   cap        the largest partition, in records (>= 1).
 *   cuts       out: *ncuts rows of k positions, row-major.  Row p holds, for
 *              every run, the position at which partition p starts: row 0 is
 *              all zeros, the last row is run_len, and partition p takes
 *              records [cuts[p][i], cuts[p+1][i]) of every run i.
 *   max_cuts   rows available in cuts; LEY_ENOMEM (with *ncuts set to the
 *              rows needed) if more are needed.
 * Partitions are about 3/4 of cap; their boundaries are exact, so merging
 * each partition's slices alone and concatenating gives the full merge.
 */
ley_status ley_plan_partitions(const void* const* runs, const uint64_t* run_len, uint32_t k,
                               uint32_t rec_bytes, uint32_t key_bytes, uint64_t cap,
                               uint64_t* cuts, uint64_t max_cuts, uint64_t* ncuts);

/*
 * K-way merge of sorted runs: the merge stage of the external sort
 * (Section 3.2, Figure 1: "a K-way merge algorithm"), exposed on its own.
 *   runs       device, run_start[k] records back to back; run r holds records
 *              run_start[r] .. run_start[r+1]-1 and must already be sorted by
 *              key (stable), e.g. by ley_sort_records.
 *   run_start  host array of k+1 record offsets, run_start[0] = 0, non-decreasing
 *              (empty runs allowed); read before the call returns.
 *   k          1..128.
 *   out        device, run_start[k] records: the stable merge, equal keys
 *              ordered by run, then by position in the run.
 * Asynchronous on `stream`.  Unsorted runs give an unspecified order (still a
 * permutation of the records).
 */
ley_status ley_merge_records(const void* runs, const uint64_t* run_start, uint32_t k, void* out,
                             uint32_t rec_bytes, uint32_t key_bytes, ley_stream_t stream);

/*
 * Device scratch (bytes) that ley_sort_records allocates for n records of
 * this geometry (Sections 1 and 4.1: a data set sorted under a memory limit),
 * so that a caller can size a sort before making it.  Host-only; needs no GPU.
 *   mem_budget == 0  the internal sort of device buffers.  (With device
 *                    buffers and a budget, the internal sort allocates the
 *                    same bytes and returns LEY_ENOMEM when they exceed the
 *                    budget.)
 *   mem_budget > 0   the sort of pinned host buffers under that budget: the
 *                    partially in-memory mode's device bytes (the resident
 *                    input, the workspace, the staging buffers) when they fit,
 *                    else the external mode's (its rotating run buffers,
 *                    workspaces and staging); LEY_ENOMEM, with *bytes = 0,
 *                    when neither fits.  The external mode's pinned host
 *                    scratch (n * rec_bytes bytes, the sorted runs) is host
 *                    memory and not counted.
 */
ley_status ley_workspace_bytes(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                               uint64_t mem_budget, uint64_t* bytes);

/*
 * Pinned host scratch (bytes) that ley_sort_records keeps for the sorted runs
 * of an external sort of n records under mem_budget (Section 3.2: the runs
 * are written out, then merged): 0 when the partially in-memory mode is used
 * (or mem_budget == 0), LEY_ENOMEM when no mode fits.  The external sort
 * keeps its last runs sorted in device memory, as many as fit the budget
 * beside its pipeline, so this is less than n * rec_bytes when the budget
 * allows; the link then carries the input in, the host runs out and back,
 * and the output out.  The scratch is allocated at the first such sort and
 * kept until ley_release_cache().  Host-only; needs no GPU.
 */
ley_status ley_host_scratch_bytes(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                                  uint64_t mem_budget, uint64_t* bytes);

/*
 * Returns the memory this library keeps between calls: the unused part of
 * each device's scratch pool and the pinned host scratch of the external
 * sort.  Call it when no sort of this library is running (on any stream);
 * later sorts allocate again.
 */
ley_status ley_release_cache(void);

/*
 * Tunables of the sort on the current device.  None of them changes a
 * result; they decide which path a bucket takes (the bigBucketThreshold and
 * tinyBucketThreshold of Section 3.1, Algorithm 1, which the paper leaves
 * unstated) and how many CTAs per SM the finishing and scatter kernels run.
 * They apply to sorts started after ley_set_tuning returns; a sort already
 * started keeps the tuning it read when it started.  The allocation-free
 * entry point always uses the defaults.
 */
typedef struct {
    uint32_t big_bucket;          /* buckets above this many tuples are scattered again;
                                     256..2048, default 2048 (one finishing CTA's capacity) */
    uint32_t tiny_bucket;         /* sub-buckets up to this many tuples are finished by
                                     comparison ranking; 32..256, default 64 */
    uint32_t finish_ctas_per_sm;  /* 0 = as many as fit (default) */
    uint32_t pass_ctas_per_sm;    /* 0 = as many as fit (default) */
} ley_tuning;

ley_status ley_get_tuning(ley_tuning* tuning);
/* NULL restores the defaults; out-of-range values are LEY_EINVAL. */
ley_status ley_set_tuning(const ley_tuning* tuning);

/*
 * Autotuner: sorts n uniform random records of this geometry (generated on
 * the device from `seed`) under each of a grid of tunings -- big bucket
 * 2048 / 1536 / 1024, tiny bucket 32 / 64 / 128, finishing CTAs per SM as
 * many as fit / 3 -- keeps the fastest (best of two timed sorts each, after
 * one warm-up), makes it the current tuning and returns it in *best.
 * Allocates 2 * n * rec_bytes bytes plus one sort's scratch; blocks.
 */
ley_status ley_autotune_records(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                                uint64_t seed, ley_tuning* best);

/*
 * The same autotuner on the caller's own records: `in` is n records of
 * rec_bytes on the device (16-byte aligned), read and never written; the
 * timed sorts go to scratch of n * rec_bytes bytes.  Thresholds that suit
 * one key distribution (say uniform) can be slower on another (say skewed),
 * so tuning on the data to be sorted is the reliable form.  The timed sorts
 * run on a stream of the library's own that first waits for the work queued
 * on `stream` before the call (the work that may still be writing `in`).
 * Blocks.
 *
 * Both autotuners time every candidate as that sort's own tuning and make
 * the winner current only when they return: sorts started by other threads
 * meanwhile keep the tuning that was current before.  Every sort reads the
 * current tuning once, when it starts, and uses that copy throughout.
 */
ley_status ley_autotune_records_on(const void* in, uint64_t n, uint32_t rec_bytes,
                                   uint32_t key_bytes, ley_tuning* best, ley_stream_t stream);

/* Static English text for a status code (never NULL). */
const char* ley_status_string(ley_status s);

/*
 * Waits for `stream`, then returns and clears the device-side status of the
 * current device: LEY_ETIMEOUT if any kernel's bounded wait gave up since the
 * last call, LEY_ECUDA if the stream reports an error, else LEY_OK.
 */
ley_status ley_last_device_status(ley_stream_t stream);

/*
 * Allocation-free record sort, for callers that cannot allocate device
 * memory: for example an application whose device memory is entirely owned by
 * its own pool allocator, or a latency-bound caller for which a cudaMalloc
 * (which can wait for the whole device) is not acceptable.  The paper has no
 * counterpart; this is an interface of this library only.
 *
 * Same sort and arguments as ley_sort_records with both buffers on the device
 * (16-byte aligned, not overlapping), but the call never allocates or frees:
 * its scratch is one fixed device array of 12 MiB inside this library, which
 * every GPU that loads the library holds until the process exits.
 *   n           at most LEY_NOALLOC_MAX_RECORDS; larger n returns LEY_ENOMEM
 *               before any work.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current).  The call waits for its work on `stream`
 * and returns its device-side status (LEY_ETIMEOUT if a bounded wait gave up).  All calls share the one
 * array and each leaves its contents behind: calls whose work overlaps on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.
 */
#define LEY_NOALLOC_MAX_RECORDS 262144ull

ley_status ley_sort_records_noalloc(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                                    uint32_t key_bytes, ley_stream_t stream);

/*
 * Failure-detection self-test: launches a kernel whose bounded wait cannot
 * succeed -- which = 0: a device word that nothing writes (the kind of wait
 * of the scan's look-back); which = 1: an mbarrier whose bytes no copy
 * delivers (the kind of wait of the standalone TMA gather of the host
 * modes) -- waits for it and returns the device status it latched, which is
 * LEY_ETIMEOUT when detection works.
 * The status word is cleared on return and the context stays usable.  Takes
 * about as long as one wait's limit (a second or less).
 */
ley_status ley_selftest_timeout(uint32_t which, ley_stream_t stream);

/* Number of kernels this library has launched in this process. */
uint64_t ley_launch_count(void);

/*
 * Per-kernel timing for tracing (Table 3 style per-phase times).  While
 * enabled, every launch of the library is bracketed by CUDA events on its
 * stream.  ley_profile_read() waits for those events and fills up to `max`
 * entries {name, launches, total milliseconds} summed since the last
 * ley_profile_enable(1); it returns the number of kernel names seen.
 */
typedef struct {
    const char* name;
    uint64_t launches;
    double total_ms;
} ley_kernel_time;

ley_status ley_profile_enable(int on);
int ley_profile_read(ley_kernel_time* out, int max);

#ifdef __cplusplus
}
#endif

#endif /* LEYSORT_H */
