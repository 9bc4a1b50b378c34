// Launch wrappers of the leysort kernels (host-side declarations).
#pragma once

#include "ley_internal.cuh"

namespace ley {

// Launches kern on stream s with programmatic stream serialization, so that
// it may be scheduled while the kernel before it in the stream still runs;
// the kernel itself waits (griddepcontrol.wait) before touching memory.
// LEY_PDL=0 launches plainly.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct LaunchCfg {
    int grid;
    int block;
    size_t smem;
    cudaStream_t stream;
};

// Records -> tuples, histogram of key byte `hist_digit`, key-difference mask
// of the whole input (list 0, slot 0).
cudaError_t launch_extract_records(const LaunchCfg& c, const uint8_t* in, unsigned long long n,
                                   uint32_t rec_bytes, KeySpec ks, const Work& w, int hist_digit);
// Same, for tiles [t_begin, t_end) only (kPassTile records each).  The
// key-difference mask is taken against the key of the record at ref_in
// (default: record 0 at `in`), which must be the same in every launch over
// one input.
cudaError_t launch_extract_records_tiles(const LaunchCfg& c, const uint8_t* in,
                                         unsigned long long n, uint32_t rec_bytes, KeySpec ks,
                                         const Work& w, int hist_digit, uint32_t t_begin,
                                         uint32_t t_end, const uint8_t* ref_in = nullptr);
cudaError_t launch_extract_pairs(const LaunchCfg& c, const uint64_t* keys, const uint32_t* idx,
                                 unsigned long long n, KeySpec ks, const Work& w);
cudaError_t launch_init(cudaStream_t s, const Work& w, unsigned long long n, int digit0);
cudaError_t launch_hist(const LaunchCfg& c, const Work& w, KeySpec ks, int level);
cudaError_t launch_scan(const LaunchCfg& c, const Work& w, int level);
cudaError_t launch_classify(const LaunchCfg& c, const Work& w, KeySpec ks, int level);
cudaError_t launch_classify_partition(cudaStream_t s, const Work& w);
cudaError_t launch_pass(const LaunchCfg& c, const Work& w, KeySpec ks, int level);
cudaError_t launch_finish_records(const LaunchCfg& c, const Work& w, KeySpec ks);
// Finish + record gather in one kernel (100-byte records): out[j] is written
// directly, no permutation; source indices are < n_in.
cudaError_t launch_finish_gather(const LaunchCfg& c, const Work& w, KeySpec ks, const uint8_t* in,
                                 uint8_t* out, unsigned long long n_in);
cudaError_t launch_finish_pairs(const LaunchCfg& c, const Work& w, KeySpec ks, uint64_t* keys_out,
                                uint32_t* idx_out);
// out[j] = in[perm[j]] for j < n; perm entries are < n_in (records at `in`).
cudaError_t launch_gather(const LaunchCfg& c, const uint8_t* in, uint8_t* out,
                          const uint32_t* perm, unsigned long long n, unsigned long long n_in,
                          uint32_t rec_bytes, int variant);
cudaError_t launch_gather_err(const LaunchCfg& c, const uint8_t* in, uint8_t* out,
                              const uint32_t* perm, unsigned long long n, unsigned long long n_in,
                              uint32_t rec_bytes, int variant, uint32_t* err);
// Keys longer than 12 bytes: tuples of the 12-byte window at koff of record
// order[j] (identity if order is null), carrying j; and the composition
// next[j] = order[pass[j]] (pass[j] if order is null).
cudaError_t launch_extract_window(const LaunchCfg& c, const uint8_t* in, const uint32_t* order,
                                  unsigned long long n, uint32_t rec, uint32_t koff, KeySpec ks,
                                  const Work& w);
cudaError_t launch_compose_order(cudaStream_t s, int grid, const uint32_t* order,
                                 const uint32_t* pass, uint32_t* next, unsigned long long n,
                                 uint32_t* err);
// Batched sorts (requests back to back in one tuple space, see BatchReq).
cudaError_t launch_batch_setup(cudaStream_t s, const BatchReq* reqs, uint32_t R, const Work& w,
                               uint32_t* tile_req, uint32_t ntiles, int digit0);
cudaError_t launch_batch_extract_records(const LaunchCfg& c, const BatchReq* reqs,
                                         const uint32_t* tile_req, uint32_t ntiles, uint32_t rec,
                                         KeySpec ks, const Work& w);
cudaError_t launch_batch_extract_pairs(const LaunchCfg& c, const BatchReq* reqs,
                                       const uint32_t* tile_req, uint32_t ntiles, const Work& w);
// Finish of a batch: 100-byte records gathered into place (pairs = false), or
// sorted keys and payloads (pairs = true), into each request's own arrays.
cudaError_t launch_batch_finish(const LaunchCfg& c, const Work& w, KeySpec ks,
                                const BatchReq* reqs, const uint32_t* tile_req, bool pairs);
cudaError_t launch_batch_gather_generic(cudaStream_t s, int grid, const BatchReq* reqs,
                                        const uint32_t* tile_req, const uint32_t* perm,
                                        unsigned long long npos, uint32_t rec, uint32_t* err);
// dst[0, bytes) = src (host), stream-ordered through kernel parameters (no
// host buffer needs to outlive the call; capturable in a CUDA graph).
cudaError_t launch_upload(cudaStream_t s, void* dst, const void* src, size_t bytes);
// A bounded wait that cannot succeed (which = 0: a device word nobody sets,
// which = 1: an mbarrier no copy completes); latches kErrTimeout in err.
cudaError_t launch_selftest_wait(cudaStream_t s, uint32_t which,
                                 const unsigned long long* never_set, uint32_t* err);
// p[0, bytes) = uniform random bytes from `seed` (8-byte aligned p).
cudaError_t launch_fill_random(cudaStream_t s, uint8_t* p, unsigned long long bytes,
                               unsigned long long seed);
cudaError_t launch_partition_out(cudaStream_t s, int grid, const Work& w, unsigned long long n,
                                 uint32_t* order_out, unsigned long long* hist_out);

// K-way merge (ley_merge.cu): one round of pairwise merge-path merges of the
// k sorted runs at src (run r at [off[r], off[r+1])) into dst.
cudaError_t launch_merge_round(cudaStream_t s, int grid, const uint4* src, uint4* dst,
                               const unsigned long long* off_dev, uint32_t k, uint32_t lo_mask);
cudaError_t launch_halve_offsets(cudaStream_t s, unsigned long long* off, uint32_t runs);
// Partition planning of the external merge on the device: for ncand
// candidates (candidate c of run i at position (c - cbase[i] + 1) * step - 1,
// cbase[k] = ncand) the co-rank in every run, split[c * k + j], and its rank
// in the merged order (key, run, position), rank[c].  Runs are device
// memory or pinned host memory mapped for the device; keys of kb <= 12 bytes.
struct PlanRun {
    const uint8_t* base;
    unsigned long long len;
};
cudaError_t launch_corank(cudaStream_t st, int sms, const PlanRun* runs, uint32_t k, uint32_t rec,
                          uint32_t kb, const unsigned long long* cbase, unsigned long long step,
                          uint32_t ncand, uint32_t* split, unsigned long long* rank,
                          uint32_t* err);
// K-way merge path in one pass (k <= kKwayMaxRuns): the sample split table
// ((S + 1) rows of k u32, S = sum over runs of ceil(len / kway_sample_step(k)))
// and the tile merges; perm[j] = w of the j-th tuple of the merge of the
// sorted runs at tup (run r at [off[r], off[r+1]), n tuples in all).
constexpr int kKwayMaxRuns = 32;
constexpr int kKwayTile = 4096;
uint32_t kway_sample_step(uint32_t k);
cudaError_t launch_kmerge(cudaStream_t st, int sms, const uint4* tup,
                          const unsigned long long* off_dev, uint32_t k, uint32_t S,
                          uint32_t lo_mask, uint32_t* table, unsigned long long table_rows,
                          uint32_t* perm, unsigned long long n, uint32_t* err);
// dst[0, count) = host[0, count), count <= kMaxOffsets, stream-ordered on s
// (the values travel in the kernel's parameters).
constexpr int kMaxOffsets = 129;  // k + 1 offsets of at most 128 runs
cudaError_t launch_set_offsets(cudaStream_t s, unsigned long long* dst,
                               const unsigned long long* host, uint32_t count);
cudaError_t launch_tuple_index(cudaStream_t s, int grid, const uint4* t, uint32_t* perm,
                               unsigned long long n);

// Occupancy-derived persistent grid sizes (blocks per SM) for a kernel kind.
enum KernelKind {
    KK_EXTRACT_REC = 0, KK_EXTRACT_PAIRS, KK_HIST, KK_SCAN, KK_PASS, KK_FINISH_REC, KK_FINISH_PAIRS,
    KK_GATHER100, KK_GATHER100_TMA, KK_GATHER_GENERIC, KK_FINISH_GATHER, KK_COUNT
};
int blocks_per_sm(KernelKind k);
size_t kernel_smem(KernelKind k);
int kernel_threads(KernelKind k);

}  // namespace ley
