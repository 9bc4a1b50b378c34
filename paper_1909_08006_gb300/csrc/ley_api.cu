// C ABI of leysort: argument checks, scratch layout, the launch sequence of
// the internal sort, and the host-memory (partially in-memory) mode.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "leysort.h"
#include "ley_kernels.h"

namespace ley {

using ull = unsigned long long;

// ------------------------------------------------------ per-device state

struct DevState {
    bool init = false;
    int sms = 0;
    uint32_t* err = nullptr;
    // The library's scratch comes from its own stream-ordered pool, which
    // keeps freed memory mapped for the next call (re-mapping tens of GB on
    // every call costs tens of milliseconds); ley_release_cache() trims it.
    cudaMemPool_t pool = nullptr;
};
static DevState g_dev[64];
static std::mutex g_mu;

// Tunables of the sort (ley_set_tuning / ley_autotune_records), per device.
// None of them changes a result: Algorithm 1's thresholds only decide which
// bucket takes which path.
struct Tuning {
    uint32_t big = kSmall;   // big-bucket threshold (bigBucketThreshold)
    uint32_t tiny = 64;      // tiny-bucket threshold (tinyBucketThreshold): measured best
                             // on skewed keys, neutral on uniform ones
    uint32_t fin_ctas = 0;   // finishing CTAs per SM, 0 = as many as fit
    uint32_t pass_ctas = 0;  // scatter CTAs per SM, 0 = as many as fit
};
static Tuning g_tune[64];

static Tuning cur_tuning() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return Tuning{};
    std::lock_guard<std::mutex> lk(g_mu);
    return g_tune[d];
}
static std::atomic<unsigned long long> g_launches{0};

// The record path reads 10..12-byte keys out of 100-byte records (extract)
// and 100-byte records at random positions (gather); at the context's
// default L2 fetch granularity each such read brings whole 64- or 128-byte
// lines in from HBM.  A 32-byte granularity fetches only the touched sectors
// (measured on GB300 at 1e8 records: extract 1.65 -> 0.98 ms, gather 5.03 ->
// 4.61 ms).  The limit is a per-context performance hint that ends with the
// context; LEY_L2_FETCH_BYTES=<0..128> picks another value, "keep" leaves the
// context's own.
static void set_l2_fetch_granularity() {
    size_t bytes = 32;
    if (const char* e = getenv("LEY_L2_FETCH_BYTES")) {
        if (strcmp(e, "keep") == 0) return;
        bytes = (size_t)strtoul(e, nullptr, 10);
        if (bytes > 128) bytes = 128;
    }
    if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, bytes) != cudaSuccess)
        (void)cudaGetLastError();  // a hint: an unsupported value changes nothing
}

static DevState* dev_state() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& s = g_dev[d];
    if (!s.init) {
        if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
            return nullptr;
        void* p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, 256) != cudaSuccess) return nullptr;
        s.err = static_cast<uint32_t*>(p);
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = d;
        if (cudaMemPoolCreate(&s.pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        if (cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
            return nullptr;
        // Memory freed on one stream is not handed to an allocation on another
        // by making the second stream wait for the first (the default): calls
        // on different streams (queued host-memory sorts, the server's slots)
        // would otherwise run one after the other.  Reuse of frees that have
        // already completed, and on the same stream, stays allowed.
        int no = 0;
        if (cudaMemPoolSetAttribute(s.pool, cudaMemPoolReuseAllowInternalDependencies, &no) !=
            cudaSuccess)
            return nullptr;
        (void)blocks_per_sm(KK_PASS);  // occupancy tables and smem attributes
        set_l2_fetch_granularity();
        s.init = true;
    }
    return &s;
}

// Stream-ordered scratch from the device's library pool.
static bool scratch_alloc(DevState* ds, void** p, size_t bytes, cudaStream_t st) {
    if (cudaMallocFromPoolAsync(p, bytes, ds->pool, st) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

uint32_t* device_err_word() {
    DevState* s = dev_state();
    return s ? s->err : nullptr;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("LEY_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// ------------------------------------------------------------- profiling

struct PendingEv {
    const char* name;
    cudaEvent_t a, b;
};
struct ProfEntry {
    const char* name;
    ull launches;
    double ms;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<PendingEv> g_pending;
static std::vector<ProfEntry> g_prof;
static std::vector<cudaEvent_t> g_ev_pool;

static cudaEvent_t take_event() {
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <class F>
static cudaError_t launch(const char* name, cudaStream_t s, F&& f) {
    cudaEvent_t a = nullptr;
    bool on;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        on = g_prof_on;
        if (on) a = take_event();
    }
    if (on) cudaEventRecord(a, s);
    cudaError_t e = f();
    g_launches.fetch_add(1);
    // LEY_DEBUG_SYNC=1: wait for every kernel and name the first that fails
    // (a debugging aid; off by default).
    static const bool dbg_sync = std::getenv("LEY_DEBUG_SYNC") != nullptr;
    if (dbg_sync && e == cudaSuccess) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            std::fprintf(stderr, "leysort: kernel %s failed: %s\n", name, cudaGetErrorString(e));
    }
    if (on) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        cudaEvent_t b = take_event();
        cudaEventRecord(b, s);
        g_pending.push_back({name, a, b});
    }
    return e;
}

// ---------------------------------------------------------------- layout

struct Layout {
    size_t tup[2], perm, ctl, segs[2], stb[2], sto[2], spass[2], hist[2], diff[2], tcnt, bb, fin,
        status;
    size_t total;
    ull cap_seg, cap_fin, cap_tiles, cap_chunks;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Scratch layout of one internal sort of n tuples; `big` (the big-bucket
// threshold of the sort's tuning) bounds the segment and task counts.
static Layout make_layout(ull n, bool with_perm, uint32_t big) {
    Layout L{};
    L.cap_seg = n / big + 2;
    L.cap_tiles = n / kPassTile + L.cap_seg + 1;
    L.cap_chunks = L.cap_tiles / kScanChunk + 1;
    L.cap_fin = 100 * (n / big + 1) + 16;
    size_t off = 0;
    auto put = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.tup[0] = put(n * sizeof(uint4));
    L.tup[1] = put(n * sizeof(uint4));
    L.perm = put(with_perm ? n * sizeof(uint32_t) : 0);
    L.ctl = put(sizeof(Ctl));
    for (int p = 0; p < 2; p++) {
        L.segs[p] = put(L.cap_seg * sizeof(Seg));
        L.stb[p] = put(L.cap_seg * sizeof(uint32_t));
        L.sto[p] = put(L.cap_tiles * sizeof(uint32_t));
        L.spass[p] = put(L.cap_seg * sizeof(uint32_t));
        L.hist[p] = put(L.cap_seg * kRadix * sizeof(uint32_t));
        L.diff[p] = put(L.cap_seg * sizeof(Diff));
    }
    L.tcnt = put(L.cap_tiles * kRadix * sizeof(uint32_t));
    L.bb = put(L.cap_seg * kRadix * sizeof(uint32_t));
    L.fin = put(L.cap_fin * sizeof(FinTask));
    L.status = put(L.cap_chunks * kRadix * sizeof(ull));
    L.total = off;
    return L;
}

static Work make_work(char* base, const Layout& L, ull n, uint32_t* err) {
    Work w{};
    w.tup[0] = reinterpret_cast<uint4*>(base + L.tup[0]);
    w.tup[1] = reinterpret_cast<uint4*>(base + L.tup[1]);
    w.perm = reinterpret_cast<uint32_t*>(base + L.perm);
    w.ctl = reinterpret_cast<Ctl*>(base + L.ctl);
    for (int p = 0; p < 2; p++) {
        w.segs[p] = reinterpret_cast<Seg*>(base + L.segs[p]);
        w.seg_tile_base[p] = reinterpret_cast<uint32_t*>(base + L.stb[p]);
        w.seg_tile_owner[p] = reinterpret_cast<uint32_t*>(base + L.sto[p]);
        w.seg_pass[p] = reinterpret_cast<uint32_t*>(base + L.spass[p]);
        w.hist[p] = reinterpret_cast<uint32_t*>(base + L.hist[p]);
        w.diff[p] = reinterpret_cast<Diff*>(base + L.diff[p]);
    }
    w.tile_cnt = reinterpret_cast<uint32_t*>(base + L.tcnt);
    w.bucket_base = reinterpret_cast<uint32_t*>(base + L.bb);
    w.fin = reinterpret_cast<FinTask*>(base + L.fin);
    w.status = reinterpret_cast<ull*>(base + L.status);
    w.err = err;
    w.cap_seg = L.cap_seg;
    w.cap_fin = L.cap_fin;
    w.cap_tiles = L.cap_tiles;
    w.cap_chunks = L.cap_chunks;
    w.n = n;
    return w;
}

static KeySpec record_keyspec(uint32_t kb, const Tuning& t) {
    KeySpec ks;
    ks.big = t.big;
    ks.tiny = t.tiny;
    ks.ndig = (int)kb;
    ks.hi_mask = kb >= 8 ? ~0ull : (~0ull << (64 - 8 * kb));
    ks.lo_mask = kb <= 8 ? 0u : (kb >= 12 ? ~0u : (~0u << (32 - 8 * (kb - 8))));
    return ks;
}

static KeySpec pair_keyspec(const Tuning& t) {
    KeySpec ks;
    ks.big = t.big;
    ks.tiny = t.tiny;
    ks.ndig = 8;
    ks.hi_mask = ~0ull;
    ks.lo_mask = 0u;
    return ks;
}

// Record gather for 100-byte records: by default the internal sort gathers
// the records inside the finishing kernel (2); the separate gather kernel
// with TMA bulk copies (1) serves the chunked host-memory modes, and
// LEY_GATHER=tma makes the internal sort use it too (a test of that kernel
// on the internal path).  Records read from host memory take the plain-load
// kernel (0), see stage_gather.
static int gather_variant() {
    const char* v = std::getenv("LEY_GATHER");
    if (v && std::strcmp(v, "tma") == 0) return 1;
    return 2;
}

// Whether an internal sort of this geometry fuses the gather into the finish
// (and so needs no permutation array).
static bool fused_gather(uint32_t rec) { return rec == 100 && gather_variant() == 2; }

// ----------------------------------------------------- the internal sort

enum Mode { MODE_RECORDS = 0, MODE_PAIRS = 1, MODE_PARTITION = 2 };

struct SortArgs {
    Mode mode;
    const uint8_t* in;        // records / partition
    uint8_t* out;             // records
    const uint64_t* keys_in;  // pairs
    const uint32_t* idx_in;
    uint64_t* keys_out;
    uint32_t* idx_out;
    uint32_t* order_out;      // partition
    ull* hist_out;
    ull n;
    uint32_t rec, kb, digit;
    bool in_host = false;     // records at `in` are pinned host memory mapped for the device
    // The tuning of this call, read once when the call starts: every layout,
    // key spec and grid of the call is sized from this copy, so a concurrent
    // ley_set_tuning (or the autotuner) cannot change it half-way.
    Tuning tune;
};

#define LEY_TRY(x)                                   \
    do {                                             \
        if ((x) != cudaSuccess) return LEY_ECUDA;    \
    } while (0)

// Stages of one internal sort, all queued on `st` with scratch described by w.

static ley_status stage_prepare(const Work& w, const Layout& L, cudaStream_t st, ull n,
                                int digit0) {
    LEY_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
    LEY_TRY(cudaMemsetAsync(w.diff[0], 0, sizeof(Diff), st));
    LEY_TRY(cudaMemsetAsync(w.status, 0, L.cap_chunks * kRadix * sizeof(ull), st));
    LEY_TRY(launch("init", st, [&] { return launch_init(st, w, n, digit0); }));
    return LEY_OK;
}

// Records [t_begin, t_end) tiles -> tuples and per-tile digit counts.
static ley_status stage_extract_records(const SortArgs& a, const Work& w, const KeySpec& ks,
                                        cudaStream_t st, int sms, int digit0, uint32_t t_begin,
                                        uint32_t t_end, const uint8_t* ref_in = nullptr) {
    LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_REC), 256, 0, st};
    LEY_TRY(launch("extract", st, [&] {
        return launch_extract_records_tiles(c, a.in, a.n, a.rec, ks, w, digit0, t_begin, t_end,
                                            ref_in);
    }));
    return LEY_OK;
}

// The MSD levels (histogram, offset scan, classify, scatter) and the
// small-bucket finish; records mode leaves the permutation in w.perm.
// Persistent grids: CTAs per SM as the tuning asks, at most what fits.
static int tuned_grid(int sms, KernelKind k, uint32_t want) {
    int b = blocks_per_sm(k);
    if (want && (int)want < b) b = (int)want;
    return sms * b;
}
static int pass_grid(int sms, const Tuning& t) { return tuned_grid(sms, KK_PASS, t.pass_ctas); }
static int fin_grid(int sms, KernelKind k, const Tuning& t) {
    return tuned_grid(sms, k, t.fin_ctas);
}

static ley_status stage_levels(const Work& w, const KeySpec& ks, cudaStream_t st, int sms,
                               const Tuning& t) {
    const LaunchCfg cp{pass_grid(sms, t), kPassThreads, kernel_smem(KK_PASS), st};
    const LaunchCfg cs{sms * blocks_per_sm(KK_SCAN), kRadix, 0, st};
    const LaunchCfg ch{sms * blocks_per_sm(KK_HIST), kHistThreads, 0, st};
    const LaunchCfg cc{8 * sms, 128, 0, st};
    for (int lvl = 0; lvl < ks.ndig; lvl++) {
        if (lvl > 0) LEY_TRY(launch("hist", st, [&] { return launch_hist(ch, w, ks, lvl); }));
        LEY_TRY(launch("scan", st, [&] { return launch_scan(cs, w, lvl); }));
        LEY_TRY(launch("classify", st, [&] { return launch_classify(cc, w, ks, lvl); }));
        LEY_TRY(launch("pass", st, [&] { return launch_pass(cp, w, ks, lvl); }));
    }
    return LEY_OK;
}

static ley_status stage_levels_finish(const SortArgs& a, const Work& w, const KeySpec& ks,
                                      cudaStream_t st, int sms, bool fuse = false) {
    ley_status s0 = stage_levels(w, ks, st, sms, a.tune);
    if (s0 != LEY_OK) return s0;
    if (a.mode == MODE_PAIRS) {
        LaunchCfg cf{fin_grid(sms, KK_FINISH_PAIRS, a.tune), kFinThreads,
                     kernel_smem(KK_FINISH_PAIRS), st};
        LEY_TRY(launch("finish", st, [&] {
            return launch_finish_pairs(cf, w, ks, a.keys_out, a.idx_out);
        }));
        return LEY_OK;
    }
    if (fuse) {  // records gathered into a.out by the finishing kernel itself
        LaunchCfg cf{fin_grid(sms, KK_FINISH_GATHER, a.tune), kFinThreads,
                     kernel_smem(KK_FINISH_GATHER), st};
        LEY_TRY(launch("finish_gather", st, [&] {
            return launch_finish_gather(cf, w, ks, a.in, a.out, a.n);
        }));
        return LEY_OK;
    }
    LaunchCfg cf{fin_grid(sms, KK_FINISH_REC, a.tune), kFinThreads, kernel_smem(KK_FINISH_REC),
                 st};
    LEY_TRY(launch("finish", st, [&] { return launch_finish_records(cf, w, ks); }));
    return LEY_OK;
}

// out_base[j - j0] = in[perm[j]] for output records j in [j0, j1).
static ley_status stage_gather(const SortArgs& a, const uint32_t* perm, cudaStream_t st, int sms,
                               ull j0, ull j1, uint8_t* out_base) {
    if (j1 <= j0) return LEY_OK;
    // Records read from host memory (over the host link) take the plain-load
    // kernel: bulk copies are only used on device memory.
    const int gv = a.rec == 100 && !a.in_host ? 1 : 0;
    const KernelKind gk = a.rec != 100 ? KK_GATHER_GENERIC
                                       : (gv == 1 ? KK_GATHER100_TMA : KK_GATHER100);
    LaunchCfg cg{sms * blocks_per_sm(gk), 0, 0, st};
    LEY_TRY(launch("gather", st, [&] {
        return launch_gather(cg, a.in, out_base, perm + j0, j1 - j0, a.n, a.rec, gv);
    }));
    return LEY_OK;
}

// Queues the whole sort on `st` using scratch at `base` (layout L).
static ley_status enqueue_sort(const SortArgs& a, char* base, const Layout& L, cudaStream_t st,
                               DevState* ds) {
    Work w = make_work(base, L, a.n, ds->err);
    const KeySpec ks = a.mode == MODE_PAIRS ? pair_keyspec(a.tune) : record_keyspec(a.kb, a.tune);
    const int sms = ds->sms;
    const int digit0 = a.mode == MODE_PARTITION ? (int)a.digit : 0;
    ley_status s = stage_prepare(w, L, st, a.n, digit0);
    if (s != LEY_OK) return s;
    if (a.mode == MODE_PAIRS) {
        LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_PAIRS), 256, 0, st};
        LEY_TRY(launch("extract", st, [&] {
            return launch_extract_pairs(c, a.keys_in, a.idx_in, a.n, ks, w);
        }));
    } else {
        s = stage_extract_records(a, w, ks, st, sms, digit0, 0, ceil_div_u64(a.n, kPassTile));
        if (s != LEY_OK) return s;
    }
    if (a.mode == MODE_PARTITION) {
        const LaunchCfg cp{pass_grid(sms, a.tune), kPassThreads, kernel_smem(KK_PASS), st};
        const LaunchCfg cs{sms * blocks_per_sm(KK_SCAN), kRadix, 0, st};
        LEY_TRY(launch("scan", st, [&] { return launch_scan(cs, w, 0); }));
        LEY_TRY(launch("classify", st, [&] { return launch_classify_partition(st, w); }));
        LEY_TRY(launch("pass", st, [&] { return launch_pass(cp, w, ks, 0); }));
        LEY_TRY(launch("partition_out", st, [&] {
            return launch_partition_out(st, sms * 4, w, a.n, a.order_out, a.hist_out);
        }));
        return LEY_OK;
    }
    const bool fuse = a.mode == MODE_RECORDS && fused_gather(a.rec);
    s = stage_levels_finish(a, w, ks, st, sms, fuse);
    if (s != LEY_OK || a.mode == MODE_PAIRS || fuse) return s;
    return stage_gather(a, w.perm, st, sms, 0, a.n, a.out);
}

// ------------------------------------------------------- batched sorts

// Sorts the requests of a batch (non-empty, offsets assigned, npos = end of
// the last request's tiles) as one sort over R top-level segments.
static ley_status run_batch(const std::vector<BatchReq>& reqs, ull npos, uint32_t rec,
                            uint32_t kb, bool pairs, ull budget, cudaStream_t st,
                            const Tuning& tune) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    const uint32_t R = (uint32_t)reqs.size();
    const bool fuse = !pairs && rec == 100;
    const Layout L = make_layout(npos, !pairs && !fuse, tune.big);
    const uint32_t ntiles = (uint32_t)(npos / kPassTile);
    const size_t rq_bytes = align_up(R * sizeof(BatchReq), 256);
    const size_t tr_bytes = align_up((size_t)ntiles * sizeof(uint32_t), 256);
    const size_t total = L.total + rq_bytes + tr_bytes;
    if (budget && total > budget) return LEY_ENOMEM;
    if (R > L.cap_seg) return LEY_EUNSUPPORTED;  // cannot happen: each request has a tile
    void* base = nullptr;
    if (!scratch_alloc(ds, &base, total, st)) return LEY_ENOMEM;
    char* b = static_cast<char*>(base);
    Work w = make_work(b, L, npos, ds->err);
    BatchReq* dreqs = reinterpret_cast<BatchReq*>(b + L.total);
    uint32_t* tile_req = reinterpret_cast<uint32_t*>(b + L.total + rq_bytes);
    const KeySpec ks = pairs ? pair_keyspec(tune) : record_keyspec(kb, tune);
    const int sms = ds->sms;
    ley_status s = LEY_OK;
    auto run = [&]() -> ley_status {
        LEY_TRY(launch("upload", st, [&] {
            return launch_upload(st, dreqs, reqs.data(), R * sizeof(BatchReq));
        }));
        ley_status t = stage_prepare(w, L, st, npos, 0);
        if (t != LEY_OK) return t;
        LEY_TRY(launch("batch_setup", st, [&] {
            return launch_batch_setup(st, dreqs, R, w, tile_req, ntiles, 0);
        }));
        LaunchCfg c{sms * blocks_per_sm(pairs ? KK_EXTRACT_PAIRS : KK_EXTRACT_REC), 256, 0, st};
        LEY_TRY(launch("extract", st, [&] {
            return pairs ? launch_batch_extract_pairs(c, dreqs, tile_req, ntiles, w)
                         : launch_batch_extract_records(c, dreqs, tile_req, ntiles, rec, ks, w);
        }));
        t = stage_levels(w, ks, st, sms, tune);
        if (t != LEY_OK) return t;
        if (pairs || fuse) {
            const KernelKind fk = pairs ? KK_FINISH_PAIRS : KK_FINISH_GATHER;
            LaunchCfg cf{fin_grid(sms, fk, tune), kFinThreads, kernel_smem(fk), st};
            LEY_TRY(launch("finish_gather", st, [&] {
                return launch_batch_finish(cf, w, ks, dreqs, tile_req, pairs);
            }));
            return LEY_OK;
        }
        LaunchCfg cf{fin_grid(sms, KK_FINISH_REC, tune), kFinThreads, kernel_smem(KK_FINISH_REC),
                     st};
        LEY_TRY(launch("finish", st, [&] { return launch_finish_records(cf, w, ks); }));
        LEY_TRY(launch("gather", st, [&] {
            return launch_batch_gather_generic(st, sms * blocks_per_sm(KK_GATHER_GENERIC), dreqs,
                                               tile_req, w.perm, npos, rec, w.err);
        }));
        return LEY_OK;
    };
    s = run();
    cudaFreeAsync(base, st);
    return s;
}

// ------------------------------------------------- keys longer than 12 bytes

// The tuple holds 12 key bytes.  A longer key is sorted window by window,
// least significant 12-byte window first; each window is one full MSD sort
// of (window, position in the order so far), so equal windows keep the order
// of the windows after them, and the composed order is the stable order of
// the whole key.  ceil(key_bytes / 12) sorts; `ord` holds two n-entry
// arrays; the final order is returned in *result.
static constexpr uint32_t kWindow = 12;

static ley_status enqueue_long_key_order(const SortArgs& a, const Work& w, const Layout& L,
                                         uint32_t* const ord[2], cudaStream_t st, int sms,
                                         const uint32_t** result) {
    const uint32_t W = (a.kb + kWindow - 1) / kWindow;
    const uint32_t* cur = nullptr;
    int nb = 0;
    for (int i = (int)W - 1; i >= 0; i--) {
        const uint32_t koff = kWindow * (uint32_t)i;
        const uint32_t wl = std::min(kWindow, a.kb - koff);
        const KeySpec ks = record_keyspec(wl, a.tune);
        ley_status s = stage_prepare(w, L, st, a.n, 0);
        if (s != LEY_OK) return s;
        LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_REC), 256, 0, st};
        LEY_TRY(launch("extract", st, [&] {
            return launch_extract_window(c, a.in, cur, a.n, a.rec, koff, ks, w);
        }));
        SortArgs b = a;
        b.kb = wl;
        s = stage_levels_finish(b, w, ks, st, sms, false);
        if (s != LEY_OK) return s;
        uint32_t* next = ord[nb];
        LEY_TRY(launch("compose", st, [&] {
            return launch_compose_order(st, sms * 4, cur, w.perm, next, a.n, w.err);
        }));
        cur = next;
        nb ^= 1;
    }
    *result = cur;
    return LEY_OK;
}

static size_t long_key_extra(ull n) { return 2 * align_up(n * sizeof(uint32_t), 256); }

static ley_status run_device_sort(const SortArgs& a, ull budget, cudaStream_t st) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    if (a.mode == MODE_RECORDS && a.kb > kWindow) {
        const Layout L = make_layout(a.n, true, a.tune.big);
        const size_t total = L.total + long_key_extra(a.n);
        if (budget && total > budget) return LEY_ENOMEM;
        void* base = nullptr;
        if (!scratch_alloc(ds, &base, total, st)) return LEY_ENOMEM;
        char* b = static_cast<char*>(base);
        Work w = make_work(b, L, a.n, ds->err);
        uint32_t* ord[2] = {reinterpret_cast<uint32_t*>(b + L.total),
                            reinterpret_cast<uint32_t*>(b + L.total + long_key_extra(a.n) / 2)};
        const uint32_t* order = nullptr;
        ley_status s = enqueue_long_key_order(a, w, L, ord, st, ds->sms, &order);
        if (s == LEY_OK) s = stage_gather(a, order, st, ds->sms, 0, a.n, a.out);
        cudaFreeAsync(base, st);
        return s;
    }
    const Layout L = make_layout(a.n, a.mode == MODE_RECORDS && !fused_gather(a.rec), a.tune.big);
    if (budget && L.total > budget) return LEY_ENOMEM;
    void* base = nullptr;
    if (!scratch_alloc(ds, &base, L.total, st)) return LEY_ENOMEM;
    ley_status s = enqueue_sort(a, static_cast<char*>(base), L, st, ds);
    cudaFreeAsync(base, st);
    return s;
}

// ------------------------------------------------- host-memory sorting

// Side streams and events of one host-memory sort (the reader and writer
// threads of Section 3.2 become two copy streams beside the compute stream).
struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaStream_t gth = nullptr;  // record gathers into the copy-out staging buffers
    std::vector<cudaEvent_t> evs;
    bool ok = true;
    // Whether the destructor waits for the side streams.  Without it the
    // streams and events are released once their work completes (CUDA defers
    // their destruction), and the caller's stream orders everything after.
    bool drain = true;
    explicit HostPipe(cudaStream_t st) {
        // the gathers feed the writer: their kernels go first when SMs free up
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        ok = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithPriority(&gth, cudaStreamNonBlocking, hi_prio) == cudaSuccess;
        if (ok) {
            cudaEvent_t e = ev();  // side streams start after the caller's prior work
            ok = e && cudaEventRecord(e, st) == cudaSuccess &&
                 cudaStreamWaitEvent(h2d, e, 0) == cudaSuccess &&
                 cudaStreamWaitEvent(d2h, e, 0) == cudaSuccess &&
                 cudaStreamWaitEvent(gth, e, 0) == cudaSuccess;
        }
    }
    // `s` waits for event e (if any).
    bool wait(cudaStream_t s, cudaEvent_t e) {
        return !e || cudaStreamWaitEvent(s, e, 0) == cudaSuccess;
    }
    // An event recorded on s now.
    cudaEvent_t record(cudaStream_t s) {
        cudaEvent_t e = ev();
        if (e && cudaEventRecord(e, s) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t ev() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        evs.push_back(e);
        return e;
    }
    // `to` waits for the work queued so far on `from`.
    bool order(cudaStream_t from, cudaStream_t to) {
        cudaEvent_t e = ev();
        return e && cudaEventRecord(e, from) == cudaSuccess &&
               cudaStreamWaitEvent(to, e, 0) == cudaSuccess;
    }
    // LEY_TRACE=1: timestamps of marked points on each stream, printed to
    // stderr (milliseconds from the first mark) when the sort ends.
    struct Mark {
        std::string what;
        cudaEvent_t e;
    };
    std::vector<Mark> marks;
    const bool trace = std::getenv("LEY_TRACE") != nullptr;
    void mark(cudaStream_t s, const char* what, long i = -1) {
        if (!trace) return;
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        std::string w = what;
        if (i >= 0) w += " " + std::to_string(i);
        w += s == h2d ? " [h2d]" : (s == d2h ? " [d2h]" : (s == gth ? " [gather]" : " [compute]"));
        marks.push_back({w, e});
    }
    ~HostPipe() {
        if (drain || !marks.empty()) {
            if (h2d) cudaStreamSynchronize(h2d);
            if (d2h) cudaStreamSynchronize(d2h);
            if (gth) cudaStreamSynchronize(gth);
        }
        if (!marks.empty()) {
            cudaEventSynchronize(marks.back().e);
            for (auto& m : marks) {
                float ms = 0.f;
                cudaEventSynchronize(m.e);
                cudaEventElapsedTime(&ms, marks[0].e, m.e);
                std::fprintf(stderr, "leysort trace %9.3f ms  %s\n", ms, m.what.c_str());
            }
            for (auto& m : marks) cudaEventDestroy(m.e);  // after the last use of marks[0]
        }
        for (auto e : evs) cudaEventDestroy(e);
        if (h2d) cudaStreamDestroy(h2d);
        if (d2h) cudaStreamDestroy(d2h);
        if (gth) cudaStreamDestroy(gth);
    }
};

// Streams sorted records to host memory: perm[j0, j1) gathered into
// kStaging rotating device staging buffers of q records on `st`, each copied
// to host_out + (j - j0) records on the writer stream as soon as it is full.
// Several buffers let the gathers run ahead of the copies, so a gather
// delayed behind other kernels does not stall the writer.
constexpr int kStaging = 4;
static ley_status stream_out(const SortArgs& a, const uint32_t* perm, ull j0, ull j1,
                             uint8_t* host_out, uint8_t* const stg[kStaging], ull q,
                             cudaStream_t st, HostPipe& hp, cudaEvent_t stg_free[kStaging],
                             int sms) {
    int b = 0;
    for (ull j = j0; j < j1; j += q, b = (b + 1) % kStaging) {
        const ull je = j + q < j1 ? j + q : j1;
        if (stg_free[b] && cudaStreamWaitEvent(st, stg_free[b], 0) != cudaSuccess) return LEY_ECUDA;
        ley_status s = stage_gather(a, perm, st, sms, j, je, stg[b]);
        if (s != LEY_OK) return s;
        if (!hp.order(st, hp.d2h)) return LEY_ECUDA;
        LEY_TRY(cudaMemcpyAsync(host_out + (j - j0) * a.rec, stg[b], (je - j) * a.rec,
                                cudaMemcpyDeviceToHost, hp.d2h));
        cudaEvent_t e = hp.ev();
        if (!e || cudaEventRecord(e, hp.d2h) != cudaSuccess) return LEY_ECUDA;
        stg_free[b] = e;
    }
    return LEY_OK;
}

// Copies host records [r0, r0+m) to dev, in chunks of whole tiles, and has
// `st` extract each chunk's tiles as soon as it has landed.
static ley_status stream_in_extract(const SortArgs& a, const uint8_t* host_in, uint8_t* dev,
                                    const Work& w, const KeySpec& ks, cudaStream_t st,
                                    HostPipe& hp, int sms) {
    const ull chunk = (ull)kPassTile * 1024;  // ~400 MB of 100-byte records
    for (ull c0 = 0; c0 < a.n; c0 += chunk) {
        const ull c1 = c0 + chunk < a.n ? c0 + chunk : a.n;
        LEY_TRY(cudaMemcpyAsync(dev + c0 * a.rec, host_in + c0 * a.rec, (c1 - c0) * a.rec,
                                cudaMemcpyHostToDevice, hp.h2d));
        if (!hp.order(hp.h2d, st)) return LEY_ECUDA;
        ley_status s = stage_extract_records(a, w, ks, st, sms, 0, (uint32_t)(c0 / kPassTile),
                                             ceil_div_u64(c1, kPassTile));
        if (s != LEY_OK) return s;
    }
    return LEY_OK;
}

static ull staging_records(ull n, uint32_t rec, ull budget) {
    ull q = (64ull << 20) / rec;  // 64 MB staging buffers
    if (budget) {  // all kStaging buffers together take at most budget / 8
        const ull cap = budget / (8ull * kStaging * rec);
        if (cap < q) q = cap;
    }
    if (q < 1024) q = 1024;
    return q < n ? q : n;
}

// Partially in-memory sort (Section 4.1's 20 GB case; the page-cache record
// scatter of Section 3.2): pinned host input and output, the input resident
// on the device, extraction overlapped with the copy in, and the sorted
// records streamed back through two staging buffers.  Blocks.  Returns
// LEY_ENOMEM without touching anything if it does not fit the budget.
// With block false the whole pipeline is only enqueued: every side stream
// joins `st` before the scratch is freed on it, so work queued on `st` later
// (or a synchronisation of `st`) comes after the sorted records are in out.
// Device bytes of the partially in-memory mode: the resident input, one
// internal sort's workspace (plus the window orders of a long key) and the
// copy-out staging buffers.
static size_t partial_need(ull n, uint32_t rec, uint32_t kb, ull budget, const Tuning& t) {
    const Layout L = make_layout(n, true, t.big);
    const size_t stg_bytes = align_up(staging_records(n, rec, budget) * rec, 256);
    return align_up(n * rec, 256) + L.total + kStaging * stg_bytes +
           (kb > kWindow ? long_key_extra(n) : 0);
}

static ley_status run_host_partial(const SortArgs& a, ull budget, cudaStream_t st,
                                   bool block = true) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    const ull bytes = a.n * a.rec;
    const Layout L = make_layout(a.n, true, a.tune.big);
    const bool long_key = a.kb > kWindow;
    const ull q = staging_records(a.n, a.rec, budget);
    const size_t stg_bytes = align_up(q * a.rec, 256);
    const size_t need = partial_need(a.n, a.rec, a.kb, budget, a.tune);
    if (budget && need > budget) return LEY_ENOMEM;
    void* dmem = nullptr;
    if (!scratch_alloc(ds, &dmem, need, st)) return LEY_ENOMEM;
    char* din = static_cast<char*>(dmem);
    char* ws = din + align_up(bytes, 256);
    uint8_t* stg[kStaging];
    for (int i = 0; i < kStaging; i++) stg[i] = reinterpret_cast<uint8_t*>(ws + L.total + i * stg_bytes);
    ley_status s = LEY_OK;
    {
        HostPipe hp(st);
        if (!hp.ok) s = LEY_ECUDA;
        hp.drain = block;
        SortArgs d = a;
        d.in = reinterpret_cast<const uint8_t*>(din);
        Work w = make_work(ws, L, a.n, ds->err);
        const KeySpec ks = record_keyspec(a.kb, a.tune);
        hp.mark(hp.h2d, "in begin");
        const uint32_t* order = w.perm;
        if (long_key) {
            // the whole input first, then one sort per 12-byte key window
            if (s == LEY_OK && cudaMemcpyAsync(din, a.in, bytes, cudaMemcpyHostToDevice, hp.h2d) !=
                                   cudaSuccess)
                s = LEY_ECUDA;
            if (s == LEY_OK && !hp.order(hp.h2d, st)) s = LEY_ECUDA;
            hp.mark(hp.h2d, "in end");
            uint32_t* ord[2] = {reinterpret_cast<uint32_t*>(ws + L.total + kStaging * stg_bytes),
                                reinterpret_cast<uint32_t*>(ws + L.total + kStaging * stg_bytes +
                                                            long_key_extra(a.n) / 2)};
            if (s == LEY_OK) s = enqueue_long_key_order(d, w, L, ord, st, ds->sms, &order);
        } else {
            if (s == LEY_OK) s = stage_prepare(w, L, st, a.n, 0);
            if (s == LEY_OK) s = stream_in_extract(d, a.in, reinterpret_cast<uint8_t*>(din), w, ks, st, hp, ds->sms);
            hp.mark(hp.h2d, "in end");
            hp.mark(st, "extracted");
            if (s == LEY_OK) s = stage_levels_finish(d, w, ks, st, ds->sms);
        }
        hp.mark(st, "sorted");
        cudaEvent_t stg_free[kStaging] = {};
        if (s == LEY_OK) s = stream_out(d, order, 0, a.n, a.out, stg, q, st, hp, stg_free, ds->sms);
        hp.mark(st, "gathered");
        hp.mark(hp.d2h, "out end");
        if (!hp.order(hp.d2h, st) && s == LEY_OK) s = LEY_ECUDA;
        if (!hp.order(hp.gth, st) && s == LEY_OK) s = LEY_ECUDA;
        if (!hp.order(hp.h2d, st) && s == LEY_OK) s = LEY_ECUDA;
        cudaFreeAsync(dmem, st);
        if (block && cudaStreamSynchronize(st) != cudaSuccess && s == LEY_OK) s = LEY_ECUDA;
    }
    return s;
}

// Pinned host scratch for the sorted runs of the external sort, kept across
// calls (pinning tens of GB takes seconds) and grown on demand.
static std::mutex g_host_scratch_mu;
static uint8_t* g_host_scratch = nullptr;
static size_t g_host_scratch_bytes = 0;

static uint8_t* host_scratch(size_t bytes) {
    if (bytes <= g_host_scratch_bytes) return g_host_scratch;
    if (g_host_scratch) cudaFreeHost(g_host_scratch);
    g_host_scratch = nullptr;
    g_host_scratch_bytes = 0;
    void* p = nullptr;
    // mapped: the partition planning reads the runs from the device
    if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_host_scratch = static_cast<uint8_t*>(p);
    g_host_scratch_bytes = bytes;
    return g_host_scratch;
}

// A sorted run in host memory.
struct HostRun {
    const uint8_t* base;
    ull len;
};

// Elements of run i ordered before the element at position ppos of run prun
// (key K there) in the order (key, run, position): the k-way co-rank used to
// cut the merge into independent partitions (Section 3.2's partitioning).
static ull corank_split(const std::vector<HostRun>& runs, size_t i, const uint8_t* K, size_t prun,
                        ull ppos, uint32_t rec, uint32_t kb) {
    if (i == prun) return ppos;
    const bool upper = i < prun;  // equal keys of lower runs come first
    ull lo = 0, hi = runs[i].len;
    while (lo < hi) {
        const ull mid = (lo + hi) / 2;
        const int c = std::memcmp(runs[i].base + mid * rec, K, kb);
        if (c < 0 || (upper && c == 0)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The partition cuts from candidates in merged order (ranks increasing, every
// two consecutive at most cap / 4 apart): from the current cut, the last
// candidate at most 3/4 cap further becomes the next cut, until the rest fits
// one partition.  cut(ci) gives candidate ci's co-rank in every run.
template <class CutOf>
static std::vector<std::vector<ull>> select_cuts(const std::vector<ull>& ranks,
                                                 const std::vector<ull>& lens, ull n, ull cap,
                                                 CutOf cut) {
    std::vector<std::vector<ull>> cuts;
    cuts.push_back(std::vector<ull>(lens.size(), 0));
    ull start = 0;
    const ull target = cap * 3 / 4 > 0 ? cap * 3 / 4 : 1;
    size_t ci = 0;
    while (n - start > cap) {
        long best = -1;
        while (ci < ranks.size() && ranks[ci] <= start + target) {
            if (ranks[ci] > start) best = (long)ci;
            ci++;
        }
        if (best < 0) break;  // cannot happen: consecutive ranks differ by <= cap/4
        cuts.push_back(cut((size_t)best));
        start = ranks[best];
    }
    cuts.push_back(lens);
    return cuts;
}

// Merge partitions: split vectors (one position per run) at increasing global
// ranks 0 = r_0 < r_1 < ... < r_P = n, each partition at most cap records.
static std::vector<std::vector<ull>> plan_partitions(const std::vector<HostRun>& runs, ull n,
                                                     ull cap, uint32_t rec, uint32_t kb) {
    const size_t k = runs.size();
    const ull step = cap / (4 * k) > 0 ? cap / (4 * k) : 1;
    struct Cand {
        size_t run;
        ull pos;
        ull rank;
    };
    std::vector<Cand> cands;
    for (size_t i = 0; i < k; i++)
        for (ull p = step - 1; p < runs[i].len; p += step) cands.push_back({i, p, 0});
    std::sort(cands.begin(), cands.end(), [&](const Cand& x, const Cand& y) {
        const int c = std::memcmp(runs[x.run].base + x.pos * rec, runs[y.run].base + y.pos * rec, kb);
        if (c != 0) return c < 0;
        if (x.run != y.run) return x.run < y.run;
        return x.pos < y.pos;
    });
    // Each candidate's rank costs k binary searches over host memory, bound
    // by memory latency: spread the candidates over the host's cores.
    auto rank_range = [&](size_t c0, size_t c1) {
        for (size_t ci = c0; ci < c1; ci++) {
            Cand& c = cands[ci];
            ull r = 0;
            for (size_t i = 0; i < k; i++)
                r += corank_split(runs, i, runs[c.run].base + c.pos * rec, c.run, c.pos, rec, kb);
            c.rank = r;
        }
    };
    const size_t nthr = std::max<size_t>(1, std::min<size_t>(16, std::thread::hardware_concurrency()));
    if (nthr == 1 || cands.size() < 64) {
        rank_range(0, cands.size());
    } else {
        std::vector<std::thread> pool;
        const size_t per = (cands.size() + nthr - 1) / nthr;
        for (size_t t = 0; t < nthr; t++) {
            const size_t c0 = t * per, c1 = std::min(cands.size(), c0 + per);
            if (c0 < c1) pool.emplace_back(rank_range, c0, c1);
        }
        for (auto& th : pool) th.join();
    }
    std::vector<ull> ranks(cands.size()), lens(k);
    for (size_t ci = 0; ci < cands.size(); ci++) ranks[ci] = cands[ci].rank;
    for (size_t i = 0; i < k; i++) lens[i] = runs[i].len;
    return select_cuts(ranks, lens, n, cap, [&](size_t ci) {
        const Cand& c = cands[ci];
        std::vector<ull> cut(k);
        for (size_t i = 0; i < k; i++)
            cut[i] = corank_split(runs, i, runs[c.run].base + c.pos * rec, c.run, c.pos, rec, kb);
        return cut;
    });
}

// Merge of the k sorted runs whose records lie back to back at dev_runs (run r
// at [off[r], off[r+1]) records, off on the host): tuples, then the k-way
// merge path in one pass (pairwise merge-path rounds first while more than
// kKwayMaxRuns runs remain), the permutation in w.perm.  Queued on st.
static ley_status stage_merge(const SortArgs& a, const uint8_t* dev_runs, const ull* off_host,
                              ull* off_dev, uint32_t k, const Work& w, const Layout& L,
                              cudaStream_t st, int sms) {
    SortArgs m = a;
    m.in = dev_runs;
    m.n = off_host[k];
    const KeySpec ks = record_keyspec(a.kb, a.tune);
    ley_status s = stage_prepare(w, L, st, m.n, 0);
    if (s != LEY_OK) return s;
    s = stage_extract_records(m, w, ks, st, sms, 0, 0, ceil_div_u64(m.n, kPassTile));
    if (s != LEY_OK) return s;
    LEY_TRY(launch("merge_offsets", st, [&] {
        return launch_set_offsets(st, off_dev, off_host, k + 1);
    }));
    std::vector<ull> off(off_host, off_host + k + 1);  // the runs of the next step, on the host
    int cur = 0;
    uint32_t runs = k;
    for (; runs > (uint32_t)kKwayMaxRuns; runs = (runs + 1) / 2) {
        LEY_TRY(launch("merge", st, [&] {
            return launch_merge_round(st, sms * 8, w.tup[cur], w.tup[cur ^ 1], off_dev, runs,
                                      ks.lo_mask);
        }));
        cur ^= 1;
        // the merged pairs are the runs of the next round
        LEY_TRY(launch("merge_offsets", st, [&] { return launch_halve_offsets(st, off_dev, runs); }));
        const uint32_t np = (runs + 1) / 2;
        for (uint32_t i = 1; i <= np; i++) off[i] = off[std::min<uint32_t>(2 * i, runs)];
        off.resize(np + 1);
    }
    // the sample split table goes to the other tuple buffer
    const uint32_t step = kway_sample_step(runs);
    ull S = 0;
    for (uint32_t i = 0; i < runs; i++) S += (off[i + 1] - off[i] + step - 1) / step;
    const ull rows_cap = (ull)(L.tup[1] - L.tup[0]) / (4ull * runs);  // u32 rows of `runs`
    if (S + 1 > rows_cap) {
        // a merge far smaller than its runs' count (a few records per run):
        // pairwise rounds to the end
        for (; runs > 1; runs = (runs + 1) / 2) {
            LEY_TRY(launch("merge", st, [&] {
                return launch_merge_round(st, sms * 8, w.tup[cur], w.tup[cur ^ 1], off_dev, runs,
                                          ks.lo_mask);
            }));
            cur ^= 1;
            if (runs > 2)
                LEY_TRY(launch("merge_offsets", st, [&] { return launch_halve_offsets(st, off_dev, runs); }));
        }
        LEY_TRY(launch("tuple_index", st, [&] {
            return launch_tuple_index(st, sms * 4, w.tup[cur], w.perm, m.n);
        }));
        return LEY_OK;
    }
    uint32_t* table = reinterpret_cast<uint32_t*>(w.tup[cur ^ 1]);
    LEY_TRY(launch("kmerge", st, [&] {
        return launch_kmerge(st, sms, w.tup[cur], off_dev, runs, (uint32_t)S, ks.lo_mask, table,
                             rows_cap, w.perm, m.n, w.err);
    }));
    return LEY_OK;
}

// External sort (Section 3.2, Figure 1).  Run formation: runs of r_len
// records are copied in on the reader stream (extraction following chunk by
// chunk), sorted on the compute stream, and gathered into staging buffers on
// the gather stream that the writer stream copies into pinned host scratch.
// Merge: the output is cut into partitions by k-way co-rank; each partition's
// slices of every run are copied in, merged by merge path, gathered and
// streamed to `out`.  kExtBufs record buffers and workspaces rotate, so that
// while one run (or partition) streams out, the next is sorted and the one
// after it is already being copied in; runs are about n / kExtRuns records,
// so that filling and draining this pipeline (the first copy in, the last
// copy out) costs little next to the copies themselves.
constexpr ull kExtRuns = 32;
constexpr int kExtBufs = 3;
constexpr ull kExtMinRun = 4ull << 20;
constexpr uint32_t kMaxRuns = 128;  // merge fan-in (the offsets travel in kernel parameters)

// The external mode's device-memory plan under a budget: runs of r_len
// records (whole tiles, about n / kExtRuns, at most what kExtBufs record
// buffers and workspaces allow beside the staging buffers), k runs, and the
// device bytes of the whole pipeline.  LEY_ENOMEM when nothing fits.
struct ExtPlan {
    ull q = 0;          // records per staging buffer
    ull r_len = 0;      // records per run (the largest merge partition too)
    uint32_t k = 0;     // runs
    uint32_t resident = 0;  // the last `resident` runs stay on the device, sorted
    ull step = 0;       // partition planning: a candidate every `step` records of a run
    uint32_t ncand = 0; // candidates in all runs
    size_t in_bytes = 0, ws_len = 0, stg_bytes = 0, plan_bytes = 0, total = 0;
    size_t host_bytes = 0;  // pinned host scratch for the runs that leave the device
};

// Runs that stay on the device: as many as fit the budget beside the
// pipeline, at most all but one (LEY_EXTERNAL_RESIDENT=<m> caps them).  Keys
// longer than 12 bytes keep every run on the host (their cuts are planned
// on the host).
static uint32_t resident_cap() {
    const char* v = std::getenv("LEY_EXTERNAL_RESIDENT");
    return v ? (uint32_t)std::strtoul(v, nullptr, 10) : 0xFFFFFFFFu;
}

static ley_status external_plan(ull n, uint32_t rec, uint32_t kb, ull budget, const Tuning& t,
                                ExtPlan* p) {
    ExtPlan e;
    e.q = staging_records(n, rec, budget);
    e.stg_bytes = align_up(e.q * rec, 256);
    const size_t fixed = kStaging * e.stg_bytes + 64 * 1024;
    if (budget <= fixed) return LEY_ENOMEM;
    // Keys longer than a tuple's 12 bytes: each run, and each merge
    // partition, is sorted window by window (its workspace grows by the two
    // order arrays); the partitions are cut by the same exact co-rank on the
    // whole key, so sorting a partition's slices stably -- ties in slice
    // order, which is (run, position) -- gives its merge.
    const bool long_key = kb > kWindow;
    auto ws_bytes = [&](ull r) {
        return make_layout(r, true, t.big).total + (long_key ? long_key_extra(r) : 0);
    };
    // the partition candidates of runs of r records: every step-th record of
    // every run (as the host planner takes them); the device planner's
    // scratch holds their co-ranks, their ranks and the run table
    auto step_of = [&](ull r, uint32_t k) { return r / (4ull * k) > 0 ? r / (4ull * k) : 1ull; };
    auto ncand_of = [&](ull r, uint32_t k, ull step) {
        ull nc = 0;
        for (uint32_t i = 0; i < k; i++) nc += std::min(r, n - (ull)i * r) / step;
        return nc;
    };
    auto plan_bytes_of = [&](ull r) -> size_t {
        if (long_key || r == 0) return 0;
        const uint32_t k = (uint32_t)std::min<ull>((n + r - 1) / r, 1ull << 20);
        const ull nc = ncand_of(r, k, step_of(r, k));
        return align_up(nc * k * sizeof(uint32_t), 256) + align_up(nc * sizeof(ull), 256) +
               align_up((k + 1) * sizeof(ull), 256) + align_up(k * sizeof(PlanRun), 256);
    };
    // largest run (whole tiles) whose record buffers, workspaces and planner fit
    auto need = [&](ull r) {
        return kExtBufs * (align_up(r * rec, 256) + ws_bytes(r)) + fixed + plan_bytes_of(r);
    };
    ull lo = 0, hi = n / kPassTile + 1;
    while (lo < hi) {
        const ull mid = (lo + hi + 1) / 2;
        if (need(mid * kPassTile) <= budget) lo = mid;
        else hi = mid - 1;
    }
    const ull r_max = lo * kPassTile;
    if (r_max == 0) return LEY_ENOMEM;
    e.r_len = ceil_div_u64(ceil_div_u64(n, kExtRuns), kPassTile) * kPassTile;
    if (e.r_len < kExtMinRun) e.r_len = kExtMinRun;
    if (e.r_len > r_max) e.r_len = r_max;
    e.k = (uint32_t)((n + e.r_len - 1) / e.r_len);
    if (e.k > kMaxRuns) return LEY_ENOMEM;  // budget too small for the merge fan-in
    e.in_bytes = align_up(e.r_len * rec, 256);
    e.ws_len = ws_bytes(e.r_len);
    e.step = step_of(e.r_len, e.k);
    e.ncand = (uint32_t)ncand_of(e.r_len, e.k, e.step);
    e.plan_bytes = plan_bytes_of(e.r_len);
    const size_t base = kExtBufs * (e.in_bytes + e.ws_len) + kStaging * e.stg_bytes + 8 * 1024 +
                        e.plan_bytes;
    if (base > budget) return LEY_ENOMEM;
    if (!long_key && e.k > 1) {
        const ull fit = (budget - base) / e.in_bytes;
        e.resident = (uint32_t)std::min<ull>(std::min<ull>(fit, e.k - 1), resident_cap());
    }
    e.total = base + e.resident * e.in_bytes;
    // the first k - resident runs
    e.host_bytes = (size_t)std::min<ull>(n, (ull)(e.k - e.resident) * e.r_len) * rec;
    *p = e;
    return LEY_OK;
}

// The partition cuts of the external merge planned on the device (keys of at
// most 12 bytes): the candidates' co-ranks in every run (k_corank, runs on
// the device or in mapped host memory), then the cuts chosen on the host
// from their ranks.  Queued on st after everything before it; blocks.
static ley_status plan_partitions_device(const std::vector<PlanRun>& runs, const ExtPlan& plan,
                                         ull n, uint32_t rec, uint32_t kb, char* scratch,
                                         cudaStream_t st, int sms, uint32_t* err,
                                         std::vector<std::vector<ull>>* cuts) {
    const uint32_t k = (uint32_t)runs.size();
    const uint32_t nc = plan.ncand;
    uint32_t* split = reinterpret_cast<uint32_t*>(scratch);
    char* c1 = scratch + align_up((size_t)nc * k * sizeof(uint32_t), 256);
    ull* rank = reinterpret_cast<ull*>(c1);
    char* c2 = c1 + align_up((size_t)nc * sizeof(ull), 256);
    ull* cbase_dev = reinterpret_cast<ull*>(c2);
    PlanRun* runs_dev = reinterpret_cast<PlanRun*>(c2 + align_up((k + 1) * sizeof(ull), 256));
    std::vector<ull> cbase(k + 1, 0), lens(k);
    for (uint32_t i = 0; i < k; i++) {
        lens[i] = runs[i].len;
        cbase[i + 1] = cbase[i] + runs[i].len / plan.step;
    }
    if (cbase[k] != nc) return LEY_EINVAL;  // the plan counted the same candidates
    LEY_TRY(launch("plan_upload", st, [&] {
        return launch_upload(st, cbase_dev, cbase.data(), (k + 1) * sizeof(ull));
    }));
    LEY_TRY(launch("plan_upload", st, [&] {
        return launch_upload(st, runs_dev, runs.data(), k * sizeof(PlanRun));
    }));
    LEY_TRY(launch("corank", st, [&] {
        return launch_corank(st, sms, runs_dev, k, rec, kb, cbase_dev, plan.step, nc, split, rank,
                             err);
    }));
    std::vector<uint32_t> split_h((size_t)nc * k);
    std::vector<ull> rank_h(nc);
    if (nc) {
        LEY_TRY(cudaMemcpyAsync(split_h.data(), split, split_h.size() * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, st));
        LEY_TRY(cudaMemcpyAsync(rank_h.data(), rank, nc * sizeof(ull), cudaMemcpyDeviceToHost, st));
    }
    LEY_TRY(cudaStreamSynchronize(st));
    // candidates in merged order (their ranks are distinct: (key, run, position) is a total order)
    std::vector<uint32_t> order(nc);
    for (uint32_t c = 0; c < nc; c++) order[c] = c;
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return rank_h[x] < rank_h[y]; });
    std::vector<ull> ranks(nc);
    for (uint32_t c = 0; c < nc; c++) ranks[c] = rank_h[order[c]];
    *cuts = select_cuts(ranks, lens, n, plan.r_len, [&](size_t ci) {
        std::vector<ull> cut(k);
        for (uint32_t j = 0; j < k; j++) cut[j] = split_h[(size_t)order[ci] * k + j];
        return cut;
    });
    return LEY_OK;
}

static ley_status run_host_external(const SortArgs& a, ull budget, cudaStream_t st) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    ExtPlan plan;
    const ley_status ps = external_plan(a.n, a.rec, a.kb, budget, a.tune, &plan);
    if (ps != LEY_OK) return ps;
    const ull q = plan.q, r_len = plan.r_len;
    const uint32_t k = plan.k, nres = plan.resident, nhost = k - nres;
    const bool long_key = a.kb > kWindow;
    const Layout L = make_layout(r_len, true, a.tune.big);
    const size_t stg_bytes = plan.stg_bytes, in_bytes = plan.in_bytes, ws_len = plan.ws_len;
    const size_t total = plan.total;
    const bool dbg = std::getenv("LEY_DEBUG") != nullptr;
    if (dbg)
        std::fprintf(stderr, "leysort: external n=%llu runs=%u of %llu records (%u stay on the "
                     "device), staging %llu, device bytes %zu of budget %llu\n", a.n, k, r_len,
                     nres, q, total, budget);
    // One external sort at a time per process: they share the host scratch.
    std::lock_guard<std::mutex> scratch_lock(g_host_scratch_mu);
    uint8_t* hs = host_scratch(plan.host_bytes);
    if (!hs) return LEY_ENOMEM;
    void* hs_dev = nullptr;  // the runs on the host as the device reads them (planning)
    if (!long_key && (cudaHostGetDevicePointer(&hs_dev, hs, 0) != cudaSuccess || !hs_dev)) {
        cudaGetLastError();
        return LEY_ECUDA;
    }
    void* dmem = nullptr;
    if (!scratch_alloc(ds, &dmem, total, st)) return LEY_ENOMEM;
    char* base = static_cast<char*>(dmem);
    uint8_t* dbuf[kExtBufs];
    char* ws[kExtBufs];
    for (int i = 0; i < kExtBufs; i++) {
        dbuf[i] = reinterpret_cast<uint8_t*>(base + i * in_bytes);
        ws[i] = base + kExtBufs * in_bytes + i * ws_len;
    }
    // the two order arrays of a long-key sort of up to r_len records in ws[b]
    auto long_ord = [&](int b, uint32_t** ord) {
        ord[0] = reinterpret_cast<uint32_t*>(ws[b] + L.total);
        ord[1] = reinterpret_cast<uint32_t*>(ws[b] + L.total + long_key_extra(r_len) / 2);
    };
    char* tail = base + kExtBufs * (in_bytes + ws_len);
    uint8_t* stg[kStaging];
    for (int i = 0; i < kStaging; i++) stg[i] = reinterpret_cast<uint8_t*>(tail + i * stg_bytes);
    ull* off_dev = reinterpret_cast<ull*>(tail + kStaging * stg_bytes);
    char* plan_scratch = tail + kStaging * stg_bytes + 8 * 1024;
    uint8_t* const res0 = reinterpret_cast<uint8_t*>(plan_scratch + plan.plan_bytes);
    auto resident = [&](uint32_t r) { return res0 + (size_t)(r - nhost) * in_bytes; };
    ley_status s = LEY_OK;
    {
        HostPipe hp(st);
        if (!hp.ok) s = LEY_ECUDA;
        const KeySpec ks = record_keyspec(a.kb, a.tune);
        cudaEvent_t stg_free[kStaging] = {};
        // buffer b and workspace b are free again once the gathers that read
        // them (kExtBufs runs or partitions back) are done
        cudaEvent_t buf_free[kExtBufs] = {};
        // --- run formation: the first nhost runs go to the host scratch, the
        // last nres are gathered into device buffers of their own
        std::vector<HostRun> runs;
        std::vector<PlanRun> pruns;
        for (uint32_t r = 0; r < k && s == LEY_OK; r++) {
            const ull r0 = (ull)r * r_len;
            const ull rn = a.n - r0 < r_len ? a.n - r0 : r_len;
            const int b = (int)(r % kExtBufs);
            if (!hp.wait(hp.h2d, buf_free[b]) || !hp.wait(st, buf_free[b])) s = LEY_ECUDA;
            SortArgs ra = a;
            ra.in = dbuf[b];
            ra.n = rn;
            Work w = make_work(ws[b], L, rn, ds->err);
            hp.mark(hp.h2d, "run in begin", r);
            const uint32_t* order = w.perm;
            if (long_key) {  // the whole run first, then one sort per 12-byte window
                if (s == LEY_OK && cudaMemcpyAsync(dbuf[b], a.in + r0 * a.rec, rn * a.rec,
                                                   cudaMemcpyHostToDevice, hp.h2d) != cudaSuccess)
                    s = LEY_ECUDA;
                if (s == LEY_OK && !hp.order(hp.h2d, st)) s = LEY_ECUDA;
                hp.mark(hp.h2d, "run in end", r);
                uint32_t* ord[2];
                long_ord(b, ord);
                if (s == LEY_OK) s = enqueue_long_key_order(ra, w, L, ord, st, ds->sms, &order);
            } else {
                if (s == LEY_OK) s = stage_prepare(w, L, st, rn, 0);
                if (s == LEY_OK)
                    s = stream_in_extract(ra, a.in + r0 * a.rec, dbuf[b], w, ks, st, hp, ds->sms);
                hp.mark(hp.h2d, "run in end", r);
                if (s == LEY_OK) s = stage_levels_finish(ra, w, ks, st, ds->sms);
            }
            hp.mark(st, "run sorted", r);
            if (s == LEY_OK && !hp.order(st, hp.gth)) s = LEY_ECUDA;
            if (r < nhost) {
                if (s == LEY_OK) s = stream_out(ra, order, 0, rn, hs + r0 * a.rec, stg, q, hp.gth, hp, stg_free, ds->sms);
                runs.push_back({hs + r0 * a.rec, rn});
                pruns.push_back({static_cast<const uint8_t*>(hs_dev) + r0 * a.rec, rn});
            } else {
                if (s == LEY_OK) s = stage_gather(ra, order, hp.gth, ds->sms, 0, rn, resident(r));
                runs.push_back({nullptr, rn});
                pruns.push_back({resident(r), rn});
            }
            hp.mark(hp.gth, "run gathered", r);
            hp.mark(hp.d2h, "run out end", r);
            if (s == LEY_OK && !(buf_free[b] = hp.record(hp.gth))) s = LEY_ECUDA;
        }
        // --- merge: the runs must be complete before they are cut (in host
        // memory, and in their device buffers)
        std::vector<std::vector<ull>> cuts;
        const auto t_plan = std::chrono::steady_clock::now();
        if (long_key) {
            if (s == LEY_OK && cudaStreamSynchronize(hp.d2h) != cudaSuccess) s = LEY_ECUDA;
            if (s == LEY_OK) cuts = plan_partitions(runs, a.n, r_len, a.rec, a.kb);
        } else {
            if (s == LEY_OK && (!hp.order(hp.d2h, st) || !hp.order(hp.gth, st))) s = LEY_ECUDA;
            if (s == LEY_OK)
                s = plan_partitions_device(pruns, plan, a.n, a.rec, a.kb, plan_scratch, st,
                                           ds->sms, ds->err, &cuts);
        }
        hp.mark(st, "partitions planned");
        if (hp.trace)
            std::fprintf(stderr, "leysort trace plan_partitions %.3f ms\n",
                         std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count());
        if (dbg) std::fprintf(stderr, "leysort: runs formed (status %d), %zu merge partitions\n",
                              (int)s, cuts.empty() ? (size_t)0 : cuts.size() - 1);
        std::vector<ull> off(k + 1);
        ull out_pos = 0;
        for (size_t p = 0; p + 1 < cuts.size() && s == LEY_OK; p++) {
            const int b = (int)(p % kExtBufs);
            off[0] = 0;
            for (uint32_t i = 0; i < k; i++) off[i + 1] = off[i] + (cuts[p + 1][i] - cuts[p][i]);
            const ull m = off[k];
            if (m > r_len) {
                s = LEY_ENOMEM;
                break;
            }
            if (m == 0) continue;
            if (!hp.wait(hp.h2d, buf_free[b]) || !hp.wait(st, buf_free[b])) s = LEY_ECUDA;
            hp.mark(hp.h2d, "part in begin", (long)p);
            for (uint32_t i = 0; i < k && s == LEY_OK; i++) {
                const ull len = cuts[p + 1][i] - cuts[p][i];
                if (!len) continue;
                // slices of the host runs over the link, of the resident runs on the device
                const bool host = i < nhost;
                if (cudaMemcpyAsync(dbuf[b] + off[i] * a.rec,
                                    (host ? runs[i].base : resident(i)) + cuts[p][i] * a.rec,
                                    len * a.rec,
                                    host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    host ? hp.h2d : st) != cudaSuccess)
                    s = LEY_ECUDA;
            }
            hp.mark(hp.h2d, "part in end", (long)p);
            if (s == LEY_OK && !hp.order(hp.h2d, st)) s = LEY_ECUDA;
            Work w = make_work(ws[b], L, m, ds->err);
            SortArgs ma = a;
            ma.in = dbuf[b];
            ma.n = m;
            const uint32_t* order = w.perm;
            if (long_key) {  // the slices in (run, position) order, sorted stably
                uint32_t* ord[2];
                long_ord(b, ord);
                if (s == LEY_OK) s = enqueue_long_key_order(ma, w, L, ord, st, ds->sms, &order);
            } else {
                if (s == LEY_OK) s = stage_merge(ma, dbuf[b], off.data(), off_dev, k, w, L, st, ds->sms);
            }
            hp.mark(st, "part merged", (long)p);
            if (s == LEY_OK && !hp.order(st, hp.gth)) s = LEY_ECUDA;
            if (s == LEY_OK) s = stream_out(ma, order, 0, m, a.out + out_pos * a.rec, stg, q, hp.gth, hp, stg_free, ds->sms);
            hp.mark(hp.gth, "part gathered", (long)p);
            hp.mark(hp.d2h, "part out end", (long)p);
            if (s == LEY_OK && !(buf_free[b] = hp.record(hp.gth))) s = LEY_ECUDA;
            out_pos += m;
        }
        if (!hp.order(hp.d2h, st) && s == LEY_OK) s = LEY_ECUDA;
        if (!hp.order(hp.gth, st) && s == LEY_OK) s = LEY_ECUDA;
        cudaFreeAsync(dmem, st);
        if (cudaStreamSynchronize(st) != cudaSuccess && s == LEY_OK) s = LEY_ECUDA;
    }
    return s;
}

// Keys-only external sort: only the (key, pointer) tuples live on the device.
// The input streams in once (chunks through a two-buffer ring, each chunk's
// tuples extracted as it lands), the tuples are sorted on the device, and
// the records are gathered by the final order straight from the pinned host
// input (the GPU reading host memory over the host link) into staging
// buffers that stream out.  The link carries n*100 bytes in for the keys,
// n*100 bytes of record reads and n*100 bytes out -- no run scratch on the
// host -- and the device holds 36 bytes per record, so it serves inputs up to
// about budget / 36 records.  Returns LEY_ENOMEM (touching nothing) when the
// tuples do not fit or the input is not mapped for the device.
static ley_status run_host_keys_only(const SortArgs& a, ull budget, cudaStream_t st) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    if (a.kb > kWindow) return LEY_ENOMEM;
    void* in_dev = nullptr;
    if (cudaHostGetDevicePointer(&in_dev, const_cast<uint8_t*>(a.in), 0) != cudaSuccess ||
        !in_dev) {
        cudaGetLastError();
        return LEY_ENOMEM;
    }
    const Layout L = make_layout(a.n, true, a.tune.big);
    // chunks of n/8 records (whole tiles), between 64 Ki and 4 Mi records
    ull chunk = (ull)ceil_div_u64(a.n / 8 + 1, kPassTile) * kPassTile;
    chunk = std::max<ull>(chunk, 16ull * kPassTile);
    chunk = std::min<ull>(chunk, 1024ull * kPassTile);
    const size_t chunk_bytes = align_up(chunk * a.rec, 256);
    const ull q = staging_records(a.n, a.rec, budget);
    const size_t stg_bytes = align_up(q * a.rec, 256);
    const size_t need = L.total + 2 * chunk_bytes + kStaging * stg_bytes;
    if (budget && need > budget) return LEY_ENOMEM;
    void* dmem = nullptr;
    if (!scratch_alloc(ds, &dmem, need, st)) return LEY_ENOMEM;
    char* ws = static_cast<char*>(dmem);
    uint8_t* ring[2] = {reinterpret_cast<uint8_t*>(ws + L.total),
                        reinterpret_cast<uint8_t*>(ws + L.total + chunk_bytes)};
    uint8_t* stg[kStaging];
    for (int i = 0; i < kStaging; i++)
        stg[i] = reinterpret_cast<uint8_t*>(ws + L.total + 2 * chunk_bytes + i * stg_bytes);
    ley_status s = LEY_OK;
    {
        HostPipe hp(st);
        if (!hp.ok) s = LEY_ECUDA;
        Work w = make_work(ws, L, a.n, ds->err);
        const KeySpec ks = record_keyspec(a.kb, a.tune);
        if (s == LEY_OK) s = stage_prepare(w, L, st, a.n, 0);
        hp.mark(hp.h2d, "in begin");
        cudaEvent_t ring_free[2] = {nullptr, nullptr};
        for (ull c0 = 0, ci = 0; c0 < a.n && s == LEY_OK; c0 += chunk, ci++) {
            const ull c1 = std::min(c0 + chunk, a.n);
            const int b = (int)(ci & 1);
            if (!hp.wait(hp.h2d, ring_free[b])) s = LEY_ECUDA;
            if (s == LEY_OK && cudaMemcpyAsync(ring[b], a.in + c0 * a.rec, (c1 - c0) * a.rec,
                                               cudaMemcpyHostToDevice, hp.h2d) != cudaSuccess)
                s = LEY_ECUDA;
            if (s == LEY_OK && !hp.order(hp.h2d, st)) s = LEY_ECUDA;
            // record i of the input sits at ring[b] + (i - c0) * rec
            SortArgs ca = a;
            ca.in = ring[b] - c0 * a.rec;
            // (the difference mask against record 0, read from the host input)
            if (s == LEY_OK)
                s = stage_extract_records(ca, w, ks, st, ds->sms, 0, (uint32_t)(c0 / kPassTile),
                                          ceil_div_u64(c1, kPassTile),
                                          static_cast<const uint8_t*>(in_dev));
            if (s == LEY_OK && !(ring_free[b] = hp.record(st))) s = LEY_ECUDA;
        }
        hp.mark(hp.h2d, "in end");
        if (s == LEY_OK) s = stage_levels_finish(a, w, ks, st, ds->sms);
        hp.mark(st, "sorted");
        SortArgs ga = a;
        ga.in = static_cast<const uint8_t*>(in_dev);
        ga.in_host = true;
        cudaEvent_t stg_free[kStaging] = {};
        if (s == LEY_OK) s = stream_out(ga, w.perm, 0, a.n, a.out, stg, q, st, hp, stg_free, ds->sms);
        hp.mark(st, "gathered");
        hp.mark(hp.d2h, "out end");
        if (!hp.order(hp.d2h, st) && s == LEY_OK) s = LEY_ECUDA;
        cudaFreeAsync(dmem, st);
        if (cudaStreamSynchronize(st) != cudaSuccess && s == LEY_OK) s = LEY_ECUDA;
    }
    return s;
}

// Which external design to use: the run formation + k-way merge (default),
// or with LEY_EXTERNAL=keys the keys-only design whenever its tuples fit the
// budget.  Measured on GB300 at 4e8 records: the keys-only design's gather
// reads host memory at about 1 GB/s (random 100-byte loads over the host
// link, latency-bound), 41 s against 0.55 s for the merge design.
static int external_design() {
    const char* v = std::getenv("LEY_EXTERNAL");
    if (v && std::strcmp(v, "keys") == 0) return 1;
    return 0;
}

// Host-memory sort: partially in-memory when it fits the budget, else external.
static ley_status run_host_sort(const SortArgs& a, ull budget, cudaStream_t st,
                                bool block = true) {
    ley_status s = run_host_partial(a, budget, st, block);
    if (s != LEY_ENOMEM || !budget) return s;
    if (external_design() == 1) {
        s = run_host_keys_only(a, budget, st);
        if (s != LEY_ENOMEM) return s;
    }
    return run_host_external(a, budget, st);
}

// ------------------------------------------------------------- validation

enum MemKind { MK_DEVICE, MK_HOST_PINNED, MK_OTHER };

static MemKind mem_kind(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return MK_OTHER;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return MK_DEVICE;
    if (at.type == cudaMemoryTypeHost) return MK_HOST_PINNED;
    return MK_OTHER;
}

static bool overlaps(const void* a, ull na, const void* b, ull nb) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace ley

namespace ley {
// Argument checks of one request of a batch (also used by the sort server
// at submission).
ley_status check_records_request(const ley_records_request& q, uint32_t rec_bytes,
                                 uint32_t key_bytes) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096 || q.n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (q.n == 0) return LEY_OK;
    if (!q.in || !q.out) return LEY_EINVAL;
    const ull bytes = q.n * rec_bytes;
    if (overlaps(q.in, bytes, q.out, bytes)) return LEY_EINVAL;
    if (!aligned16(q.in) || !aligned16(q.out)) return LEY_EINVAL;
    if (mem_kind(q.in) != MK_DEVICE || mem_kind(q.out) != MK_DEVICE) return LEY_EINVAL;
    return LEY_OK;
}

ley_status check_pairs_request(const ley_pairs_request& q) {
    if (q.n >= (1ull << 32)) return LEY_EUNSUPPORTED;
    if (q.n == 0) return LEY_OK;
    if (!q.keys_in || !q.idx_in || !q.keys_out || !q.idx_out) return LEY_EINVAL;
    const ull n = q.n;
    if (overlaps(q.keys_in, n * 8, q.keys_out, n * 8) ||
        overlaps(q.idx_in, n * 4, q.idx_out, n * 4) ||
        overlaps(q.keys_in, n * 8, q.idx_out, n * 4) ||
        overlaps(q.idx_in, n * 4, q.keys_out, n * 8))
        return LEY_EINVAL;
    if (((uintptr_t)q.keys_in & 7u) || ((uintptr_t)q.keys_out & 7u) ||
        ((uintptr_t)q.idx_in & 3u) || ((uintptr_t)q.idx_out & 3u))
        return LEY_EINVAL;
    if (mem_kind(q.keys_in) != MK_DEVICE || mem_kind(q.idx_in) != MK_DEVICE ||
        mem_kind(q.keys_out) != MK_DEVICE || mem_kind(q.idx_out) != MK_DEVICE)
        return LEY_EINVAL;
    return LEY_OK;
}
}  // namespace ley

// ================================================================ C ABI

using namespace ley;

extern "C" {

static ley_status sort_records(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                               uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream,
                               bool block, const Tuning& tune) {
    if (key_bytes < 1 || key_bytes > rec_bytes ||
        rec_bytes > 4096 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (n == 0) return LEY_OK;
    if (!in || !out) return LEY_EINVAL;
    const ull bytes = n * rec_bytes;
    if (overlaps(in, bytes, out, bytes)) return LEY_EINVAL;
    const MemKind ki = mem_kind(in), ko = mem_kind(out);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SortArgs a{};
    a.mode = MODE_RECORDS;
    a.in = static_cast<const uint8_t*>(in);
    a.out = static_cast<uint8_t*>(out);
    a.n = n;
    a.rec = rec_bytes;
    a.kb = key_bytes;
    a.tune = tune;
    if (ki == MK_DEVICE && ko == MK_DEVICE) {
        if (!aligned16(in) || !aligned16(out)) return LEY_EINVAL;
        return run_device_sort(a, mem_budget, st);
    }
    if (ki == MK_HOST_PINNED && ko == MK_HOST_PINNED) return run_host_sort(a, mem_budget, st, block);
    return LEY_EINVAL;
}

ley_status ley_sort_records(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                            uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream) {
    return sort_records(in, out, n, rec_bytes, key_bytes, mem_budget, stream, true, cur_tuning());
}

ley_status ley_sort_records_async(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                                  uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream) {
    return sort_records(in, out, n, rec_bytes, key_bytes, mem_budget, stream, false,
                        cur_tuning());
}

ley_status ley_sort_keys_index(const uint64_t* keys_in, const uint32_t* idx_in,
                               uint64_t* keys_out, uint32_t* idx_out, uint64_t n,
                               uint64_t mem_budget, ley_stream_t stream) {
    if (n >= (1ull << 32)) return LEY_EUNSUPPORTED;
    if (n == 0) return LEY_OK;
    if (!keys_in || !idx_in || !keys_out || !idx_out) return LEY_EINVAL;
    if (overlaps(keys_in, n * 8, keys_out, n * 8) || overlaps(idx_in, n * 4, idx_out, n * 4) ||
        overlaps(keys_in, n * 8, idx_out, n * 4) || overlaps(idx_in, n * 4, keys_out, n * 8))
        return LEY_EINVAL;
    if (mem_kind(keys_in) != MK_DEVICE || mem_kind(idx_in) != MK_DEVICE ||
        mem_kind(keys_out) != MK_DEVICE || mem_kind(idx_out) != MK_DEVICE)
        return LEY_EINVAL;
    if (((uintptr_t)keys_in & 7u) || ((uintptr_t)keys_out & 7u) || ((uintptr_t)idx_in & 3u) || ((uintptr_t)idx_out & 3u))
        return LEY_EINVAL;
    SortArgs a{};
    a.mode = MODE_PAIRS;
    a.keys_in = keys_in;
    a.idx_in = idx_in;
    a.keys_out = keys_out;
    a.idx_out = idx_out;
    a.n = n;
    a.kb = 8;
    a.tune = cur_tuning();
    return run_device_sort(a, mem_budget, static_cast<cudaStream_t>(stream));
}


ley_status ley_sort_records_batch(const ley_records_request* reqs, uint32_t count,
                                  uint32_t rec_bytes, uint32_t key_bytes, uint64_t mem_budget,
                                  ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096)
        return LEY_EUNSUPPORTED;
    if (count == 0) return LEY_OK;
    if (!reqs) return LEY_EINVAL;
    std::vector<BatchReq> v;
    v.reserve(count);
    ull npos = 0;
    for (uint32_t r = 0; r < count; r++) {
        const ley_records_request& q = reqs[r];
        const ley_status c = check_records_request(q, rec_bytes, key_bytes);
        if (c != LEY_OK) return c;
        if (q.n == 0) continue;
        BatchReq b{};
        b.in = static_cast<const uint8_t*>(q.in);
        b.out = static_cast<uint8_t*>(q.out);
        b.n = q.n;
        b.off = npos;
        npos += (ull)ceil_div_u64(q.n, kPassTile) * kPassTile;
        v.push_back(b);
    }
    if (v.empty()) return LEY_OK;
    if (npos >= (1ull << 32)) return LEY_EUNSUPPORTED;
    return run_batch(v, npos, rec_bytes, key_bytes, false, mem_budget,
                     static_cast<cudaStream_t>(stream), cur_tuning());
}

ley_status ley_sort_keys_index_batch(const ley_pairs_request* reqs, uint32_t count,
                                     uint64_t mem_budget, ley_stream_t stream) {
    if (count == 0) return LEY_OK;
    if (!reqs) return LEY_EINVAL;
    std::vector<BatchReq> v;
    v.reserve(count);
    ull npos = 0;
    for (uint32_t r = 0; r < count; r++) {
        const ley_pairs_request& q = reqs[r];
        const ley_status c = check_pairs_request(q);
        if (c != LEY_OK) return c;
        if (q.n == 0) continue;
        const ull n = q.n;
        BatchReq b{};
        b.in = reinterpret_cast<const uint8_t*>(q.keys_in);
        b.out = reinterpret_cast<uint8_t*>(q.keys_out);
        b.idx_in = q.idx_in;
        b.idx_out = q.idx_out;
        b.n = n;
        b.off = npos;
        npos += (ull)ceil_div_u64(n, kPassTile) * kPassTile;
        v.push_back(b);
    }
    if (v.empty()) return LEY_OK;
    if (npos >= (1ull << 32)) return LEY_EUNSUPPORTED;
    return run_batch(v, npos, 8, 8, true, mem_budget, static_cast<cudaStream_t>(stream),
                     cur_tuning());
}

ley_status ley_partition_records(const void* in, uint64_t n, uint32_t rec_bytes,
                                 uint32_t key_bytes, uint32_t digit, uint32_t* order_out,
                                 uint64_t* hist_out, ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (digit >= key_bytes) return LEY_EINVAL;
    if (!in || !order_out || !hist_out) return LEY_EINVAL;
    if (mem_kind(in) != MK_DEVICE || mem_kind(order_out) != MK_DEVICE ||
        mem_kind(hist_out) != MK_DEVICE)
        return LEY_EINVAL;
    if (!aligned16(in) || ((uintptr_t)order_out & 3u) || ((uintptr_t)hist_out & 7u))
        return LEY_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        return cudaMemsetAsync(hist_out, 0, 256 * sizeof(uint64_t), st) == cudaSuccess
                   ? LEY_OK
                   : LEY_ECUDA;
    }
    SortArgs a{};
    a.mode = MODE_PARTITION;
    a.in = static_cast<const uint8_t*>(in);
    a.order_out = order_out;
    a.hist_out = reinterpret_cast<ull*>(hist_out);
    a.n = n;
    a.rec = rec_bytes;
    a.kb = key_bytes;
    a.digit = digit;
    a.tune = cur_tuning();
    return run_device_sort(a, 0, st);
}

ley_status ley_plan_partitions(const void* const* runs, const uint64_t* run_len, uint32_t k,
                               uint32_t rec_bytes, uint32_t key_bytes, uint64_t cap,
                               uint64_t* cuts, uint64_t max_cuts, uint64_t* ncuts) {
    if (key_bytes < 1 || key_bytes > rec_bytes || rec_bytes < 1 || rec_bytes > 4096)
        return LEY_EUNSUPPORTED;
    if (k < 1 || k > 4096 || cap < 1 || !run_len || !cuts || !ncuts || !runs) return LEY_EINVAL;
    std::vector<HostRun> rs(k);
    ull n = 0;
    for (uint32_t i = 0; i < k; i++) {
        if (run_len[i] && !runs[i]) return LEY_EINVAL;
        rs[i] = {static_cast<const uint8_t*>(runs[i]), run_len[i]};
        n += run_len[i];
    }
    const std::vector<std::vector<ull>> c = plan_partitions(rs, n, cap, rec_bytes, key_bytes);
    *ncuts = c.size();
    if (c.size() > max_cuts) return LEY_ENOMEM;
    for (size_t p = 0; p < c.size(); p++)
        for (uint32_t i = 0; i < k; i++) cuts[p * k + i] = c[p][i];
    return LEY_OK;
}

ley_status ley_merge_records(const void* runs, const uint64_t* run_start, uint32_t k, void* out,
                             uint32_t rec_bytes, uint32_t key_bytes, ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096)
        return LEY_EUNSUPPORTED;
    if (k < 1 || k > 128) return LEY_EUNSUPPORTED;
    if (!run_start) return LEY_EINVAL;
    std::vector<ull> off(run_start, run_start + k + 1);
    if (off[0] != 0) return LEY_EINVAL;
    for (uint32_t i = 0; i < k; i++)
        if (off[i + 1] < off[i]) return LEY_EINVAL;
    const ull n = off[k];
    if (n >= (1ull << 32)) return LEY_EUNSUPPORTED;
    if (n == 0) return LEY_OK;
    if (!runs || !out) return LEY_EINVAL;
    if (overlaps(runs, n * rec_bytes, out, n * rec_bytes)) return LEY_EINVAL;
    if (mem_kind(runs) != MK_DEVICE || mem_kind(out) != MK_DEVICE) return LEY_EINVAL;
    if (!aligned16(runs) || !aligned16(out)) return LEY_EINVAL;
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Tuning tune = cur_tuning();
    const Layout L = make_layout(n, true, tune.big);
    const size_t total = L.total + align_up(sizeof(ull) * (k + 1), 256);
    void* base = nullptr;
    if (!scratch_alloc(ds, &base, total, st)) return LEY_ENOMEM;
    SortArgs a{};
    a.mode = MODE_RECORDS;
    a.in = static_cast<const uint8_t*>(runs);
    a.out = static_cast<uint8_t*>(out);
    a.n = n;
    a.rec = rec_bytes;
    a.kb = key_bytes;
    a.tune = tune;
    Work w = make_work(static_cast<char*>(base), L, n, ds->err);
    ull* off_dev = reinterpret_cast<ull*>(static_cast<char*>(base) + L.total);
    ley_status s = stage_merge(a, a.in, off.data(), off_dev, k, w, L, st, ds->sms);
    if (s == LEY_OK) s = stage_gather(a, w.perm, st, ds->sms, 0, n, a.out);
    cudaFreeAsync(base, st);
    return s;
}

ley_status ley_workspace_bytes(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                               uint64_t mem_budget, uint64_t* bytes) {
    if (!bytes) return LEY_EINVAL;
    *bytes = 0;
    if (key_bytes < 1 || key_bytes > rec_bytes || rec_bytes > 4096 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (n == 0) return LEY_OK;
    const Tuning tune = cur_tuning();
    if (mem_budget == 0) {  // the internal sort of device buffers
        *bytes = key_bytes > kWindow ? make_layout(n, true, tune.big).total + long_key_extra(n)
                                     : make_layout(n, !fused_gather(rec_bytes), tune.big).total;
        return LEY_OK;
    }
    // pinned host buffers under the budget: the partial mode if it fits, else
    // the external mode
    const size_t part = partial_need(n, rec_bytes, key_bytes, mem_budget, tune);
    if (part <= mem_budget) {
        *bytes = part;
        return LEY_OK;
    }
    ExtPlan plan;
    const ley_status s = external_plan(n, rec_bytes, key_bytes, mem_budget, tune, &plan);
    if (s != LEY_OK) return s;
    *bytes = plan.total;
    return LEY_OK;
}

ley_status ley_host_scratch_bytes(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                                  uint64_t mem_budget, uint64_t* bytes) {
    if (!bytes) return LEY_EINVAL;
    *bytes = 0;
    if (key_bytes < 1 || key_bytes > rec_bytes || rec_bytes > 4096 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (n == 0 || mem_budget == 0) return LEY_OK;
    const Tuning tune = cur_tuning();
    if (partial_need(n, rec_bytes, key_bytes, mem_budget, tune) <= mem_budget) return LEY_OK;
    ExtPlan plan;
    const ley_status s = external_plan(n, rec_bytes, key_bytes, mem_budget, tune, &plan);
    if (s != LEY_OK) return s;
    *bytes = plan.host_bytes;
    return LEY_OK;
}

ley_status ley_get_tuning(ley_tuning* t) {
    if (!t) return LEY_EINVAL;
    const Tuning c = cur_tuning();
    t->big_bucket = c.big;
    t->tiny_bucket = c.tiny;
    t->finish_ctas_per_sm = c.fin_ctas;
    t->pass_ctas_per_sm = c.pass_ctas;
    return LEY_OK;
}

ley_status ley_set_tuning(const ley_tuning* t) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return LEY_ECUDA;
    Tuning c;
    if (t) {
        if (t->big_bucket < 256 || t->big_bucket > (uint32_t)kSmall) return LEY_EINVAL;
        if (t->tiny_bucket < (uint32_t)kTiny || t->tiny_bucket > (uint32_t)kWarpMax) return LEY_EINVAL;
        if (t->finish_ctas_per_sm > 64 || t->pass_ctas_per_sm > 64) return LEY_EINVAL;
        c.big = t->big_bucket;
        c.tiny = t->tiny_bucket;
        c.fin_ctas = t->finish_ctas_per_sm;
        c.pass_ctas = t->pass_ctas_per_sm;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune[d] = c;
    return LEY_OK;
}

}  // extern "C"

namespace ley {
// Times sorts of the n records at `in` (device) into `out` under a grid of
// tunings -- Algorithm 1's two thresholds and the finishing CTAs per SM; the
// first candidate is the default -- keeps the fastest (best of two timed
// sorts after one warm-up) as the current tuning and returns it.  Each timed
// sort gets its candidate as its own tuning; the current tuning is written
// only once, at the end, so sorts that other threads start meanwhile run with
// the tuning that was current before.
static ley_status autotune_on(const void* in, void* out, ull n, uint32_t rec_bytes,
                              uint32_t key_bytes, cudaStream_t st, ley_tuning* best) {
    ley_status s = LEY_OK;
    std::vector<Tuning> cands;
    for (uint32_t big : {2048u, 1536u, 1024u})
        for (uint32_t tiny : {32u, 64u, 128u})
            for (uint32_t fc : {0u, 3u}) {
                Tuning c;
                c.big = big;
                c.tiny = tiny;
                c.fin_ctas = fc;
                cands.push_back(c);
            }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = LEY_ECUDA;
    float best_ms = 1e30f;
    Tuning best_t = cands[0];
    for (size_t i = 0; i < cands.size() && s == LEY_OK; i++) {
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && s == LEY_OK; rep++) {  // first run warms up
            cudaEventRecord(e0, st);
            s = sort_records(in, out, n, rec_bytes, key_bytes, 0, st, true, cands[i]);
            cudaEventRecord(e1, st);
            if (s == LEY_OK && cudaEventSynchronize(e1) != cudaSuccess) s = LEY_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
        }
        if (s == LEY_OK && ms < best_ms) {
            best_ms = ms;
            best_t = cands[i];
        }
    }
    if (s == LEY_OK) s = ley_last_device_status(st);
    if (s == LEY_OK) {
        std::lock_guard<std::mutex> lk(g_mu);
        int d = 0;
        cudaGetDevice(&d);
        g_tune[d] = best_t;
    }
    if (best) {
        best->big_bucket = best_t.big;
        best->tiny_bucket = best_t.tiny;
        best->finish_ctas_per_sm = best_t.fin_ctas;
        best->pass_ctas_per_sm = best_t.pass_ctas;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return s;
}
}  // namespace ley

extern "C" {

ley_status ley_autotune_records(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                                uint64_t seed, ley_tuning* best) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096 || n == 0 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LEY_ECUDA;
    const ull bytes = n * rec_bytes;
    void *in = nullptr, *out = nullptr;
    ley_status s = LEY_OK;
    if (!scratch_alloc(ds, &in, align_up(bytes, 256), st) ||
        !scratch_alloc(ds, &out, align_up(bytes, 256), st))
        s = LEY_ENOMEM;
    if (s == LEY_OK && launch_fill_random(st, static_cast<uint8_t*>(in), bytes, seed) != cudaSuccess)
        s = LEY_ECUDA;
    if (s == LEY_OK) s = autotune_on(in, out, n, rec_bytes, key_bytes, st, best);
    if (in) cudaFreeAsync(in, st);
    if (out) cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ley_status ley_autotune_records_on(const void* in, uint64_t n, uint32_t rec_bytes,
                                   uint32_t key_bytes, ley_tuning* best, ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096 || n == 0 || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    if (!in) return LEY_EINVAL;
    if (mem_kind(in) != MK_DEVICE || !aligned16(in)) return LEY_EINVAL;
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LEY_ECUDA;
    // The timed sorts read `in` only after the work the caller queued on
    // `stream` before this call (which may still be writing it).
    {
        cudaEvent_t ready = nullptr;
        const bool ok = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventRecord(ready, static_cast<cudaStream_t>(stream)) == cudaSuccess &&
                        cudaStreamWaitEvent(st, ready, 0) == cudaSuccess;
        if (ready) cudaEventDestroy(ready);
        if (!ok) {
            cudaGetLastError();
            cudaStreamDestroy(st);
            return LEY_ECUDA;
        }
    }
    void* out = nullptr;
    ley_status s = LEY_OK;
    if (!scratch_alloc(ds, &out, align_up(n * rec_bytes, 256), st)) s = LEY_ENOMEM;
    if (s == LEY_OK) s = autotune_on(in, out, n, rec_bytes, key_bytes, st, best);
    if (out) cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return s;
}

ley_status ley_selftest_timeout(uint32_t which, ley_stream_t stream) {
    if (which > 1) return LEY_EINVAL;
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* word = nullptr;
    if (!scratch_alloc(ds, &word, 256, st)) return LEY_ENOMEM;
    ley_status s = LEY_OK;
    if (cudaMemsetAsync(word, 0, 256, st) != cudaSuccess ||
        launch_selftest_wait(st, which, static_cast<const unsigned long long*>(word), ds->err) !=
            cudaSuccess)
        s = LEY_ECUDA;
    cudaFreeAsync(word, st);
    const ley_status d = ley_last_device_status(stream);
    return s != LEY_OK ? s : d;
}

ley_status ley_release_cache(void) {
    {
        std::lock_guard<std::mutex> lk(g_host_scratch_mu);
        if (g_host_scratch && cudaFreeHost(g_host_scratch) != cudaSuccess) return LEY_ECUDA;
        g_host_scratch = nullptr;
        g_host_scratch_bytes = 0;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& d : g_dev)
        if (d.init && d.pool && cudaMemPoolTrimTo(d.pool, 0) != cudaSuccess) return LEY_ECUDA;
    return LEY_OK;
}

const char* ley_status_string(ley_status s) {
    switch (s) {
        case LEY_OK: return "ok";
        case LEY_EINVAL: return "invalid argument";
        case LEY_ENOMEM: return "scratch would exceed the memory budget, or allocation failed";
        case LEY_EUNSUPPORTED: return "record or key geometry not supported";
        case LEY_ECUDA: return "CUDA runtime error";
        case LEY_ETIMEOUT: return "a device-side bounded wait gave up";
    }
    return "unknown status";
}

ley_status ley_last_device_status(ley_stream_t stream) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return LEY_ECUDA;
    uint32_t ev[2] = {0, 0};
    if (cudaMemcpy(ev, ds->err, sizeof(ev), cudaMemcpyDeviceToHost) != cudaSuccess) return LEY_ECUDA;
    const uint32_t v = ev[0];
    if (v && cudaMemset(ds->err, 0, sizeof(ev)) != cudaSuccess) return LEY_ECUDA;
    if (v && std::getenv("LEY_DEBUG"))
        std::fprintf(stderr, "leysort: device error bits 0x%x first raised at file %u line %u\n", v,
                     ev[1] >> 16, ev[1] & 0xFFFFu);
    if (v & kErrTimeout) return LEY_ETIMEOUT;
    if (v & kErrCapacity) return LEY_ENOMEM;
    return LEY_OK;
}

uint64_t ley_launch_count(void) { return g_launches.load(); }

ley_status ley_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    if (g_prof_on) {
        for (auto& p : g_pending) {
            g_ev_pool.push_back(p.a);
            g_ev_pool.push_back(p.b);
        }
        g_pending.clear();
        g_prof.clear();
    }
    return LEY_OK;
}

int ley_profile_read(ley_kernel_time* out, int max) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess) cudaEventElapsedTime(&ms, p.a, p.b);
        bool found = false;
        for (auto& e : g_prof) {
            if (std::strcmp(e.name, p.name) == 0) {
                e.launches++;
                e.ms += ms;
                found = true;
                break;
            }
        }
        if (!found) g_prof.push_back({p.name, 1, (double)ms});
        g_ev_pool.push_back(p.a);
        g_ev_pool.push_back(p.b);
    }
    g_pending.clear();
    int k = 0;
    for (auto& e : g_prof) {
        if (k < max && out) {
            out[k].name = e.name;
            out[k].launches = e.launches;
            out[k].total_ms = e.ms;
        }
        k++;
    }
    return k;
}

}  // extern "C"

// ===================================================== allocation-free sort
//
// ley_sort_records_noalloc serves callers that cannot allocate device memory:
// for example an application whose device memory is entirely owned by its own
// pool allocator, or a latency-bound caller for which a cudaMalloc (which can
// wait for the whole device) is not acceptable.  Its scratch is one file-scope
// device array, so the call itself never allocates or frees.

namespace ley {

// Largest input of the allocation-free sort, and its fixed scratch size: the
// workspace of an internal sort of that many records plus one 256-byte block
// at the end for the call's device status words.
constexpr unsigned long long kNoAllocMaxRecords = LEY_NOALLOC_MAX_RECORDS;
constexpr size_t kNoAllocBytes = 12u << 20;
constexpr size_t kNoAllocStatusBytes = 256;

// The scratch array.  It lives in every device's copy of this library's
// device code, from the time that code is loaded until the process exits.
// Host code must not use its name as an address: it resolves the device
// address with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDev {
    bool init = false;
    char* base = nullptr;   // device address of g_noalloc_scratch
    int sms = 0;
};
static NoAllocDev g_noalloc[64];
static std::mutex g_noalloc_mu;

// Once per device, with that device current: the scratch array's device
// address and the SM count.  Allocates nothing.
static NoAllocDev* noalloc_setup() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDev& s = g_noalloc[d];
    if (!s.init) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return nullptr;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
            return nullptr;
        s.base = static_cast<char*>(p);
        s.sms = sms;
        s.init = true;
    }
    return &s;
}

// The internal record sort of enqueue_sort, with all scratch at `base` and
// device errors latched in `err` (no per-device state of the library used).
static ley_status enqueue_records_noalloc(const SortArgs& a, char* base, const Layout& L,
                                          cudaStream_t st, int sms, uint32_t* err) {
    Work w = make_work(base, L, a.n, err);
    const KeySpec ks = record_keyspec(a.kb, Tuning{});  // fixed scratch: default thresholds
    LEY_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
    LEY_TRY(cudaMemsetAsync(w.diff[0], 0, sizeof(Diff), st));
    LEY_TRY(cudaMemsetAsync(w.status, 0, L.cap_chunks * kRadix * sizeof(ull), st));
    LEY_TRY(launch_init(st, w, a.n, 0));
    {
        LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_REC), 256, 0, st};
        LEY_TRY(launch_extract_records(c, a.in, a.n, a.rec, ks, w, 0));
    }
    const LaunchCfg cp{sms * blocks_per_sm(KK_PASS), kPassThreads, kernel_smem(KK_PASS), st};
    const LaunchCfg cs{sms * blocks_per_sm(KK_SCAN), kRadix, 0, st};
    const LaunchCfg ch{sms * blocks_per_sm(KK_HIST), kHistThreads, 0, st};
    const LaunchCfg cc{8 * sms, 128, 0, st};
    for (int lvl = 0; lvl < ks.ndig; lvl++) {
        if (lvl > 0) LEY_TRY(launch_hist(ch, w, ks, lvl));
        LEY_TRY(launch_scan(cs, w, lvl));
        LEY_TRY(launch_classify(cc, w, ks, lvl));
        LEY_TRY(launch_pass(cp, w, ks, lvl));
    }
    LaunchCfg cf{sms * blocks_per_sm(KK_FINISH_REC), kFinThreads, kernel_smem(KK_FINISH_REC), st};
    LEY_TRY(launch_finish_records(cf, w, ks));
    const int gv = a.rec == 100 ? 1 : 0;
    const KernelKind gk = a.rec != 100 ? KK_GATHER_GENERIC
                                       : (gv == 1 ? KK_GATHER100_TMA : KK_GATHER100);
    LaunchCfg cg{sms * blocks_per_sm(gk), 0, 0, st};
    LEY_TRY(launch_gather_err(cg, a.in, a.out, w.perm, a.n, a.n, a.rec, gv, err));
    return LEY_OK;
}

}  // namespace ley

extern "C" ley_status ley_sort_records_noalloc(const void* in, void* out, uint64_t n,
                                               uint32_t rec_bytes, uint32_t key_bytes,
                                               ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes ||
        rec_bytes > 4096)
        return LEY_EUNSUPPORTED;
    if (n > kNoAllocMaxRecords) return LEY_ENOMEM;
    if (n == 0) return LEY_OK;
    if (!in || !out) return LEY_EINVAL;
    const ull bytes = n * rec_bytes;
    if (overlaps(in, bytes, out, bytes)) return LEY_EINVAL;
    if (mem_kind(in) != MK_DEVICE || mem_kind(out) != MK_DEVICE) return LEY_EINVAL;
    if (!aligned16(in) || !aligned16(out)) return LEY_EINVAL;
    NoAllocDev* dev = noalloc_setup();
    if (!dev) return LEY_ECUDA;
    const Layout L = make_layout(n, true, kSmall);
    if (L.total + kNoAllocStatusBytes > kNoAllocBytes) return LEY_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* err = reinterpret_cast<uint32_t*>(dev->base + kNoAllocBytes - kNoAllocStatusBytes);
    // The array keeps the previous call's contents: clear the status words
    // (the sort itself clears its counters, statuses and digit masks).
    if (cudaMemsetAsync(err, 0, kNoAllocStatusBytes, st) != cudaSuccess) return LEY_ECUDA;
    SortArgs a{};
    a.mode = MODE_RECORDS;
    a.in = static_cast<const uint8_t*>(in);
    a.out = static_cast<uint8_t*>(out);
    a.n = n;
    a.rec = rec_bytes;
    a.kb = key_bytes;
    const ley_status s = enqueue_records_noalloc(a, dev->base, L, st, dev->sms, err);
    if (s != LEY_OK) return s;
    uint32_t ev[2] = {0, 0};
    if (cudaMemcpyAsync(ev, err, sizeof(ev), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LEY_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LEY_ECUDA;
    if (ev[0] & kErrTimeout) return LEY_ETIMEOUT;
    if (ev[0] & kErrCapacity) return LEY_ENOMEM;
    return LEY_OK;
}
