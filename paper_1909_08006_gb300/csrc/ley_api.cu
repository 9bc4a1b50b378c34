// C ABI of leysort: argument checks, scratch layout, the launch sequence of
// the internal sort, and the host-memory (partially in-memory) mode.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
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
};
static DevState g_dev[64];
static std::mutex g_mu;
static std::atomic<unsigned long long> g_launches{0};

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
        (void)blocks_per_sm(KK_PASS);  // occupancy tables and smem attributes
        s.init = true;
    }
    return &s;
}

uint32_t* device_err_word() {
    DevState* s = dev_state();
    return s ? s->err : nullptr;
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

static Layout make_layout(ull n, bool with_perm) {
    Layout L{};
    L.cap_seg = n / kSmall + 2;
    L.cap_tiles = n / kPassTile + L.cap_seg + 1;
    L.cap_chunks = L.cap_tiles / kScanChunk + 1;
    L.cap_fin = 100 * (n / kSmall + 1) + 16;
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

static KeySpec record_keyspec(uint32_t kb) {
    KeySpec ks;
    ks.ndig = (int)kb;
    ks.hi_mask = kb >= 8 ? ~0ull : (~0ull << (64 - 8 * kb));
    ks.lo_mask = kb <= 8 ? 0u : (kb >= 12 ? ~0u : (~0u << (32 - 8 * (kb - 8))));
    return ks;
}

static KeySpec pair_keyspec() {
    KeySpec ks;
    ks.ndig = 8;
    ks.hi_mask = ~0ull;
    ks.lo_mask = 0u;
    return ks;
}

// Record gather kernel: TMA bulk copies (default) or plain vector loads
// (LEY_GATHER=lsu), kept for comparison.
static int gather_variant() {
    const char* v = std::getenv("LEY_GATHER");
    if (v && std::strcmp(v, "lsu") == 0) return 0;
    return 1;
}

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
};

#define LEY_TRY(x)                                   \
    do {                                             \
        if ((x) != cudaSuccess) return LEY_ECUDA;    \
    } while (0)

// Queues the whole sort on `st` using scratch at `base` (layout L).
static ley_status enqueue_sort(const SortArgs& a, char* base, const Layout& L, cudaStream_t st,
                               DevState* ds) {
    Work w = make_work(base, L, a.n, ds->err);
    const KeySpec ks = a.mode == MODE_PAIRS ? pair_keyspec() : record_keyspec(a.kb);
    const int sms = ds->sms;
    LEY_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), st));
    LEY_TRY(cudaMemsetAsync(w.diff[0], 0, sizeof(Diff), st));
    LEY_TRY(cudaMemsetAsync(w.status, 0, L.cap_chunks * kRadix * sizeof(ull), st));
    const int digit0 = a.mode == MODE_PARTITION ? (int)a.digit : 0;
    LEY_TRY(launch("init", st, [&] { return launch_init(st, w, a.n, digit0); }));
    if (a.mode == MODE_PAIRS) {
        LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_PAIRS), 256, 0, st};
        LEY_TRY(launch("extract", st, [&] {
            return launch_extract_pairs(c, a.keys_in, a.idx_in, a.n, ks, w);
        }));
    } else {
        LaunchCfg c{sms * blocks_per_sm(KK_EXTRACT_REC), 256, 0, st};
        LEY_TRY(launch("extract", st, [&] {
            return launch_extract_records(c, a.in, a.n, a.rec, ks, w, digit0);
        }));
    }
    const LaunchCfg cp{sms * blocks_per_sm(KK_PASS), kPassThreads, kernel_smem(KK_PASS), st};
    const LaunchCfg cs{sms * blocks_per_sm(KK_SCAN), kRadix, 0, st};
    if (a.mode == MODE_PARTITION) {
        LEY_TRY(launch("scan", st, [&] { return launch_scan(cs, w, 0); }));
        LEY_TRY(launch("classify", st, [&] { return launch_classify_partition(st, w); }));
        LEY_TRY(launch("pass", st, [&] { return launch_pass(cp, w, ks, 0); }));
        LEY_TRY(launch("partition_out", st, [&] {
            return launch_partition_out(st, sms * 4, w, a.n, a.order_out, a.hist_out);
        }));
        return LEY_OK;
    }
    const LaunchCfg ch{sms * blocks_per_sm(KK_HIST), kHistThreads, 0, st};
    const LaunchCfg cc{2 * sms, 128, 0, st};
    for (int lvl = 0; lvl < ks.ndig; lvl++) {
        if (lvl > 0) LEY_TRY(launch("hist", st, [&] { return launch_hist(ch, w, ks, lvl); }));
        LEY_TRY(launch("scan", st, [&] { return launch_scan(cs, w, lvl); }));
        LEY_TRY(launch("classify", st, [&] { return launch_classify(cc, w, ks, lvl); }));
        LEY_TRY(launch("pass", st, [&] { return launch_pass(cp, w, ks, lvl); }));
    }
    if (a.mode == MODE_PAIRS) {
        LaunchCfg cf{sms * blocks_per_sm(KK_FINISH_PAIRS), kFinThreads,
                     kernel_smem(KK_FINISH_PAIRS), st};
        LEY_TRY(launch("finish", st, [&] {
            return launch_finish_pairs(cf, w, ks, a.keys_out, a.idx_out);
        }));
        return LEY_OK;
    }
    LaunchCfg cf{sms * blocks_per_sm(KK_FINISH_REC), kFinThreads, kernel_smem(KK_FINISH_REC), st};
    LEY_TRY(launch("finish", st, [&] { return launch_finish_records(cf, w, ks); }));
    const int gv = a.rec == 100 ? gather_variant() : 0;
    const KernelKind gk = a.rec != 100 ? KK_GATHER_GENERIC
                                       : (gv == 1 ? KK_GATHER100_TMA : KK_GATHER100);
    LaunchCfg cg{sms * blocks_per_sm(gk), 0, 0, st};
    LEY_TRY(launch("gather", st, [&] {
        return launch_gather(cg, a.in, a.out, w.perm, a.n, a.rec, gv);
    }));
    return LEY_OK;
}

static ley_status run_device_sort(const SortArgs& a, ull budget, cudaStream_t st) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    const Layout L = make_layout(a.n, a.mode == MODE_RECORDS);
    if (budget && L.total > budget) return LEY_ENOMEM;
    void* base = nullptr;
    if (cudaMallocAsync(&base, L.total, st) != cudaSuccess) {
        cudaGetLastError();
        return LEY_ENOMEM;
    }
    ley_status s = enqueue_sort(a, static_cast<char*>(base), L, st, ds);
    cudaFreeAsync(base, st);
    return s;
}

// ------------------------------------------------- host-memory sorting

// Partially in-memory sort (Section 4.1's 20 GB case, the page-cache scatter
// of Section 3.2): pinned host input and output, the input resident on the
// device for the sort, the sorted records streamed back.  Blocks.
static ley_status run_host_partial(const SortArgs& a, ull budget, cudaStream_t st) {
    DevState* ds = dev_state();
    if (!ds) return LEY_ECUDA;
    const ull bytes = a.n * a.rec;
    const Layout L = make_layout(a.n, true);
    const size_t need = align_up(bytes, 256) * 2 + L.total;
    if (budget && need > budget) return LEY_ENOMEM;
    void* dmem = nullptr;
    if (cudaMallocAsync(&dmem, need, st) != cudaSuccess) {
        cudaGetLastError();
        return LEY_ENOMEM;
    }
    char* din = static_cast<char*>(dmem);
    char* dout = din + align_up(bytes, 256);
    char* ws = dout + align_up(bytes, 256);
    ley_status s = LEY_OK;
    if (cudaMemcpyAsync(din, a.in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) s = LEY_ECUDA;
    if (s == LEY_OK) {
        SortArgs d = a;
        d.in = reinterpret_cast<const uint8_t*>(din);
        d.out = reinterpret_cast<uint8_t*>(dout);
        s = enqueue_sort(d, ws, L, st, ds);
    }
    if (s == LEY_OK &&
        cudaMemcpyAsync(a.out, dout, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = LEY_ECUDA;
    cudaFreeAsync(dmem, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return LEY_ECUDA;
    return s;
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

// ================================================================ C ABI

using namespace ley;

extern "C" {

ley_status ley_sort_records(const void* in, void* out, uint64_t n, uint32_t rec_bytes,
                            uint32_t key_bytes, uint64_t mem_budget, ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes || rec_bytes < 4 ||
        rec_bytes > 4096 || (rec_bytes & 3u) || n >= (1ull << 32))
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
    if (ki == MK_DEVICE && ko == MK_DEVICE) {
        if (!aligned16(in) || !aligned16(out)) return LEY_EINVAL;
        return run_device_sort(a, mem_budget, st);
    }
    if (ki == MK_HOST_PINNED && ko == MK_HOST_PINNED) return run_host_partial(a, mem_budget, st);
    return LEY_EINVAL;
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
    return run_device_sort(a, mem_budget, static_cast<cudaStream_t>(stream));
}

ley_status ley_partition_records(const void* in, uint64_t n, uint32_t rec_bytes,
                                 uint32_t key_bytes, uint32_t digit, uint32_t* order_out,
                                 uint64_t* hist_out, ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes || rec_bytes < 4 ||
        rec_bytes > 4096 || (rec_bytes & 3u) || n >= (1ull << 32))
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
    return run_device_sort(a, 0, st);
}

ley_status ley_workspace_bytes(uint64_t n, uint32_t rec_bytes, uint32_t key_bytes,
                               uint64_t* bytes) {
    if (!bytes) return LEY_EINVAL;
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes || rec_bytes < 4 ||
        rec_bytes > 4096 || (rec_bytes & 3u) || n >= (1ull << 32))
        return LEY_EUNSUPPORTED;
    *bytes = n ? make_layout(n, true).total : 0;
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
    const KeySpec ks = record_keyspec(a.kb);
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
    const LaunchCfg cc{2 * sms, 128, 0, st};
    for (int lvl = 0; lvl < ks.ndig; lvl++) {
        if (lvl > 0) LEY_TRY(launch_hist(ch, w, ks, lvl));
        LEY_TRY(launch_scan(cs, w, lvl));
        LEY_TRY(launch_classify(cc, w, ks, lvl));
        LEY_TRY(launch_pass(cp, w, ks, lvl));
    }
    LaunchCfg cf{sms * blocks_per_sm(KK_FINISH_REC), kFinThreads, kernel_smem(KK_FINISH_REC), st};
    LEY_TRY(launch_finish_records(cf, w, ks));
    const int gv = a.rec == 100 ? gather_variant() : 0;
    const KernelKind gk = a.rec != 100 ? KK_GATHER_GENERIC
                                       : (gv == 1 ? KK_GATHER100_TMA : KK_GATHER100);
    LaunchCfg cg{sms * blocks_per_sm(gk), 0, 0, st};
    LEY_TRY(launch_gather_err(cg, a.in, a.out, w.perm, a.n, a.rec, gv, err));
    return LEY_OK;
}

}  // namespace ley

extern "C" ley_status ley_sort_records_noalloc(const void* in, void* out, uint64_t n,
                                               uint32_t rec_bytes, uint32_t key_bytes,
                                               ley_stream_t stream) {
    if (key_bytes < 1 || key_bytes > 12 || key_bytes > rec_bytes || rec_bytes < 4 ||
        rec_bytes > 4096 || (rec_bytes & 3u))
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
    const Layout L = make_layout(n, true);
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
