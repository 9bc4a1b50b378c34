// A sort server: continuous batching of sort requests on one GPU.
//
// Requests (100-byte-class records, or (u64 key, u32 payload) pairs) are
// submitted from any host thread with their device buffers already resident.
// A scheduler thread admits pending requests in arrival order into a batch
// while a launch slot (a CUDA stream) is free and their device memory -- the
// request's own input and output plus the batch's sort scratch -- fits the
// server's budget, and launches the batch with the batched sorts of this
// library.  Requests that arrive while batches run are admitted into the next
// batch as soon as a slot and memory free up, so batches of different slots
// overlap on the device.  A completion thread waits for each batch's event,
// stamps its requests' completion times and returns their memory.  Each
// request is sorted exactly as its own ley_sort_records / ley_sort_keys_index
// call would sort it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "leysort.h"
#include "ley_internal.cuh"

namespace ley {

using ull = unsigned long long;
using Clock = std::chrono::steady_clock;

ley_status check_records_request(const ley_records_request& q, uint32_t rec_bytes,
                                 uint32_t key_bytes);  // ley_api.cu
ley_status check_pairs_request(const ley_pairs_request& q);

struct SrvReq {
    ull ticket;
    int kind;  // 0 records, 1 pairs
    ley_records_request rec;
    ley_pairs_request pairs;
    uint32_t rec_bytes, key_bytes;
    ull bytes;  // device bytes charged while the request is in flight
    double t_submit, t_start, t_done;
    double dev_start, dev_done;  // device clock: the batch's start and completion events
    ull batch;                   // number of the batch that carried it
    int status;  // -1 pending, else ley_status
};

struct Batch {
    int slot;
    ull id;
    cudaEvent_t start, done;  // timing events on the slot stream around the batch's work
    std::vector<ull> tickets;
    ull bytes;
    double t_launch;
};

}  // namespace ley

struct ley_server {
    int device = 0;
    unsigned long long budget = 0;
    uint32_t max_batch = 0;
    int nslots = 0;
    std::vector<cudaStream_t> slots;
    std::vector<bool> slot_busy;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<unsigned long long> pending;
    std::unordered_map<unsigned long long, ley::SrvReq> reqs;
    std::deque<ley::Batch> inflight;
    unsigned long long next_ticket = 1, in_use = 0, launched_batches = 0;
    bool stop = false, sched_done = false;
    std::thread sched, compl_;
    ley::Clock::time_point t0 = ley::Clock::now();
    // Recorded when the server is created: the origin of the device-clock
    // batch intervals (cudaEventElapsedTime against it).
    cudaEvent_t t0_ev = nullptr;

    double now() const {
        return std::chrono::duration<double>(ley::Clock::now() - t0).count();
    }
};

namespace ley {

// Device bytes a request holds while admitted: its buffers plus its share of
// the batch scratch (36 bytes per tuple slot of its tile-rounded size, plus a
// permutation for record sizes other than 100).
static ull request_bytes(const SrvReq& r) {
    const ull n = r.kind == 0 ? r.rec.n : r.pairs.n;
    const ull slots = (n + kPassTile - 1) / kPassTile * kPassTile;
    ull scratch = slots * 36 + 64 * 1024;
    if (r.kind == 0 && r.rec_bytes != 100) scratch += slots * 4;
    const ull own = r.kind == 0 ? 2 * n * r.rec_bytes : 2 * n * 12;
    return own + scratch;
}

static void scheduler(ley_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_sched.wait(lk, [&] {
            if (S->pending.empty()) return S->stop;
            for (bool b : S->slot_busy)
                if (!b) return true;
            return false;
        });
        if (S->pending.empty()) break;  // stopping, and everything submitted is launched
        int slot = -1;
        for (int i = 0; i < S->nslots; i++)
            if (!S->slot_busy[i]) {
                slot = i;
                break;
            }
        if (slot < 0) continue;
        // Admit in arrival order while memory fits (a request larger than the
        // whole budget is admitted alone once nothing else is in flight).
        std::vector<ull> take;
        ull bytes = 0;
        while (!S->pending.empty() && take.size() < S->max_batch) {
            SrvReq& r = S->reqs[S->pending.front()];
            const bool fits = S->in_use + bytes + r.bytes <= S->budget;
            const bool alone = take.empty() && S->in_use == 0;
            if (!fits && !alone) break;
            take.push_back(r.ticket);
            bytes += r.bytes;
            S->pending.pop_front();
        }
        if (take.empty()) {
            // memory is held by batches in flight: wait for a completion
            S->cv_sched.wait(lk);
            continue;
        }
        S->in_use += bytes;
        S->slot_busy[slot] = true;
        // Group the batch by kind and geometry; each group is one batched call.
        std::vector<ley_records_request> rq;
        std::vector<ley_pairs_request> pq;
        std::vector<std::pair<std::pair<uint32_t, uint32_t>, std::vector<ley_records_request>>> geo;
        const double t_launch = S->now();
        for (ull t : take) {
            SrvReq& r = S->reqs[t];
            r.t_start = t_launch;
            if (r.kind == 1) {
                pq.push_back(r.pairs);
                continue;
            }
            auto key = std::make_pair(r.rec_bytes, r.key_bytes);
            auto it = std::find_if(geo.begin(), geo.end(), [&](auto& g) { return g.first == key; });
            if (it == geo.end()) {
                geo.push_back({key, {}});
                it = geo.end() - 1;
            }
            it->second.push_back(r.rec);
        }
        cudaStream_t st = S->slots[slot];
        const ull batch_id = S->launched_batches + 1;
        lk.unlock();
        ley_status s = LEY_OK;
        // The batch's device interval: from a timing event recorded on its
        // slot stream before its first launch to its completion event.
        cudaEvent_t ev0 = nullptr;
        if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventRecord(ev0, st) != cudaSuccess) {
            cudaGetLastError();
            s = LEY_ECUDA;
        }
        for (auto& g : geo)
            if (s == LEY_OK)
                s = ley_sort_records_batch(g.second.data(), (uint32_t)g.second.size(), g.first.first,
                                           g.first.second, 0, st);
        if (s == LEY_OK && !pq.empty())
            s = ley_sort_keys_index_batch(pq.data(), (uint32_t)pq.size(), 0, st);
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess) {
            cudaGetLastError();
            if (s == LEY_OK) s = LEY_ECUDA;
        }
        lk.lock();
        if (s != LEY_OK) {  // nothing (more) in flight for this batch
            if (ev) cudaEventSynchronize(ev);
            if (ev) cudaEventDestroy(ev);
            if (ev0) cudaEventDestroy(ev0);
            const double t = S->now();
            for (ull tk : take) {
                SrvReq& r = S->reqs[tk];
                r.status = s;
                r.t_done = t;
            }
            S->in_use -= bytes;
            S->slot_busy[slot] = false;
            S->cv_done.notify_all();
            continue;
        }
        S->launched_batches++;
        S->inflight.push_back(Batch{slot, batch_id, ev0, ev, std::move(take), bytes, t_launch});
        S->cv_done.notify_all();
    }
    S->sched_done = true;
    S->cv_done.notify_all();
}

static void completer(ley_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_done.wait(lk, [&] { return !S->inflight.empty() || S->sched_done; });
        if (S->inflight.empty()) break;  // the scheduler has exited and nothing is in flight
        Batch b = S->inflight.front();
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(b.done);
        const double t = S->now();
        ley_status st = e == cudaSuccess ? ley_last_device_status(S->slots[b.slot]) : LEY_ECUDA;
        float ms0 = 0.f, ms1 = 0.f;
        if (e == cudaSuccess && (cudaEventElapsedTime(&ms0, S->t0_ev, b.start) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms1, S->t0_ev, b.done) != cudaSuccess)) {
            cudaGetLastError();
            ms0 = ms1 = -1.f;  // not timed (reported as negative)
        }
        cudaEventDestroy(b.start);
        cudaEventDestroy(b.done);
        lk.lock();
        S->inflight.pop_front();
        for (ull tk : b.tickets) {
            SrvReq& r = S->reqs[tk];
            r.status = st;
            r.t_done = t;
            r.dev_start = ms0 * 1e-3;
            r.dev_done = ms1 * 1e-3;
            r.batch = b.id;
        }
        S->in_use -= b.bytes;
        S->slot_busy[b.slot] = false;
        S->cv_sched.notify_all();
        S->cv_done.notify_all();
    }
}

static ley_status submit(ley_server* S, SrvReq r, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return LEY_EINVAL;
    r.ticket = S->next_ticket++;
    r.bytes = request_bytes(r);
    r.t_submit = S->now();
    r.t_start = r.t_done = 0;
    r.dev_start = r.dev_done = -1;
    r.batch = 0;
    r.status = -1;
    S->reqs[r.ticket] = r;
    S->pending.push_back(r.ticket);
    if (ticket) *ticket = r.ticket;
    S->cv_sched.notify_all();
    return LEY_OK;
}

}  // namespace ley

using namespace ley;

extern "C" {

ley_status ley_server_create(ley_server** out, uint64_t mem_budget, uint32_t max_batch,
                             uint32_t slots) {
    if (!out) return LEY_EINVAL;
    *out = nullptr;
    if (mem_budget == 0 || max_batch == 0 || slots == 0 || slots > 16) return LEY_EINVAL;
    ley_server* S = new ley_server();
    cudaGetDevice(&S->device);
    S->budget = mem_budget;
    S->max_batch = max_batch;
    S->nslots = (int)slots;
    S->slots.resize(slots);
    S->slot_busy.assign(slots, false);
    for (auto& s : S->slots) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto& t : S->slots)
                if (t) cudaStreamDestroy(t);
            delete S;
            return LEY_ECUDA;
        }
    }
    if (cudaEventCreate(&S->t0_ev) != cudaSuccess || cudaEventRecord(S->t0_ev, S->slots[0]) != cudaSuccess ||
        cudaEventSynchronize(S->t0_ev) != cudaSuccess) {
        cudaGetLastError();
        if (S->t0_ev) cudaEventDestroy(S->t0_ev);
        for (auto& t : S->slots) cudaStreamDestroy(t);
        delete S;
        return LEY_ECUDA;
    }
    S->sched = std::thread(scheduler, S);
    S->compl_ = std::thread(completer, S);
    *out = S;
    return LEY_OK;
}

ley_status ley_server_submit_records(ley_server* S, const void* in, void* out, uint64_t n,
                                     uint32_t rec_bytes, uint32_t key_bytes, uint64_t* ticket) {
    if (!S) return LEY_EINVAL;
    SrvReq r{};
    r.kind = 0;
    r.rec.in = in;
    r.rec.out = out;
    r.rec.n = n;
    r.rec_bytes = rec_bytes;
    r.key_bytes = key_bytes;
    const ley_status c = check_records_request(r.rec, rec_bytes, key_bytes);
    if (c != LEY_OK) return c;
    return submit(S, r, ticket);
}

ley_status ley_server_submit_pairs(ley_server* S, const uint64_t* keys_in, const uint32_t* idx_in,
                                   uint64_t* keys_out, uint32_t* idx_out, uint64_t n,
                                   uint64_t* ticket) {
    if (!S) return LEY_EINVAL;
    SrvReq r{};
    r.kind = 1;
    r.pairs.keys_in = keys_in;
    r.pairs.idx_in = idx_in;
    r.pairs.keys_out = keys_out;
    r.pairs.idx_out = idx_out;
    r.pairs.n = n;
    r.rec_bytes = 12;
    r.key_bytes = 8;
    const ley_status c = check_pairs_request(r.pairs);
    if (c != LEY_OK) return c;
    return submit(S, r, ticket);
}

ley_status ley_server_wait(ley_server* S, uint64_t ticket, ley_server_times* times) {
    if (!S) return LEY_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return LEY_EINVAL;
    S->cv_done.wait(lk, [&] { return S->reqs[ticket].status >= 0; });
    const SrvReq& r = S->reqs[ticket];
    if (times) {
        times->submit_s = r.t_submit;
        times->start_s = r.t_start;
        times->done_s = r.t_done;
        times->dev_start_s = r.dev_start;
        times->dev_done_s = r.dev_done;
        times->batch = r.batch;
    }
    const ley_status st = (ley_status)r.status;
    S->reqs.erase(ticket);
    return st;
}

ley_status ley_server_stats(ley_server* S, ley_server_counters* c) {
    if (!S || !c) return LEY_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    c->pending = S->pending.size();
    c->inflight_batches = S->inflight.size();
    c->launched_batches = S->launched_batches;
    c->bytes_in_use = S->in_use;
    return LEY_OK;
}

ley_status ley_server_destroy(ley_server* S) {
    if (!S) return LEY_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_sched.notify_all();
        S->cv_done.notify_all();
    }
    S->sched.join();
    S->compl_.join();
    for (auto& s : S->slots) cudaStreamDestroy(s);
    if (S->t0_ev) cudaEventDestroy(S->t0_ev);
    delete S;
    return LEY_OK;
}

}  // extern "C"
